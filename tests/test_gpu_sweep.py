"""Batched transport sweep (cdi_sweep_transport): every member of a fused
sweep gives the single run's result bit for bit, and a member agrees with
the oracle at the parity tolerances."""
import numpy as np
import pytest

import oracle as O
from paper_2110_13055_gb300 import cdi, inputs

pytestmark = pytest.mark.gpu

Z, D = (1, -1), (1.33e-9, 2.03e-9)
COMBOS = [(1e-4, 1.0), (3e-4, 1.0), (1e-4, 0.6), (0.0, 0.2), (1e-3, 0.6)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def single_runs(d, combos, lam, c0, Ka, n_steps):
    gam, cout, dts = [], [], []
    for U, V in combos:
        d.set_velocity(U)
        d.set_potential(V, c_bulk=c0, lambda_D=lam, tol=1e-12)
        dts.append(d.init_transport(Z, D, c0=c0, Ka=Ka))
        d.step(n_steps)
        gam.append(d.adsorbed())
        cout.append(d.outlet())
    return np.array(gam), np.array(cout), np.array(dts)


@pytest.mark.parametrize("prec", [cdi.FP64, cdi.FP32, cdi.FP32_CPAIR])
@pytest.mark.parametrize("shape", [(23, 37), (9, 11, 17)])
def test_sweep_members_equal_single_runs(prec, shape):
    m, _ = inputs.grain_pack(shape, 0.6, 1.5, 4.0, seed=21)
    lam, c0, Ka, n = 1.5e-7, 10.0, 1e-6, 131   # 131 = 2 graphs of 64 + 3 single steps
    with cdi.Domain(m, precision=prec) as d:
        d.solve_flow(tol=0.0, max_steps=600, U_target=1e-4)
        g_sw, c_sw, dt_sw = d.sweep(COMBOS, lambda_D=lam, c0=c0, Ka=Ka, n_steps=n)
        with pytest.raises(cdi.CDIError) as e:   # the sweep leaves no transport state
            d.step(1)
        assert e.value.status == 6
        g1, c1, dt1 = single_runs(d, COMBOS, lam, c0, Ka, n)
    assert np.array_equal(dt_sw, dt1)
    assert np.array_equal(g_sw, g1)
    assert np.array_equal(c_sw, c1)


def test_sweep_member_against_oracle():
    m, _ = inputs.grain_pack((23, 37), 0.6, 1.5, 4.0, seed=21)
    with cdi.Domain(m, precision=cdi.FP64) as d:
        d.solve_flow(tol=0.0, max_steps=600, U_target=1e-4)
        g_sw, c_sw, dt_sw = d.sweep([(2e-4, 0.8), (5e-5, 0.4)], lambda_D=1.5e-7, c0=10.0,
                                    n_steps=300)
    for i, (U, V) in enumerate([(2e-4, 0.8), (5e-5, 0.4)]):
        r = O.run_case(m, flow_tol=0.0, max_flow_steps=600, U_target=U, applied_V=V,
                       lambda_D=1.5e-7, n_np_steps=300)
        assert abs(dt_sw[i] - r["dt"]) <= 1e-11 * r["dt"]
        np.testing.assert_allclose(g_sw[i], r["Gamma"], rtol=1e-11)
        np.testing.assert_allclose(c_sw[i], r["C_out"], rtol=1e-11)


def test_sweep_argument_errors():
    m, _ = inputs.grain_pack((23, 37), 0.6, 1.5, 4.0, seed=21)
    with cdi.Domain(m) as d:
        with pytest.raises(cdi.CDIError) as e:     # no flow yet
            d.sweep([(1e-4, 1.0)], n_steps=1)
        assert e.value.status == 6
        d.solve_flow(tol=0.0, max_steps=100)
        with pytest.raises(cdi.CDIError) as e:
            d.sweep([(1e-4, 1.0)], z=(1,) * 5, D=(1e-9,) * 5, n_steps=1)
        assert e.value.status == 1
        g, c, dt = d.sweep([(1e-4, 1.0)], n_steps=0)
        assert np.all(g == 0)


@pytest.mark.parametrize("prec", [cdi.FP64, cdi.FP32, cdi.FP32_CPAIR])
@pytest.mark.parametrize("dim", [2, 3])
def test_batch_over_uneven_geometries_equals_single_runs(prec, dim):
    """cdi_sweep_batch: members of several uneven geometries in one launch per
    step; every member equals its domain's single run bit for bit."""
    shapes = [(23, 37), (31, 45), (17, 70)] if dim == 2 else [(9, 11, 17), (7, 13, 21)]
    masks = [inputs.grain_pack(s, 0.6, 1.5, 4.0, seed=30 + i)[0] for i, s in enumerate(shapes)]
    combos = COMBOS[:3]
    lam, c0, Ka, n = 1.5e-7, 10.0, 1e-6, 131
    doms = [cdi.Domain(m, precision=prec) for m in masks]
    try:
        for d in doms:
            d.solve_flow(tol=0.0, max_steps=600, U_target=1e-4)
        g_b, c_b, dt_b = cdi.batch(doms, combos, lambda_D=lam, c0=c0, Ka=Ka, n_steps=n)
        for i, d in enumerate(doms):
            g1, c1, dt1 = single_runs(d, combos, lam, c0, Ka, n)
            assert np.array_equal(dt_b[i], dt1)
            assert np.array_equal(g_b[i], g1)
            assert np.array_equal(c_b[i], c1)
    finally:
        for d in doms:
            d.close()


def test_batch_argument_errors():
    m, _ = inputs.grain_pack((23, 37), 0.6, 1.5, 4.0, seed=21)
    m3, _ = inputs.grain_pack((9, 11, 17), 0.6, 1.5, 4.0, seed=21)
    with cdi.Domain(m) as a, cdi.Domain(m) as b, cdi.Domain(m3) as c:
        with pytest.raises(cdi.CDIError) as e:       # no solved flow
            cdi.batch([a, b], COMBOS[:1], n_steps=1)
        assert e.value.status == 6
        a.solve_flow(tol=0.0, max_steps=200)
        c.solve_flow(tol=0.0, max_steps=200)
        with pytest.raises(cdi.CDIError) as e:       # mixed dimensions
            cdi.batch([a, c], COMBOS[:1], n_steps=1)
        assert e.value.status == 1
        with pytest.raises(cdi.CDIError) as e:       # the same domain twice
            cdi.batch([a, a], COMBOS[:1], n_steps=1)
        assert e.value.status == 1


@pytest.mark.parametrize("prec,dim", [(cdi.FP64, 2), (cdi.FP32_SPLIT, 2), (cdi.FP32, 3),
                                      (cdi.FP32_CPAIR, 3)])
def test_flow_batch_members_equal_single_solves(prec, dim):
    """cdi_solve_flow_batch: uneven geometries advance in one launch per
    step and leave the batch at their own first converged check; each
    member's step count, residual and velocity field equal its own
    cdi_solve_flow bit for bit."""
    shapes = [(23, 37), (31, 45), (17, 70)] if dim == 2 else [(9, 11, 17), (7, 13, 21)]
    masks = [inputs.grain_pack(s, 0.6, 1.5, 4.0, seed=50 + i)[0] for i, s in enumerate(shapes)]
    tol = 1e-7
    single = []
    for m in masks:
        with cdi.Domain(m, precision=prec) as d:
            st, r, _ = d.solve_flow(tol=tol, max_steps=200_000, U_target=1e-4)
            single.append((st, r, d.u_lattice(), d.u()))
    doms = [cdi.Domain(m, precision=prec) for m in masks]
    try:
        steps, res, status = cdi.flow_batch(doms, tol=tol, max_steps=200_000, U_target=1e-4)
        assert list(status) == [0] * len(doms)
        assert len(set(steps)) > 1          # the members stop at different checks
        for i, d in enumerate(doms):
            assert steps[i] == single[i][0]
            assert res[i] == single[i][1]
            assert np.array_equal(d.u_lattice(), single[i][2])
            assert np.array_equal(d.u(), single[i][3])
        # the transport that follows runs on the batched flows
        g_b, c_b, _ = cdi.batch(doms, COMBOS[:2], n_steps=40)
        assert np.all(np.isfinite(g_b)) and np.all(g_b > 0)
    finally:
        for d in doms:
            d.close()


def test_flow_batch_limits_and_errors():
    m, _ = inputs.grain_pack((23, 37), 0.6, 1.5, 4.0, seed=21)
    m3, _ = inputs.grain_pack((9, 11, 17), 0.6, 1.5, 4.0, seed=21)
    with cdi.Domain(m) as a, cdi.Domain(m) as b, cdi.Domain(m3) as c:
        with pytest.raises(cdi.CDIError) as e:       # mixed dimensions
            cdi.flow_batch([a, c], max_steps=100)
        assert e.value.status == 1
        with pytest.raises(cdi.CDIError) as e:       # the same domain twice
            cdi.flow_batch([a, a], max_steps=100)
        assert e.value.status == 1
        steps, res, st = cdi.flow_batch([a, b], tol=1e-30, max_steps=300,
                                        allow_not_converged=True)
        assert list(steps) == [300, 300] and list(st) == [4, 4]
        steps, res, st = cdi.flow_batch([a, b], tol=0.0, max_steps=200)
        assert list(steps) == [200, 200] and list(st) == [0, 0]
        a.set_potential(1.0)
        a.init_transport()
        a.step(5)
