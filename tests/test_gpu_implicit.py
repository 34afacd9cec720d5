"""The implicit (backward Euler) finite-volume transport of Sec. 2 on the GPU
(cdi_set_implicit) against the oracle's implicit steps (sparse LU of the
same operator), element by element, at time steps far beyond the explicit
bound; the accounts close the mass balance; switching back gives the
explicit scheme."""
import numpy as np
import pytest

import oracle as O
from paper_2110_13055_gb300 import cdi, inputs

pytestmark = pytest.mark.gpu
Z, D = (1, -1), (1.33e-9, 2.03e-9)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


CASES = {
    "discs24x40": lambda: inputs.grain_pack((24, 40), 0.6, 2.0, 4.0, seed=61)[0],
    "spheres10x12x16": lambda: inputs.grain_pack((10, 12, 16), 0.55, 1.5, 3.0, seed=62)[0],
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [cdi.FP64, cdi.FP32_CPAIR])
def test_implicit_steps_match_oracle(case, prec):
    m = CASES[case]()
    r = O.run_case(m, flow_tol=0.0, max_flow_steps=800, U_target=1e-4, applied_V=0.8,
                   lambda_D=1.5e-7, n_np_steps=0)
    dt = 30 * r["dt"]                      # 30 times the explicit bound
    n = 40
    Co, Go, Io, Oo = O.np_implicit_run(m, r["u"], r["psi"], Z, D, c0=10.0, dt=dt, n_steps=n)
    with cdi.Domain(m, precision=prec) as d:
        d.solve_flow(tol=0.0, max_steps=800, U_target=1e-4)
        d.set_potential(0.8, c_bulk=10.0, lambda_D=1.5e-7, tol=1e-13)
        d.init_transport(Z, D, c0=10.0, Ka=1e-6, dt=dt)
        d.set_implicit(1e-14, 2000)
        d.step(n)
        C = d.C()
        M, G, I, Ou = d.mass_balance()
    tol = 1e-9 if prec == cdi.FP64 else 1e-5
    assert C.min() >= 0.0
    assert rel(C, Co) < tol
    np.testing.assert_allclose(G, Go, rtol=tol)
    np.testing.assert_allclose(I, Io, rtol=tol)
    np.testing.assert_allclose(Ou, Oo, rtol=tol, atol=tol * np.abs(Io).max())
    M0 = 10.0 * (m == 0).sum() * 1e-7 ** m.ndim
    np.testing.assert_allclose(M + G + Ou - I, M0, rtol=1e-12 if prec == cdi.FP64 else 1e-7)


def test_switching_back_gives_the_explicit_scheme():
    m = CASES["discs24x40"]()

    def run(implicit_first):
        with cdi.Domain(m, precision=cdi.FP64) as d:
            d.solve_flow(tol=0.0, max_steps=400, U_target=1e-4)
            d.set_potential(0.8, c_bulk=10.0, lambda_D=1.5e-7, tol=1e-13)
            d.init_transport(Z, D, c0=10.0, Ka=1e-6)
            if implicit_first:
                d.set_implicit(1e-13)
                d.set_implicit(0.0)
            d.step(100)
            return d.C(), d.adsorbed()

    a, b = run(False), run(True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_implicit_limits():
    m = CASES["discs24x40"]()
    with cdi.Domain(m) as d:
        d.solve_flow(tol=0.0, max_steps=200, U_target=1e-4)
        d.set_potential(0.8, c_bulk=10.0, lambda_D=1.5e-7)
        dt = d.init_transport(Z, D, c0=10.0, Ka=1e-6, dt=0.0)
        d.init_transport(Z, D, c0=10.0, Ka=1e-6, dt=1000 * dt)
        with pytest.raises(cdi.CDIError) as e:
            d.set_implicit(1e-12, 0)
        assert e.value.status == 1
        d.set_implicit(1e-30, 3)           # unreachable tolerance, 3 iterations
        with pytest.raises(cdi.CDIError) as e:
            d.step(1)
        assert e.value.status == 4
