"""Coupled Poisson-Nernst-Planck on the GPU (cdi_set_coupling, Eq. 3-5)
against the coupled oracle, element by element, and Sec. 3's half-channel
validation (Eq. 9-10) reached by the GPU path itself."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2110_13055_gb300 import cdi, inputs

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "v2_half_channel.json")
Z, D = (1, -1), (1.33e-9, 2.03e-9)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def half_channel(n):
    gold = json.load(open(GOLD))
    W, c, psi0 = gold["width_m"], gold["c_inf_molm3"], gold["psi_wall_V"]
    vt = gold["k_B_JK"] * O.T_DEFAULT / gold["e_C"]
    h = W / n
    m = np.zeros((1, n + 1), np.uint8)
    m[0, -1] = 1
    y = (n - 1 - np.arange(n)) * h + h / 2
    eq10 = 4 * vt * np.arctanh(np.tanh(psi0 / (4 * vt)) * np.exp(-y / O.debye_length(c)))
    pf = np.zeros(m.shape)
    pf[0, :n] = eq10
    dt = 0.5 * O.np_dt(m, np.zeros((2,) + m.shape), pf, Z, D, dx=h, Ka=0.0)
    return m, h, c, psi0, dt, eq10, vt


def gpu_coupled(m, h, c, psi0, dt, K, steps, prec):
    with cdi.Domain(m, dx=h, precision=prec) as d:
        d.solve_flow(tol=0.0, max_steps=0, U_target=0.0)
        d.set_potential(-psi0, tol=1e-13)
        d.init_transport(Z, D, c0=c, Ka=0.0, dt=dt)
        d.set_coupling(K)
        d.step(steps)
        return d.C(), d.psi(), d.adsorbed()


@pytest.mark.parametrize("prec,tol", [(cdi.FP64, 1e-9), (cdi.FP32, 1e-4)])
def test_coupled_half_channel_matches_oracle(prec, tol):
    """Concentrations at the parity bars.  The coupled potential is solved
    (in FP64) from the charge F (C_Na - C_Cl) of Eq. 5, a difference of two
    nearly equal FP32 concentrations away from the wall: its error is the
    concentrations' absolute error divided by |C_Na - C_Cl|, i.e. their
    relative error amplified by c / |C_Na - C_Cl|.  In this channel the
    charge sits in the resolved double layer, where |C_Na - C_Cl| is of the
    order of c, so the amplification is of order one: psi is held to twice
    the FP32 concentration bar of 1e-4, 2e-4 (measured in FP32: 7.9e-5; FP64:
    1e-9)."""
    m, h, c, psi0, dt, eq10, vt = half_channel(50)
    K, steps = 10, 3001
    C, ps, _ = gpu_coupled(m, h, c, psi0, dt, K, steps, prec)
    Co, _, _, _, pso = O.pnp_run(m, np.zeros((2,) + m.shape), Z, D, c0=c, dt=dt,
                                 n_steps=steps, K=K, psi_s=psi0, dx=h, Ka=0.0)
    assert rel(C, Co) < tol
    assert rel(ps, pso) < (1e-9 if prec == cdi.FP64 else 2e-4)


def test_coupled_2d_pack_with_flow_matches_oracle():
    m, _ = inputs.grain_pack((12, 20), 0.6, 1.5, 3.0, seed=5)
    dx, c, psi_s, Ka, K, steps = 2e-8, 1e-2, -0.02, 1e-5, 7, 400
    with cdi.Domain(m, dx=dx, precision=cdi.FP64) as d:
        d.solve_flow(tol=0.0, max_steps=2000, U_target=1e-4)
        u = d.u()
        pf0, _, _ = O.psi(m, psi_s, dx=dx, mode="laplace")
        dt = 0.5 * O.np_dt(m, u, pf0, Z, D, dx=dx, Ka=Ka)
        d.set_potential(-psi_s, tol=1e-13, mode="laplace")
        d.init_transport(Z, D, c0=c, Ka=Ka, dt=dt)
        d.set_coupling(K)
        d.step(steps)
        C, G = d.C(), d.adsorbed()
    Co, Go, _, _, _ = O.pnp_run(m, u, Z, D, c0=c, dt=dt, n_steps=steps, K=K, psi_s=psi_s,
                                dx=dx, Ka=Ka)
    assert rel(C, Co) < 1e-9
    np.testing.assert_allclose(G, Go, rtol=1e-9)


def test_coupled_gpu_reaches_gouy_chapman():
    """The GPU's own coupled steady state in Sec. 3's half channel is Eq. 10
    (to the discretisation error the oracle pin measures) with Eq. 9's
    Boltzmann concentrations."""
    m, h, c, psi0, dt, eq10, vt = half_channel(50)
    steps = int(round(6e-3 / dt))
    C, ps, G = gpu_coupled(m, h, c, psi0, dt, 10, steps, cdi.FP64)
    n = m.shape[1] - 1
    assert np.max(np.abs(ps[0, :n] - eq10)) / abs(psi0) < 6e-3
    for k, zk in enumerate(Z):
        np.testing.assert_allclose(C[k, 0, :n], c * np.exp(-zk * ps[0, :n] / vt), rtol=1e-8)
    assert np.all(G == 0)


def test_coupling_needs_a_potential_and_survives_checkpoint():
    m, h, c, psi0, dt, eq10, vt = half_channel(20)
    with cdi.Domain(m, dx=h) as d:
        with pytest.raises(cdi.CDIError) as e:
            d.set_coupling(5)
        assert e.value.status == 6
        d.solve_flow(tol=0.0, max_steps=0, U_target=0.0)
        d.set_potential(-psi0, tol=1e-13)
        d.init_transport(Z, D, c0=c, Ka=0.0, dt=dt)
        d.set_coupling(5)
        d.step(13)
        st = d.save_state()
        d.step(40)
        ref = d.C()
    with cdi.Domain(m, dx=h) as b:
        b.load_state(st)
        b.step(40)
        assert np.array_equal(b.C(), ref)
