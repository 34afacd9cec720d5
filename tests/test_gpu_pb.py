"""The nonlinear Poisson-Boltzmann potential (cdi_set_potential mode 2:
Eq. 4 with the Boltzmann charge of Eq. 9, Newton around the device CG)
against the oracle's Newton / sparse-LU solve, its small-potential limit, and
a transport run on the field it gives."""
import numpy as np
import pytest

import oracle as O
from paper_2110_13055_gb300 import cdi, inputs

pytestmark = pytest.mark.gpu
Z, D = (1, -1), (1.33e-9, 2.03e-9)


@pytest.fixture(scope="session", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


CASES = {
    "discs128x64": lambda: inputs.disc_pack_128x64()[0],
    "spheres19x13x11": lambda: inputs.grain_pack((11, 13, 19), 0.6, 1.5, 3.0, seed=4)[0],
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("lam", [1.5e-7, None])
def test_pb_matches_oracle(case, lam):
    """0.8 V at the surface (31 V_T): with a Debye length of 1.5 cells the
    field is far from the linear regime; with the default 10 mol/m^3
    (lambda_D = 3 nm) it is screened within the first cell."""
    m = CASES[case]()
    ref, steps, rr = O.psi_pb(m, -0.8, dx=1e-7, c_bulk=10.0, lambda_D=lam, tol=1e-13)
    assert rr < 1e-13 and steps > 1
    with cdi.Domain(m) as d:
        d.solve_flow(tol=0.0, max_steps=0, U_target=0.0)
        it, res = d.set_potential(0.8, c_bulk=10.0, lambda_D=lam or 0.0, mode="pb", tol=1e-13)
        ps = d.psi()
    assert res < 1e-13
    assert rel(ps, ref) < 1e-10
    assert np.all(ps[m == 1] == 0.0)


def test_pb_small_potential_is_the_screened_field():
    """At 1e-5 V the nonlinear and the Debye-Hueckel fields agree to 1e-7."""
    m = CASES["discs128x64"]()
    with cdi.Domain(m) as d:
        d.solve_flow(tol=0.0, max_steps=0, U_target=0.0)
        d.set_potential(1e-5, lambda_D=1.5e-7, mode="pb", tol=1e-13)
        pb = d.psi()
        d.set_potential(1e-5, lambda_D=1.5e-7, mode="debye", tol=1e-14)
        dh = d.psi()
    assert np.max(np.abs(pb - dh)) < 1e-7 * 1e-5


@pytest.mark.parametrize("prec", [cdi.FP64, cdi.FP32_CPAIR])
def test_transport_on_the_pb_field(prec):
    """200 transport steps without flow on the nonlinear field equal the
    oracle's steps on the oracle's field (FP64 1e-11; pair concentrations at
    the FP32 bars)."""
    m = CASES["discs128x64"]()
    with cdi.Domain(m, precision=prec) as d:
        d.solve_flow(tol=0.0, max_steps=0, U_target=0.0)
        d.set_potential(0.8, c_bulk=10.0, lambda_D=2e-7, mode="pb", tol=1e-13)
        dt = d.init_transport(Z, D, c0=10.0, Ka=1e-6)
        d.step(200)
        C = d.C()
        G = d.adsorbed()
    ps, *_ = O.psi_pb(m, -0.8, c_bulk=10.0, lambda_D=2e-7, tol=1e-13)
    u0 = np.zeros((2,) + m.shape)
    dt_ref = O.np_dt(m, u0, ps, Z, D)
    assert abs(dt - dt_ref) < 1e-12 * dt_ref
    Cr, Gr, _, _ = O.np_run(m, u0, ps, Z, D, c0=10.0, dt=dt_ref, n_steps=200)
    tol_c, tol_g = (1e-11, 1e-11) if prec == cdi.FP64 else (1e-4, 1e-6)
    assert rel(C, Cr) < tol_c
    assert np.max(np.abs(G - Gr) / np.abs(Gr)) < tol_g
