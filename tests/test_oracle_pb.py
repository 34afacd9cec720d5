"""Pins for the oracle's nonlinear Poisson-Boltzmann potential (Eq. 4 with
the Boltzmann charge of Eq. 9-10): its face rules against the pinned C
potential solver, its small-potential limit, and the Gouy-Chapman profile of
Eq. 10 at second order in the cell size."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

import oracle as O
from paper_2110_13055_gb300.inputs import grain_pack

GOLD = os.path.join(os.path.dirname(__file__), "golden", "v2_half_channel.json")


def row(n_pore):
    """1D row along x: the inlet feed one cell before cell 0, a solid face
    half a cell beyond the last pore cell."""
    m = np.zeros((1, n_pore + 1), np.uint8)
    m[0, -1] = 1
    return m


@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("dim", [2, 3])
def test_face_rules_equal_the_c_solver(dim, walls):
    """The sparse face rules, solved linearly, give the C oracle's screened
    and Laplace fields (the C solver is pinned by closed forms)."""
    shape = (20, 28) if dim == 2 else (9, 10, 12)
    m, _ = grain_pack(shape, 0.6, 1.5, 3.0, seed=7)
    A0, b, cells = O.psi_operator(m, -0.4, lateral_walls=walls)
    for mode, kdx2 in [("laplace", 0.0), ("debye", 0.7)]:
        lam = 1e-7 / np.sqrt(kdx2) if kdx2 else None
        ref, *_ = O.psi(m, -0.4, dx=1e-7, mode=mode, lambda_D=lam, lateral_walls=walls,
                        tol=1e-15)
        x = spl.spsolve((A0 + kdx2 * sp.identity(A0.shape[0])).tocsc(), b)
        np.testing.assert_allclose(x, ref.reshape(-1)[cells], rtol=1e-10, atol=1e-14)


def test_small_potential_is_debye_hueckel():
    """sinh(x) = x + x^3/6 + ...: at |psi_s| = 1e-5 V (4e-4 V_T) the nonlinear
    field equals the linearised (Debye-Hueckel) one to 1e-7 relative."""
    m, _ = grain_pack((24, 30), 0.6, 1.5, 3.0, seed=8)
    lam = 1.5e-7
    pb, it, rel = O.psi_pb(m, -1e-5, dx=1e-7, lambda_D=lam, tol=1e-14)
    dh, *_ = O.psi(m, -1e-5, dx=1e-7, lambda_D=lam, tol=1e-15)
    assert rel < 1e-14 and it <= 4
    assert np.max(np.abs(pb - dh)) < 1e-7 * 1e-5


@pytest.mark.parametrize("psi_s,hs", [(-0.1, (0.04, 0.02, 0.01)),
                                      (-0.2, (0.01, 0.005, 0.0025))])
def test_row_converges_to_gouy_chapman(psi_s, hs):
    """Resolving the Debye length, the wall field converges to Eq. 10,
    phi = 4 artanh(tanh(phi_s / 4) exp(-y / lambda)), at second order in dx,
    for wall potentials of 3.9 and 7.8 V_T (far beyond the linear regime; the
    steeper profile of the higher potential needs finer cells to reach the
    asymptotic order)."""
    lam, W = 1.0, 10.0
    vt = O.thermal_voltage()
    errs = []
    for h in hs:
        n = int(round(W / h))
        ps, it, rel = O.psi_pb(row(n), psi_s, dx=h, lambda_D=lam, tol=1e-13)
        assert rel < 1e-13
        y = (n - 1 - np.arange(n)) * h + h / 2       # distance from the wall
        eq10 = 4 * vt * np.arctanh(np.tanh(psi_s / (4 * vt)) * np.exp(-y / lam))
        near = y < 5 * lam
        errs.append(np.max(np.abs(ps[0, :n][near] - eq10[near])) / abs(psi_s))
    assert 3.3 < errs[0] / errs[1] < 4.7 and 3.3 < errs[1] / errs[2] < 4.7, errs
    assert errs[-1] < 2e-4


def test_v2_half_channel_matches_eq10_closer_than_the_linearisation():
    """Sec. 3's half channel (1 um, 1e-2 mol/m^3, -10 mV), resolved at 2 nm:
    the nonlinear field matches Eq. 10 to the discretisation error, well
    inside the linearisation gap the screened field shows."""
    gold = json.load(open(GOLD))
    W, c, psi0 = gold["width_m"], gold["c_inf_molm3"], gold["psi_wall_V"]
    vt = gold["k_B_JK"] * O.T_DEFAULT / gold["e_C"]
    lam = O.debye_length(c)
    h = 2e-9
    n = int(round(W / h))
    pb, *_ = O.psi_pb(row(n), psi0, dx=h, c_bulk=c, tol=1e-13)
    dh, *_ = O.psi(row(n), psi0, dx=h, c_bulk=c, tol=1e-14)
    y = (n - 1 - np.arange(n)) * h + h / 2
    eq10 = 4 * vt * np.arctanh(np.tanh(psi0 / (4 * vt)) * np.exp(-y / lam))
    near = y < 3 * lam
    e_pb = np.max(np.abs(pb[0, :n][near] - eq10[near])) / abs(psi0)
    e_dh = np.max(np.abs(dh[0, :n][near] - eq10[near])) / abs(psi0)
    assert e_pb < 1e-4 and e_pb < e_dh / 20, (e_pb, e_dh)


def test_sign_symmetry_and_bounds():
    """The equation is odd in psi: psi(-psi_s) = -psi(psi_s); the field lies
    between psi_s and 0 (maximum principle) and is 0 in solid cells."""
    m, _ = grain_pack((18, 26), 0.6, 1.5, 3.0, seed=9)
    a, *_ = O.psi_pb(m, -0.5, dx=1e-7, lambda_D=1e-7, tol=1e-13)
    b, *_ = O.psi_pb(m, 0.5, dx=1e-7, lambda_D=1e-7, tol=1e-13)
    np.testing.assert_allclose(a, -b, rtol=0, atol=1e-15)
    assert np.all(a[m == 1] == 0) and a.min() >= -0.5 and a.max() <= 0.0


def test_first_newton_step_is_the_screened_field():
    """At psi = 0 the Jacobian is A0 + kdx2 and the right-hand side b: one
    Newton step gives exactly the Debye-Hueckel field of the C solver."""
    m, _ = grain_pack((20, 26), 0.6, 1.5, 3.0, seed=10)
    one, it, _ = O.psi_pb(m, -0.8, dx=1e-7, lambda_D=1.5e-7, max_newton=1)
    dh, *_ = O.psi(m, -0.8, dx=1e-7, lambda_D=1.5e-7, tol=1e-15)
    assert it == 1
    np.testing.assert_allclose(one, dh, rtol=1e-10, atol=1e-14)
