"""Pins for the oracle's frozen potential (Eq. 4-5, Dirichlet at the solid
surface, zero potential in the feed) against closed forms."""
import json
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "v2_half_channel.json")


def row(n_pore):
    """1D row along x: n_pore pore cells followed by one solid cell.  The
    inlet feed (psi = 0) sits one cell before cell 0; the solid face half a
    cell after the last pore cell.  ny = 1 with periodic y adds no y flux."""
    m = np.zeros((1, n_pore + 1), np.uint8)
    m[0, -1] = 1
    return m


@pytest.mark.parametrize("kdx2", [0.0, 0.05, 1.0, 30.0])
def test_row_discrete_closed_form(kdx2):
    """On the row the scheme is psi_{j-1} - (2 + k) psi_j + psi_{j+1} = 0 with
    psi_{-1} = 0 and a solid face at distance dx/2 beyond the last cell m.  Its
    exact solution is psi_j = A sinh((j+1) theta), cosh(theta) = 1 + k/2
    (psi_j = A (j+1) for k = 0), A fixed by the last cell."""
    n, psi_s = 25, -0.3
    m = row(n)
    dx = 1e-7
    lam = dx / np.sqrt(kdx2) if kdx2 > 0 else None
    ps, it, rel = O.psi(m, psi_s, dx=dx, mode="laplace" if kdx2 == 0 else "debye",
                        lambda_D=lam, tol=1e-14)
    j = np.arange(n)
    last = n - 1
    if kdx2 == 0:
        A = 2 * psi_s / (2 * last + 3)
        expect = A * (j + 1)
    else:
        th = np.arccosh(1 + kdx2 / 2)
        A = 2 * psi_s / ((3 + kdx2) * np.sinh((last + 1) * th) - np.sinh(last * th))
        expect = A * np.sinh((j + 1) * th)
    np.testing.assert_allclose(ps[0, :n], expect, rtol=1e-11, atol=1e-15)
    assert ps[0, -1] == 0.0


def test_laplace_row_equals_continuum():
    """With zero charge (the electroneutral start) the 1D potential is the
    linear profile between psi = 0 at the feed-cell centre and psi_s at the
    solid surface, exactly."""
    n, psi_s = 10, -1.0
    ps, *_ = O.psi(row(n), psi_s, mode="laplace", tol=1e-14)
    x = np.arange(n) + 1.0          # distance from the feed-cell centre
    L = n + 0.5                      # distance from the feed centre to the wall
    np.testing.assert_allclose(ps[0, :n], psi_s * x / L, rtol=1e-12)


def test_screened_profile_converges_to_exponential():
    """Resolving the Debye length, the screened field of a wall converges to
    psi_s exp(-y / lambda) (the small-potential limit of Eq. 10) at second
    order in dx."""
    lam, W, psi_s = 1.0, 12.0, -1e-3
    errs = []
    for h in (0.2, 0.1, 0.05):
        n = int(round(W / h))
        m = row(n)                    # feed on the left, wall on the right
        ps, *_ = O.psi(m, psi_s, dx=h, lambda_D=lam, tol=1e-14)
        y = (n - 1 - np.arange(n)) * h + h / 2   # distance from the wall
        near = y < 4 * lam
        errs.append(np.max(np.abs(ps[0, :n][near] - psi_s * np.exp(-y[near] / lam))) / abs(psi_s))
    assert 3.3 < errs[0] / errs[1] < 4.7 and 3.3 < errs[1] / errs[2] < 4.7, errs


def test_v2_wall_potential_matches_eq10():
    """Sec. 3's half channel (1 um, 1e-2 mol/m^3, -10 mV at the wall): the
    screened field, resolved at 2 nm, matches Eq. 10 to within the
    linearisation gap of the small potential (|psi_0| < 0.4 k_B T / e)."""
    gold = json.load(open(GOLD))
    W, c, psi0 = gold["width_m"], gold["c_inf_molm3"], gold["psi_wall_V"]
    VT = gold["k_B_JK"] * O.T_DEFAULT / gold["e_C"]
    lam = O.debye_length(c)
    assert 9.0e-8 < lam < 1.0e-7
    h = 2e-9
    n = int(round(W / h))
    ps, *_ = O.psi(row(n), psi0, dx=h, c_bulk=c, tol=1e-14)
    y = (n - 1 - np.arange(n)) * h + h / 2
    eq10 = 4 * VT * np.arctanh(np.tanh(psi0 / (4 * VT)) * np.exp(-y / lam))
    near = y < 3 * lam
    err = np.max(np.abs(ps[0, :n][near] - eq10[near])) / abs(psi0)
    assert err < 1e-2


def test_solid_cells_zero_and_symmetry_2d():
    """psi is 0 in solid cells, between psi_s and 0 in the pore space, and a
    geometry symmetric about the channel axis gives a symmetric field."""
    m = np.zeros((9, 12), np.uint8)
    m[0, :] = 1
    m[-1, :] = 1
    m[4, 5:8] = 1
    ps, *_ = O.psi(m, -0.5, dx=1e-7, lambda_D=2e-7)
    assert np.all(ps[m == 1] == 0)
    assert ps.min() >= -0.5 and ps.max() <= 0.0
    np.testing.assert_allclose(ps, ps[::-1, :], rtol=0, atol=1e-14)
