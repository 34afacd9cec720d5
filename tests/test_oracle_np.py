"""Pins for the oracle's explicit finite-volume Nernst-Planck update (Eq. 3)
with the adsorption flux of Eq. 6, against closed forms, the paper's
electromigration validation (Sec. 3, Eq. 9-10) and exact invariants."""
import json
import os

import numpy as np
import pytest
from scipy.special import erfc

import oracle as O
from paper_2110_13055_gb300.inputs import grain_pack

GOLD = os.path.join(os.path.dirname(__file__), "golden", "v2_half_channel.json")
VT = O.thermal_voltage()


def row(n_pore):
    """n_pore pore cells along x then one solid cell; the inlet feed ghost
    sits before cell 0."""
    m = np.zeros((1, n_pore + 1), np.uint8)
    m[0, -1] = 1
    return m


def test_uniform_state_is_preserved():
    """With no flow, no potential and no adsorption, C = c0 everywhere is a
    fixed point of the update (inlet feed at c0, zero-gradient outlet)."""
    m, _ = grain_pack((20, 30), 0.6, 2.0, 4.0, seed=7)
    u = np.zeros((2,) + m.shape)
    ps = np.zeros(m.shape)
    C, G, I, Ou = O.np_run(m, u, ps, [1, -1], [1.33e-9, 2.03e-9], c0=10.0,
                           dt=1e-6, n_steps=50, Ka=0.0)
    assert np.all(C[:, m == 0] == 10.0)
    assert np.all(G == 0) and np.all(I == 0) and np.all(Ou == 0)


def _steady(m, u, ps, z, D, c0, Ka, dx, n_steps, C=None, dt=None):
    if dt is None:
        dt = O.np_dt(m, u, ps, z, D, dx=dx, Ka=Ka)
    return O.np_run(m, u, ps, z, D, c0=c0, dt=dt, n_steps=n_steps, dx=dx, Ka=Ka, C=C)


def test_boltzmann_distribution_v2():
    """Sec. 3 validation: half channel of 1 um, psi from Eq. 10 with
    psi_0 = -10 mV at the wall, 1e-2 mol/m^3 and psi = 0 at the centreline
    (the feed ghost), no flux at the wall.  The steady state of the scheme is
    the Boltzmann distribution of Eq. 9 at the cell centres, for both ions."""
    gold = json.load(open(GOLD))
    W, c, psi0 = gold["width_m"], gold["c_inf_molm3"], gold["psi_wall_V"]
    vt = gold["k_B_JK"] * O.T_DEFAULT / gold["e_C"]
    lam = O.debye_length(c)
    n = 50
    h = W / n
    m = row(n)
    y = (n - 1 - np.arange(n)) * h + h / 2               # distance from the wall
    ps = np.zeros(m.shape)
    ps[0, :n] = 4 * vt * np.arctanh(np.tanh(psi0 / (4 * vt)) * np.exp(-y / lam))
    u = np.zeros((2,) + m.shape)
    D = [1.33e-9, 2.03e-9]
    C, G, I, Ou = _steady(m, u, ps, [1, -1], D, c, 0.0, h, 150000)
    eq9 = np.stack([c * np.exp(-zk * ps[0, :n] / vt) for zk in (1, -1)])
    for k in range(2):
        np.testing.assert_allclose(C[k, 0, :n], eq9[k], rtol=1e-9)
    assert np.all(G == 0)
    # and Eq. 9 is a fixed point of a single step, to roundoff
    Cb = np.zeros((2,) + m.shape)
    Cb[:, 0, :n] = eq9
    C1, *_ = _steady(m, u, ps, [1, -1], D, c, 0.0, h, 1, C=Cb)
    np.testing.assert_allclose(C1[:, 0, :n], eq9, rtol=1e-14)


@pytest.mark.parametrize("U,E", [(0.0, 0.0), (1e-3, 0.0), (-5e-4, 0.0),
                                 (0.0, 0.02), (4e-4, -0.01)])
def test_row_steady_state_closed_form(U, E):
    """Row with the feed at c0 on the left and an adsorbing solid face on the
    right, uniform velocity U and a uniform field (psi_j = E (j+1)).  At
    steady state every face carries the same flux, the profile is
    C_j = a + b exp(P (j+1)) with P = U dx/D - z E / V_T (exponential
    fitting is nodally exact), C_{-1} = c0, and the last cell obeys Eq. 6
    closed over half a cell: J = K_eff C_m with K_eff = Ka / (1 + Ka dx/(2D))."""
    n, dx, c0, Ka = 20, 1e-7, 10.0, 1e-4
    m = row(n)
    u = np.zeros((2,) + m.shape)
    u[0, 0, :n] = U
    ps = np.zeros(m.shape)
    ps[0, :n] = E * (np.arange(n) + 1)
    D = [1e-9, 1.5e-9]
    z = [1, -1]
    C, G, I, Ou = _steady(m, u, ps, z, D, c0, Ka, dx, 120000)
    j = np.arange(n)
    last = n - 1
    for k in range(2):
        Keff = Ka / (1 + Ka * dx / (2 * D[k]))
        P = U * dx / D[k] - z[k] * E / VT
        if P == 0.0:
            # linear profile: C_j = c0 + s (j+1), flux -D s / dx = K_eff C_last
            s = -Keff * c0 / (D[k] / dx + Keff * (last + 1))
            expect = c0 + s * (j + 1)
        else:
            q = np.exp(P * (last + 1))
            a = Keff * c0 * q / (D[k] * P / dx + Keff * (q - 1))
            b = c0 - a
            expect = a + b * np.exp(P * (j + 1))
        np.testing.assert_allclose(C[k, 0, :n], expect, rtol=1e-10)


def test_diffusion_transient_matches_erfc_at_second_order():
    """u = 0, psi = 0: a feed at c0 diffusing into an empty semi-infinite
    row follows c0 erfc(x / (2 sqrt(D t))), x measured from the feed-cell
    centre; halving dx (with dt ~ dx^2) cuts the error about fourfold."""
    D, c0, T_end, Lx = 1e-9, 1.0, 4e-6, 2e-6
    errs = []
    for n in (40, 80, 160):
        dx = Lx / n
        m = np.zeros((1, n), np.uint8)          # long row, far end untouched
        u = np.zeros((2, 1, n))
        ps = np.zeros((1, n))
        dt = 0.2 * dx * dx / D
        steps = int(round(T_end / dt))
        dt = T_end / steps
        C0 = np.zeros((1, 1, n))
        C, *_ = O.np_run(m, u, ps, [0], [D], c0=c0, dt=dt, n_steps=steps,
                         dx=dx, Ka=0.0, C=C0)
        x = (np.arange(n) + 1) * dx
        errs.append(np.max(np.abs(C[0, 0] - c0 * erfc(x / (2 * np.sqrt(D * T_end))))))
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0, errs


def _porous_case(seed=11, U=1e-4, V=1.0, lam=None):
    m, _ = grain_pack((24, 40), 0.6, 2.0, 5.0, seed=seed)
    uf, *_ = O.lbm(m, tol=0.0, check_every=50, max_steps=1500)
    u, _ = O.velocity_export(m, uf, U)
    ps, *_ = O.psi(m, -V, dx=1e-7, c_bulk=10.0, lambda_D=lam)
    return m, u, ps


def test_mass_balance_is_exact():
    """Dissolved + adsorbed + outflow - inflow is conserved to roundoff: the
    conservative update moves every face flux between two cells or into one
    of the Gamma/In/Out accounts (Eq. 3 in divergence form with Eq. 6)."""
    m, u, ps = _porous_case(lam=1.5e-7)
    z, D, dx, c0 = [1, -1], [1.33e-9, 2.03e-9], 1e-7, 10.0
    dt = O.np_dt(m, u, ps, z, D, dx=dx, Ka=1e-4)
    C0 = np.where(m[None] == 0, c0, 0.0) * np.ones((2,) + m.shape)
    M0 = O.mass(m, C0, dx)
    C, G, I, Ou = O.np_run(m, u, ps, z, D, c0=c0, dt=dt, n_steps=400, dx=dx, Ka=1e-4)
    M = O.mass(m, C, dx)
    assert np.all(G > 0) and np.all(I != 0) and np.all(Ou > 0)
    np.testing.assert_allclose(M + G + Ou - I, M0, rtol=1e-13)


def test_positivity_at_the_bound():
    """With dt at the explicit bound (safety 1) every update coefficient is
    non-negative, so a non-negative state stays non-negative even under a
    strong field."""
    m, u, ps = _porous_case(U=1e-3, V=1.2, lam=1e-7)
    z, D = [1, -1], [1.33e-9, 2.03e-9]
    dt = O.np_dt(m, u, ps, z, D, Ka=1e-3, safety=1.0)
    rs = np.random.default_rng(0)
    Cinit = rs.random((2,) + m.shape) * (m[None] == 0)
    Cinit[:, 3:6, :] = 0.0
    C, *_ = O.np_run(m, u, ps, z, D, c0=0.0, dt=dt, n_steps=200, Ka=1e-3, C=Cinit)
    assert C.min() >= 0.0
    # beyond the bound positivity is lost for some state
    C2, *_ = O.np_run(m, u, ps, z, D, c0=0.0, dt=3.0 * dt, n_steps=30, Ka=1e-3, C=Cinit)
    assert C2.min() < 0.0


def test_outputs():
    """Outlet concentration is flux weighted (uniform C gives c0), salt
    removal follows Sec. 4.1, column means average pore cells only."""
    m = np.zeros((4, 6), np.uint8)
    m[1, 2] = 1
    u = np.zeros((2, 4, 6))
    u[0, :, -1] = [1.0, 2.0, 3.0, 4.0]
    C = np.full((1, 4, 6), 3.0)
    C[0, :, -1] = [1.0, 1.0, 1.0, 5.0]
    assert O.outlet_concentration(m, u, C)[0] == pytest.approx((1 + 2 + 3 + 20) / 10)
    assert O.salt_removal(10.0, 2.5) == pytest.approx(0.75)
    C[0, 0, 2] = 7.0
    cm = O.column_means(m, C)
    assert cm[0, 2] == pytest.approx((7 + 3 + 3) / 3)


def test_explicit_step_is_an_m_matrix_map_and_marches_to_its_fixed_point():
    """Brute force on a tiny grid: one explicit step is the affine map
    C' = A C + b (columns from unit states, b from the empty state).  At the
    time-step bound A is non-negative (positivity), and every column sum is at
    most 1 — exactly 1 for a cell with no solid, inlet or outlet face (the
    update conserves mass).  n steps equal A^n C0 + sum_k A^k b, and a long
    run reaches the algebraic steady state (I - A)^-1 b."""
    m = np.zeros((3, 5), np.uint8)
    m[1, 2] = 1
    rng = np.random.default_rng(2)
    u = np.zeros((2,) + m.shape)
    u[0][m == 0] = 2e-4 * (1 + 0.3 * rng.random(int((m == 0).sum())))
    ps = np.zeros(m.shape)
    ps[m == 0] = 0.01 * rng.standard_normal(int((m == 0).sum()))
    z, Dk, c0, Ka, dx = [1], [1.33e-9], 1.0, 1e-5, 1e-7
    dt = O.np_dt(m, u, ps, z, Dk, dx=dx, Ka=Ka)
    pores = np.argwhere(m == 0)
    n = len(pores)

    def step(Cvec, steps=1):
        C = np.zeros((1,) + m.shape)
        for (y, x), v in zip(pores, Cvec):
            C[0, y, x] = v
        Cn, *_ = O.np_run(m, u, ps, z, Dk, c0=c0, dt=dt, n_steps=steps, dx=dx, Ka=Ka, C=C)
        return np.array([Cn[0, y, x] for (y, x) in pores])

    b = step(np.zeros(n))
    A = np.stack([step(np.eye(n)[j]) - b for j in range(n)], axis=1)
    assert np.all(A >= -1e-15)
    col = A.sum(axis=0)
    assert np.all(col <= 1 + 1e-12)
    interior = [j for j, (y, x) in enumerate(pores)
                if 0 < x < m.shape[1] - 1 and not any(
                    m[(y + dy) % m.shape[0], x + dxx] for dy, dxx in ((0, 1), (0, -1), (1, 0), (-1, 0)))]
    assert interior
    np.testing.assert_allclose(col[interior], 1.0, rtol=0, atol=1e-12)
    C0 = rng.random(n)
    ref = C0.copy()
    for _ in range(7):
        ref = A @ ref + b
    np.testing.assert_allclose(step(C0, 7), ref, rtol=1e-12, atol=1e-14)
    steady = np.linalg.solve(np.eye(n) - A, b)
    np.testing.assert_allclose(step(C0, 20000), steady, rtol=1e-9)
