"""Pins of the coupled Poisson-Nernst-Planck oracle (Eq. 3-5): the potential
re-solved from the net charge of the current concentrations.

* The Poisson solve with a charge term agrees with a dense direct solve of
  the same system on a tiny grid (brute force).
* Sec. 3's half-channel validation: with the coupling on, the steady state of
  Eq. 3-5 is the Gouy-Chapman double layer of Eq. 10 (potential) with the
  Boltzmann concentrations of Eq. 9; the discrete potential converges to
  Eq. 10 at second order in the cell size.
* Mass balance stays exact with the coupling on.
"""
import json
import os

import numpy as np

import oracle as O
from paper_2110_13055_gb300.inputs import grain_pack

GOLD = os.path.join(os.path.dirname(__file__), "golden", "v2_half_channel.json")


def test_psi_with_charge_matches_dense_solve():
    """6x5 grid with solids, periodic rows, inlet feed at 0 on the left,
    no flux at the outlet: assemble A psi = b cell by cell and solve it
    directly."""
    rng = np.random.default_rng(3)
    m = np.zeros((5, 6), np.uint8)
    m[1, 2] = m[3, 4] = m[0, 5] = 1
    src = rng.normal(size=m.shape)
    psi_s = -0.3
    ny, nx = m.shape
    idx = {(y, x): k for k, (y, x) in enumerate(zip(*np.nonzero(m == 0)))}
    A = np.zeros((len(idx), len(idx)))
    b = np.zeros(len(idx))
    for (y, x), k in idx.items():
        b[k] += src[y, x]
        for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
            X, Y = x + dx, (y + dy) % ny
            if X < 0:                       # inlet feed, psi = 0 one cell away
                A[k, k] += 1.0
            elif X >= nx:                   # outlet: no flux
                pass
            elif m[Y, X]:                   # solid face: psi_s half a cell away
                A[k, k] += 2.0
                b[k] += 2.0 * psi_s
            else:
                A[k, k] += 1.0
                A[k, idx[(Y, X)]] -= 1.0
    sol = np.linalg.solve(A, b)
    ps, it, rel = O.psi_src(m, psi_s, src, tol=1e-14)
    got = np.array([ps[y, x] for (y, x) in idx])
    np.testing.assert_allclose(got, sol, rtol=0, atol=1e-11 * np.max(np.abs(sol)))
    assert np.all(ps[m == 1] == 0.0)


def _half_channel(n):
    gold = json.load(open(GOLD))
    W, c, psi0 = gold["width_m"], gold["c_inf_molm3"], gold["psi_wall_V"]
    vt = gold["k_B_JK"] * O.T_DEFAULT / gold["e_C"]
    lam = O.debye_length(c)
    h = W / n
    m = np.zeros((1, n + 1), np.uint8)
    m[0, -1] = 1                                   # the wall after the last cell
    y = (n - 1 - np.arange(n)) * h + h / 2         # distance from the wall
    eq10 = 4 * vt * np.arctanh(np.tanh(psi0 / (4 * vt)) * np.exp(-y / lam))
    u = np.zeros((2,) + m.shape)
    D = [1.33e-9, 2.03e-9]
    pf = np.zeros(m.shape)
    pf[0, :n] = eq10
    dt = 0.5 * O.np_dt(m, u, pf, [1, -1], D, dx=h, Ka=0.0)
    steps = int(round(6e-3 / dt))                  # ~20 relaxation times of the slowest mode
    C, G, I, Ou, ps = O.pnp_run(m, u, [1, -1], D, c0=c, dt=dt, n_steps=steps, K=10,
                                psi_s=psi0, dx=h, Ka=0.0)
    return C[:, 0, :n], ps[0, :n], eq10, c, vt, psi0


def test_coupled_steady_state_is_gouy_chapman():
    """Sec. 3 (Fig. 3): the coupled steady state reproduces Eq. 10 and Eq. 9."""
    errs = []
    for n in (25, 50):
        C, ps, eq10, c, vt, psi0 = _half_channel(n)
        errs.append(np.max(np.abs(ps - eq10)) / abs(psi0))
        # Boltzmann (Eq. 9) in the computed potential: the scheme's zero-flux
        # state
        for k, zk in enumerate((1, -1)):
            np.testing.assert_allclose(C[k], c * np.exp(-zk * ps / vt), rtol=1e-9)
    assert errs[1] < 6e-3
    assert errs[0] / errs[1] > 3.0                 # second order in the cell size


def test_coupled_mass_balance_is_exact():
    m, _ = grain_pack((12, 20), 0.6, 1.5, 3.0, seed=5)
    rng = np.random.default_rng(1)
    u = np.zeros((2,) + m.shape)
    u[0][m == 0] = 1e-4 * (1 + 0.2 * rng.random(int((m == 0).sum())))
    z, D, c0, dx, Ka = [1, -1], [1.33e-9, 2.03e-9], 1e-2, 2e-8, 1e-5
    pf, _, _ = O.psi(m, -0.02, dx=dx, mode="laplace")
    dt = 0.5 * O.np_dt(m, u, pf, z, D, dx=dx, Ka=Ka)
    C, G, I, Ou, ps = O.pnp_run(m, u, z, D, c0=c0, dt=dt, n_steps=400, K=7, psi_s=-0.02,
                                dx=dx, Ka=Ka)
    vol = dx * dx
    M0 = c0 * (m == 0).sum() * vol
    M = C.sum(axis=(1, 2)) * vol
    np.testing.assert_allclose(M + G + Ou - I, M0, rtol=1e-12)
    assert np.all(C >= 0)
