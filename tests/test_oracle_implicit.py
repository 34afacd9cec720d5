"""Pins of the oracle's implicit (backward Euler) finite-volume transport, the
scheme Sec. 2 describes: it reaches the explicit scheme's steady state, it
is first order in dt against the exact time integral of the same
semi-discrete system, it conserves mass exactly with its accounts, and it
stays positive at time steps far beyond the explicit bound."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_2110_13055_gb300 import inputs

Z, D = (1, -1), (1.33e-9, 2.03e-9)


@pytest.fixture(scope="module")
def case():
    m, _ = inputs.grain_pack((10, 16), 0.6, 1.5, 3.0, seed=5)
    uf, *_ = O.lbm(m, tol=0.0, max_steps=2000)
    u, _ = O.velocity_export(m, uf, 1e-4)
    ps, *_ = O.psi(m, -0.5, lambda_D=1.5e-7)
    dt = O.np_dt(m, u, ps, Z, D)
    return m, u, ps, dt


def test_operator_reproduces_the_explicit_step(case):
    """One explicit step equals C - dt (A C - b) with the exported operator."""
    m, u, ps, dt = case
    rs = np.random.default_rng(3)
    C0 = np.where(m[None] == 0, rs.uniform(5, 15, (2,) + m.shape), 0.0)
    C1, *_ = O.np_run(m, u, ps, Z, D, c0=10.0, dt=dt, n_steps=1, C=C0)
    for k in range(2):
        A, b = O.np_operator(m, u, ps, Z[k], D[k], c0=10.0)
        want = C0[k].ravel() - dt * (A @ C0[k].ravel() - b)
        np.testing.assert_allclose(C1[k].ravel(), want, rtol=1e-13, atol=1e-12)


def test_reaches_the_explicit_steady_state():
    """Both schemes end at the algebraic steady state A C = b (a milder
    double layer, -0.1 V, so that both get there in a few seconds)."""
    m, _ = inputs.grain_pack((10, 16), 0.6, 1.5, 3.0, seed=5)
    uf, *_ = O.lbm(m, tol=0.0, max_steps=2000)
    u, _ = O.velocity_export(m, uf, 1e-4)
    ps, *_ = O.psi(m, -0.1, lambda_D=1.5e-7)
    dt = O.np_dt(m, u, ps, Z, D)
    Ce, *_ = O.np_run(m, u, ps, Z, D, c0=10.0, dt=dt, n_steps=60000)
    Ci, *_ = O.np_implicit_run(m, u, ps, Z, D, c0=10.0, dt=2000 * dt, n_steps=60)
    assert np.max(np.abs(Ci - Ce)) / np.max(Ce) < 1e-11


def test_first_order_in_dt_against_the_exact_integral(case):
    """C(t) = C* + exp(-t A)(C0 - C*), C* = A^-1 b, is the exact solution of
    the semi-discrete system both schemes discretise in time."""
    m, u, ps, dt = case
    pore = (m == 0).ravel()
    t_end = 40 * dt
    A, b = O.np_operator(m, u, ps, Z[0], D[0], c0=10.0)
    Ad = A.toarray()[np.ix_(pore, pore)]
    bd = b[pore]
    Cs = np.linalg.solve(Ad, bd)
    exact = Cs + sla.expm(-t_end * Ad) @ (10.0 - Cs)
    errs = []
    for n in (20, 40, 80):
        C, *_ = O.np_implicit_run(m, u, ps, Z[:1], D[:1], c0=10.0, dt=t_end / n, n_steps=n)
        errs.append(np.max(np.abs(C[0].ravel()[pore] - exact)))
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


def test_exact_mass_balance_and_positivity_beyond_the_explicit_bound(case):
    m, u, ps, dt = case
    C, G, I, Ou = O.np_implicit_run(m, u, ps, Z, D, c0=10.0, dt=100 * dt, n_steps=30)
    assert C.min() >= 0.0
    M = O.mass(m, C, 1e-7)
    M0 = O.mass(m, np.where(m[None] == 0, 10.0, 0.0) * np.ones((2,) + m.shape), 1e-7)
    np.testing.assert_allclose(M + G + Ou - I, M0, rtol=1e-13)
    # the explicit scheme at that time step is not positive
    Ce, *_ = O.np_run(m, u, ps, Z, D, c0=10.0, dt=100 * dt, n_steps=3)
    assert Ce.min() < 0.0
