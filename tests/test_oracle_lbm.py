"""Pins for the oracle's lattice Boltzmann Stokes solve (Sec. 2, Eq. 7-8).

Each test checks the oracle against something other than itself: a closed
form of the continuum or of the discrete scheme, or an exact symmetry.
"""
import numpy as np
import pytest

import oracle as O


def slit(nx, H, dim=2, nz=4):
    """Channel of H pore rows between two solid rows (walls at y = 1/2 and
    y = H + 1/2 in cell units, lateral directions periodic)."""
    if dim == 2:
        m = np.zeros((H + 2, nx), np.uint8)
        m[0, :] = 1
        m[-1, :] = 1
    else:
        m = np.zeros((nz, H + 2, nx), np.uint8)
        m[:, 0, :] = 1
        m[:, -1, :] = 1
    return m


def poiseuille(H, g, tau):
    """Body-force-driven plane Poiseuille profile of Eq. 2 with nu = (tau-1/2)/3
    (the viscosity relation of Sec. 2), evaluated at the H pore-cell centres."""
    nu = (tau - 0.5) / 3.0
    y = np.arange(H) + 0.5
    return g * y * (H - y) / (2.0 * nu)


TAU_EXACT = 0.5 + np.sqrt(3.0) / 4.0  # (tau - 1/2)^2 = 3/16


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("mirror", [False, True])
def test_poiseuille_exact_at_magic_tau(dim, mirror):
    """With BGK and halfway bounce-back the plane Poiseuille profile is
    reproduced exactly when (tau - 1/2)^2 = 3/16 (the wall sits exactly
    halfway between the last pore node and the first solid node)."""
    H, g = 12, 1e-6
    m = slit(6, H, dim)
    u, steps, res, st = O.lbm(m, mirror=mirror, tau=TAU_EXACT, force=g,
                              tol=1e-13, check_every=200, max_steps=400_000)
    assert st == 0
    ua = poiseuille(H, g, TAU_EXACT)
    ux = u[0][1:-1, 0] if dim == 2 else u[0][1, 1:-1, 0]
    assert np.max(np.abs(ux - ua)) / ua.max() < 1e-9
    # no cross flow
    assert np.max(np.abs(u[1])) < 1e-12 * ua.max()


def test_poiseuille_second_order_at_tau_one():
    """At tau = 1 the bounce-back wall error is second order: the error of
    the maximum velocity shrinks about fourfold per doubling of H."""
    errs = []
    for H in (8, 16, 32):
        m = slit(4, H)
        u, *_ = O.lbm(m, mirror=False, tau=1.0, force=1e-6, tol=1e-12,
                      check_every=200, max_steps=2_000_000)
        ua = poiseuille(H, 1e-6, 1.0)
        errs.append(np.max(np.abs(u[0][1:-1, 0] - ua)) / ua.max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, errs


@pytest.mark.parametrize("dim", [2, 3])
def test_free_acceleration(dim):
    """In a fully periodic pore space the body force adds exactly F of
    momentum per step, so u = (t + 1/2) F after t steps (the half-step shift
    of the force term)."""
    shape = (5, 7) if dim == 2 else (3, 5, 7)
    m = np.zeros(shape, np.uint8)
    g = 1e-6
    for t in (2, 10):
        u, steps, *_ = O.lbm(m, mirror=False, tau=0.8, force=g, tol=0.0,
                             check_every=2, max_steps=t)
        assert steps == t
        np.testing.assert_allclose(u[0], (t + 0.5) * g, rtol=1e-12)
        assert np.max(np.abs(u[1:])) < 1e-20


@pytest.mark.parametrize("dim", [2, 3])
def test_mirror_reflection_symmetry(dim):
    """The doubled (mirrored) pore space is symmetric under x -> 2nx-1-x.  A
    Stokes flow driven along x then satisfies u_x(Rx) = u_x(x) and
    u_y(Rx) = -u_y(x) (reflection plus linearity), at every step."""
    from paper_2110_13055_gb300.inputs import grain_pack
    shape = (24, 20) if dim == 2 else (10, 12, 14)
    m, _ = grain_pack(shape, 0.65, 2.5, 3.5, seed=5)
    u, *_ = O.lbm(m, mirror=True, tau=1.0, force=1e-6, tol=0.0,
                  check_every=10, max_steps=300)
    R = u[..., ::-1]
    np.testing.assert_allclose(R[0], u[0], rtol=0, atol=1e-14 * np.abs(u[0]).max())
    for a in range(1, dim):
        np.testing.assert_allclose(R[a], -u[a], rtol=0, atol=1e-14 * np.abs(u[0]).max())


def test_solid_cells_carry_no_flow_and_flow_is_linear():
    """u = 0 in solid cells; the Stokes-linear scheme scales exactly with the
    force (Eq. 2 is linear)."""
    from paper_2110_13055_gb300.inputs import grain_pack
    m, _ = grain_pack((16, 24), 0.6, 2.0, 4.0, seed=3)
    u1, *_ = O.lbm(m, mirror=True, force=1e-6, tol=0.0, check_every=20, max_steps=400)
    u2, *_ = O.lbm(m, mirror=True, force=2e-6, tol=0.0, check_every=20, max_steps=400)
    flow_mask = np.concatenate([m, m[:, ::-1]], axis=1)
    assert np.all(u1[:, flow_mask == 1] == 0.0)
    np.testing.assert_allclose(u2, 2.0 * u1, rtol=1e-12, atol=1e-24)


@pytest.mark.parametrize("dim,tau", [(2, 1.0), (2, 0.8), (3, 0.9)])
def test_permeability_tensor_is_symmetric(dim, tau):
    """Onsager reciprocity of Stokes flow: on a doubly periodic porous image
    the mean flow across the force equals the mean flow along it when the
    force is turned across (K_xy = K_yx).  Forcing along y is forcing along x
    on the image with x and y swapped, so K_yx is the mean u_y of the image
    and K_xy the mean u_y of the swapped image.  The discrete steady operator
    has this symmetry exactly when every blocked link returns its population
    to the opposite slot of the same site, on flat walls and at every convex
    or concave corner alike; the image is a grain pack with scattered solid
    voxels, so it is full of corners and has no mirror symmetry that would
    make both sides zero.  (A convex-corner rule that reflects a diagonal
    population specularly passes the Poiseuille pins and misses this by
    0.7 %.)"""
    from paper_2110_13055_gb300.inputs import grain_pack
    rng = np.random.default_rng(3 + dim)
    shape = (24, 24) if dim == 2 else (10, 12, 14)
    m, _ = grain_pack(shape, 0.6, 1.5 if dim == 2 else 1.2, 4.0 if dim == 2 else 2.5,
                      seed=11 if dim == 2 else 21)
    m = m.copy()
    m[rng.random(shape) < (0.08 if dim == 2 else 0.06)] = 1
    mT = np.ascontiguousarray(np.swapaxes(m, -1, -2))
    kw = dict(mirror=False, lateral_walls=False, tau=tau, force=1e-6, tol=1e-13,
              check_every=200, max_steps=3_000_000)
    uA, _, _, stA = O.lbm(m, **kw)
    uB, _, _, stB = O.lbm(mT, **kw)
    assert stA == 0 and stB == 0
    Kxx, Kyx, Kxy = uA[0].sum(), uA[1].sum(), uB[1].sum()
    assert abs(Kyx) > 1e-3 * abs(Kxx)          # the cross term is not trivially zero
    assert abs(Kyx - Kxy) < 1e-10 * abs(Kxx)


def test_convergence_stops_at_a_check():
    """The steady-state test fires at a multiple of the check interval, with
    a residual below the tolerance."""
    m = slit(4, 10)
    u, steps, res, st = O.lbm(m, mirror=False, tau=1.0, force=1e-6, tol=1e-8,
                              check_every=50, max_steps=1_000_000)
    assert st == 0 and steps % 50 == 0 and res < 1e-8
    u, steps, res, st = O.lbm(m, mirror=False, tau=1.0, force=1e-6, tol=1e-30,
                              check_every=50, max_steps=500)
    assert st == 1 and steps == 500


def test_velocity_export_matches_pore_mean():
    """The exported velocity has pore-mean x velocity U = sum u / (N phi)
    (Sec. 4) equal to the requested value."""
    from paper_2110_13055_gb300.inputs import grain_pack
    m, _ = grain_pack((16, 24), 0.6, 2.0, 4.0, seed=3)
    u, *_ = O.lbm(m, mirror=True, tol=0.0, check_every=20, max_steps=200)
    up, U_lat = O.velocity_export(m, u, 1e-4)
    assert up.shape == (2, 16, 24)
    assert abs(up[0][m == 0].mean() - 1e-4) < 1e-16
    assert np.all(up[:, m == 1] == 0)
