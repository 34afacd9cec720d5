"""Oracle pins for the Sec. 4 / Sec. 4.1 figures: porosity, specific surface
(l_c = pi / s), the pore-mean velocity U, Pe, Da, salt removal and the
adsorbed-amount formula, each against values worked out by hand."""
import numpy as np
import pytest

import oracle as O


def test_single_solid_voxel_2d_and_3d():
    m = np.zeros((5, 5), np.uint8)
    m[2, 2] = 1
    dx = 1e-7
    assert O.interface_faces(m) == 4
    assert O.specific_surface(m, dx) == pytest.approx(4 / (25 * dx), rel=1e-15)
    assert O.porosity(m) == 24 / 25
    m3 = np.zeros((3, 3, 3), np.uint8)
    m3[1, 1, 1] = 1
    assert O.interface_faces(m3) == 6
    assert O.specific_surface(m3, dx) == pytest.approx(6 / (27 * dx), rel=1e-15)


def test_slit_and_boundary_rules():
    """A slit between solid rows: two interface faces per column, so
    s = 2 / (ny dx) and l_c = pi ny dx / 2.  One solid row on the lateral
    edge: two faces per column when the rows wrap, one with walls.  Faces
    across the inlet and outlet planes never count."""
    nx, H, dx = 7, 4, 2e-7
    m = np.zeros((H + 2, nx), np.uint8)
    m[[0, -1], :] = 1
    for walls in (False, True):
        s = O.specific_surface(m, dx, lateral_walls=walls)
        assert s == pytest.approx(2 / ((H + 2) * dx), rel=1e-15)
    e = np.zeros((4, nx), np.uint8)
    e[0, :] = 1
    assert O.interface_faces(e) == 2 * nx
    assert O.interface_faces(e, lateral_walls=True) == nx
    c = np.zeros((3, 6), np.uint8)
    c[:, 0] = 1          # a solid inlet column: its -x faces are the inlet plane
    c[:, -1] = 1         # a solid outlet column
    assert O.interface_faces(c) == 2 * 3


def test_dimensionless_groups_by_hand():
    """Uniform x velocity 1e-4 m/s in the pore cells of the 5x5 image with one
    solid voxel: U = 1e-4; l_c = 25 pi dx / 4; Pe = U l_c / D, Da = Ka l_c / D."""
    m = np.zeros((5, 5), np.uint8)
    m[2, 2] = 1
    dx, D, Ka = 1e-7, np.array([1e-9, 2e-9]), 1e-6
    u = np.zeros((2,) + m.shape)
    u[0][m == 0] = 1e-4
    r = O.derived(m, u, [5.0, 2.0], c0=10.0, D=D, Ka=Ka, dx=dx, dt=1e-6, n_steps=10)
    l_c = 25 * np.pi * dx / 4
    assert r["U_mps"] == pytest.approx(1e-4, rel=1e-15)
    assert r["l_c_m"] == pytest.approx(l_c, rel=1e-15)
    np.testing.assert_allclose(r["Pe"], 1e-4 * l_c / D, rtol=1e-15)
    np.testing.assert_allclose(r["Da"], Ka * l_c / D, rtol=1e-15)
    np.testing.assert_allclose(r["removal"], [0.5, 0.8], rtol=1e-15)
    assert r["elapsed_s"] == pytest.approx(1e-5, rel=1e-15)


def test_amount_is_one_after_one_pore_volume_at_full_removal():
    """U A P_rm dt / (V_t phi): with every ion removed (P_rm = 1) over the
    time the inflow U A takes to bring in one pore volume V_t phi, the
    formula gives exactly 1 (2D per metre of depth and 3D)."""
    for shape in ((6, 9), (4, 5, 9)):
        m = np.zeros(shape, np.uint8)
        m.reshape(-1)[::7] = 1
        m[..., 0] = 0
        dx, U = 1e-7, 3e-5
        u = np.zeros((m.ndim,) + m.shape)
        u[0][m == 0] = U
        phi = O.porosity(m)
        A = shape[0] * dx if m.ndim == 2 else shape[0] * shape[1] * dx * dx
        t_pore = m.size * dx ** m.ndim * phi / (U * A)
        r = O.derived(m, u, [0.0], c0=1.0, D=[1e-9], Ka=1e-6, dx=dx, dt=t_pore / 8, n_steps=8)
        assert r["amount"][0] == pytest.approx(1.0, rel=1e-14)
