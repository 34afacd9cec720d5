"""Device geometry query (Sec. 4: porosity and specific surface) against a
direct numpy count of the same definition, and the Sec. 5 trend: at fixed
porosity, thinner fibres expose more pore-solid interface."""
import numpy as np
import pytest

from paper_2110_13055_gb300 import cdi, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def faces_numpy(mask, walls):
    """Pore-solid faces: x faces never cross the inlet/outlet planes; lateral
    faces wrap periodically unless the lateral boundary is a wall."""
    m = mask.astype(bool)
    pore = ~m
    total = 0
    for ax in range(m.ndim):
        for s in (1, -1):
            nb = np.roll(m, -s, axis=ax)
            valid = np.ones_like(m)
            if ax == m.ndim - 1 or walls:
                idx = [slice(None)] * m.ndim
                idx[ax] = -1 if s == 1 else 0
                valid[tuple(idx)] = False
            total += int(np.count_nonzero(pore & nb & valid))
    return total


CASES = {
    "discs128x64": lambda: inputs.disc_pack_128x64()[0],
    "ragged37x23": lambda: inputs.grain_pack((23, 37), 0.62, 2.0, 4.5, seed=9)[0],
    "spheres19x13x11": lambda: inputs.grain_pack((11, 13, 19), 0.6, 1.5, 3.0, seed=4)[0],
    "fibres40": lambda: inputs.fibre_pack(40, 0.7, 4.0, seed=3)[0],
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("walls", [False, True])
def test_geometry_matches_count(case, walls):
    m = CASES[case]()
    dx = 1e-6
    with cdi.Domain(m, precision=cdi.FP32, dx=dx, mirror=not walls, lateral_walls=walls) as d:
        phi, s = d.geometry()
    assert phi == np.count_nonzero(m == 0) / m.size
    assert s == pytest.approx(faces_numpy(m, walls) / (m.size * dx), rel=0, abs=0)


def test_fibre_surface_grows_as_diameter_shrinks():
    """Overlapping cylinders of diameter d at solid fraction 1 - phi have a
    continuum specific surface 4 (1 - phi) / d when they do not overlap;
    voxel stair-steps and overlaps move it, but halving d must raise s."""
    dx = 1e-6
    out = []
    for dia in (8.0, 4.0):
        m, _ = inputs.fibre_pack(64, 0.8, dia, seed=11)
        with cdi.Domain(m, precision=cdi.FP32, dx=dx) as d:
            out.append(d.geometry())
    (p8, s8), (p4, s4) = out
    assert abs(p8 - 0.8) < 0.02 and abs(p4 - 0.8) < 0.02
    assert s4 > 1.5 * s8


@pytest.mark.parametrize("case", ["ragged37x23", "spheres19x13x11"])
@pytest.mark.parametrize("prec", [cdi.FP64, cdi.FP32_CPAIR])
def test_derived_figures_match_oracle(case, prec):
    """cdi_query_derived (Sec. 4: phi, s, l_c = pi / s, U, Pe, Da; Sec. 4.1:
    P_rm and U A P_rm dt / (V_t phi)) against the oracle's functions on the
    oracle's own run.  Geometry figures are exact counts; U is a sum of the
    stored (FP32 or FP64) velocities; the removal figures follow the outlet
    concentration, so they carry its tolerance."""
    import oracle as O
    m = CASES[case]()
    Z, D, c0, Ka, n = (1, -1), (1.33e-9, 2.03e-9), 10.0, 1e-6, 300
    r = O.run_case(m, flow_tol=0.0, max_flow_steps=600, U_target=1e-4, applied_V=1.0,
                   lambda_D=1.5e-7, n_np_steps=n)
    with cdi.Domain(m, precision=prec) as d:
        with pytest.raises(cdi.CDIError) as e:
            d.derived()
        assert e.value.status == 6
        d.solve_flow(tol=0.0, max_steps=600, U_target=1e-4)
        d.set_potential(1.0, c_bulk=c0, lambda_D=1.5e-7, tol=1e-13)
        d.init_transport(Z, D, c0=c0, Ka=Ka, dt=r["dt"])
        d.step(n)
        g = d.derived()
    o = O.derived(m, r["u"], r["C_out"], c0=c0, D=D, Ka=Ka, dx=1e-7, dt=r["dt"], n_steps=n)
    for k in ("porosity", "specific_surface", "l_c_m", "elapsed_s"):
        assert g[k] == pytest.approx(o[k], rel=1e-14), k
    fp64 = prec == cdi.FP64
    np.testing.assert_allclose(g["U_mps"], o["U_mps"], rtol=1e-12 if fp64 else 1e-6)
    np.testing.assert_allclose(g["Pe"], o["Pe"], rtol=1e-12 if fp64 else 1e-6)
    np.testing.assert_allclose(g["Da"], o["Da"], rtol=1e-14)
    # P_rm = 1 - C_out / c0: an outlet-concentration error d gives d / c0
    tol_c = 1e-10 if fp64 else 1e-4
    bound = tol_c * np.asarray(r["C_out"]) / c0
    assert np.all(np.abs(g["removal"] - o["removal"]) <= bound), (g["removal"], o["removal"])
    per_removal = o["amount"] / np.where(o["removal"] != 0, o["removal"], 1.0)
    assert np.all(np.abs(g["amount"] - o["amount"])
                  <= np.abs(per_removal) * bound + 1e-6 * np.abs(o["amount"])), \
        (g["amount"], o["amount"])
