"""The seeded geometry generators: determinism, porosity, structure."""
import numpy as np

from paper_2110_13055_gb300 import inputs as I


def test_splitmix64_published_sequence():
    """First outputs of SplitMix64 seeded with 0 (the values of the reference
    description of the generator)."""
    g = I.SplitMix64(0)
    assert g.next_u64() == 0xE220A8397B1DCDAF
    assert g.next_u64() == 0x6E789E6AA1B965F4
    assert g.next_u64() == 0x06C45D188009454F


def test_disc_pack_128x64_is_reproducible():
    m1, i1 = I.disc_pack_128x64()
    m2, i2 = I.disc_pack_128x64()
    assert m1.shape == (64, 128) and m1.dtype == np.uint8
    assert i1.sha256 == i2.sha256
    assert 0.58 < i1.porosity <= 0.6


def test_non_overlapping_discs_do_not_touch():
    m, info = I.grain_pack((40, 60), 0.7, 4.0, 4.0, seed=3, overlap=False)
    assert info.porosity <= 0.7
    # every disc of radius 4 covers ~50 voxels; no overlap means the solid
    # count is close to n_objects * area
    assert abs(m.sum() - info.n_objects * np.pi * 16) < 0.1 * m.sum()


def test_sphere_pack_porosity():
    m, info = I.grain_pack((24, 24, 24), 0.5, 3.0, 5.0, seed=2)
    assert m.shape == (24, 24, 24)
    assert 0.45 < info.porosity <= 0.5


def _fibres_brute_force(n, porosity, diameter, seed):
    """The fibre recipe with a full-volume distance test per fibre."""
    rng = I.SplitMix64(seed)
    solid = np.zeros((n, n, n), np.uint8)
    c = np.arange(n) + 0.5
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    r2 = (0.5 * diameter) ** 2
    while 1.0 - solid.sum() / solid.size > porosity:
        p = [rng.uniform() * n for _ in range(3)]
        cz = 2.0 * rng.uniform() - 1.0
        ph = 2.0 * np.pi * rng.uniform()
        s = np.sqrt(1.0 - cz * cz)
        d = (s * np.cos(ph), s * np.sin(ph), cz)
        vx, vy, vz = X - p[0], Y - p[1], Z - p[2]
        t = vx * d[0] + vy * d[1] + vz * d[2]
        solid[vx * vx + vy * vy + vz * vz - t * t <= r2] = 1
    return solid


def test_fibre_pack_matches_brute_force():
    """The windowed fibre stamping marks exactly the voxels a full distance
    test marks (straight fibres through the box, Sec. 5)."""
    for n, phi, dia, seed in ((24, 0.7, 4.0, 1), (20, 0.5, 6.0, 2)):
        m, info = I.fibre_pack(n, phi, dia, seed)
        assert np.array_equal(m, _fibres_brute_force(n, phi, dia, seed))
        assert info.porosity <= phi


def test_sweep_and_serve_recipes():
    """The batched-sweep geometries span 256x256..1024x512 in multiples of 32
    with porosity in [0.4, 0.7]; the serving requests are half 2D 512^2, half
    3D n^3 with n in {64, ..., 192}, porosity in [0.4, 0.6], V in [0.2, 1.2];
    both are reproducible from their seeds."""
    for seed in range(10, 16):
        m, info = I.sweep_instance(seed)
        ny, nx = m.shape
        assert nx % 32 == 0 and ny % 32 == 0 and 256 <= nx <= 1024 and 256 <= ny <= 512
        assert 0.38 <= info.porosity <= 0.7
        assert np.array_equal(m, I.sweep_instance(seed)[0])
    kinds = []
    for seed in range(100, 108):
        m, V = I.serve_instance(seed)
        assert 0.2 <= V <= 1.2
        phi = float((m == 0).mean())
        assert 0.38 <= phi <= 0.6
        if m.ndim == 2:
            assert m.shape == (512, 512)
        else:
            assert m.shape[0] == m.shape[1] == m.shape[2] and m.shape[0] in (64, 96, 128, 160, 192)
        kinds.append(m.ndim)
    assert 2 in kinds and 3 in kinds
