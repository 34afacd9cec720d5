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
