"""Host-side arithmetic of bench.py's roofline: the method's bytes per
launch (per site and per cell), the layout bytes reported beside
them, the L2/HBM bound and the source-hash gate on recorded DRAM traffic."""
import json
import os

import bench
from paper_2110_13055_gb300 import cdi


def test_method_bytes_per_site_and_cell():
    n_fp, n_pore = 1_000_000, 480_000
    lbm, lbm_layout, npb, np_layout = bench.algorithmic_bytes(cdi.FP32_CPAIR, 3, n_fp, n_pore)
    assert lbm == 152 * n_fp                       # 19 populations read + written, 4 B
    assert npb == 49 * n_pore                      # 2 species as pairs, u, psi, mask
    tiles = (n_fp + 31) // 32
    assert lbm_layout == (12 * n_fp + 8 * 4 * tiles) // 2   # odd step only, averaged
    assert np_layout == 21 * n_pore                # psi low word, flags, 4 lateral ranks
    lbm, lbm_layout, npb, _ = bench.algorithmic_bytes(cdi.FP32_SPLIT, 2, n_fp, n_pore)
    assert lbm == 144 * n_fp                       # 9 populations as pairs
    assert lbm_layout == (8 * n_fp + 2 * 4 * tiles) // 2
    assert npb == (2 * 2 * 8 + 2 * 4 + 4 + 1) * n_pore
    lbm, _, npb, _ = bench.algorithmic_bytes(cdi.FP32, 3, n_fp, n_pore)
    assert lbm == 152 * n_fp and npb == 33 * n_pore   # plain FP32 storage in 3D
    lbm, _, npb, _ = bench.algorithmic_bytes(cdi.FP64, 2, n_fp, n_pore)
    assert lbm == 144 * n_fp and npb == (2 * 2 * 8 + 2 * 8 + 8 + 1) * n_pore


def test_bound_follows_recorded_traffic():
    assert bench.roofline_bound(None, 100, 10) == "hbm"
    assert bench.roofline_bound(95, 100, 10) == "hbm"
    assert bench.roofline_bound(40, 75, 2) == "l2"       # the L2-resident 2D pack


def test_recorded_traffic_needs_the_current_source(monkeypatch):
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    entry = rec["k_lbm_step"]["3d-256"]
    monkeypatch.setattr(bench, "kernel_hash", lambda k: entry["source_sha"])
    assert bench.recorded_traffic("k_lbm_step", "3d-256") == entry["dram_bytes_per_launch"]
    monkeypatch.setattr(bench, "kernel_hash", lambda k: "0" * 16)
    assert bench.recorded_traffic("k_lbm_step", "3d-256") is None
    assert bench.recorded_traffic("k_lbm_step", "no-such-workload") is None
