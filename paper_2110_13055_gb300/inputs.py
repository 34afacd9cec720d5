"""Seeded synthetic inputs: voxel masks of porous electrodes.

The paper's geometries (a digitised SEM image, Sec. 4 / Fig. 4, and random
fibre packs, Sec. 5) are not available, so seeded disc and sphere packs with
the same structure stand in for them: grains of a few to a few tens of voxels
in a 2D or 3D voxel grid with one voxel per grid block (the MAC grid of
Sec. 2), porosity 0.4-0.8.

This module holds input generation only.  It contains none of the solver's
arithmetic, and both the CUDA path and the CPU oracle take their masks from it.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written here from its published
definition.

Mask convention: ``uint8`` array of shape ``(ny, nx)`` (2D) or ``(nz, ny, nx)``
(3D), C order so x is the fastest index, 1 = solid, 0 = pore (fluid).
"""
from __future__ import annotations

import hashlib
from dataclasses import dataclass

import numpy as np

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator; ``uniform()`` returns a double in [0, 1)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_range(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()


@dataclass
class PackInfo:
    porosity: float
    n_objects: int
    sha256: str


def _stamp(solid: np.ndarray, centre, r: float, periodic_axes) -> int:
    """Mark voxels whose centre lies within ``r`` of ``centre`` (axis order
    matches ``solid.shape``; periodic wrap on the listed axes).  Returns the
    number of voxels that turned solid."""
    slices = []
    coords = []
    for ax, (c, n) in enumerate(zip(centre, solid.shape)):
        lo = int(np.floor(c - r - 0.5))
        hi = int(np.ceil(c + r + 0.5))
        idx = np.arange(lo, hi + 1)
        if ax in periodic_axes:
            keep = idx
        else:
            keep = idx[(idx >= 0) & (idx < n)]
        coords.append((keep + 0.5 - c) ** 2)
        slices.append(np.mod(keep, n) if ax in periodic_axes else keep)
    d2 = coords[0]
    for extra in coords[1:]:
        d2 = np.add.outer(d2, extra)
    hit = d2 <= r * r
    if solid.ndim == 2:
        ii, jj = np.nonzero(hit)
        idx = (slices[0][ii], slices[1][jj])
    else:
        ii, jj, kk = np.nonzero(hit)
        idx = (slices[0][ii], slices[1][jj], slices[2][kk])
    # a box wider than a periodic axis visits a voxel twice: count each once
    flat = np.unique(np.ravel_multi_index(idx, solid.shape))
    view = solid.reshape(-1)
    new = int(np.count_nonzero(view[flat] == 0))
    view[flat] = 1
    return new


def _periodic_dist2(a, b, shape, periodic_axes) -> float:
    s = 0.0
    for ax, (x, y, n) in enumerate(zip(a, b, shape)):
        d = abs(x - y)
        if ax in periodic_axes:
            d = min(d, n - d)
        s += d * d
    return s


def grain_pack(shape, porosity: float, r_min: float, r_max: float, seed: int,
               overlap: bool = True, lateral_periodic: bool = True,
               max_attempts: int = 1_000_000):
    """Random sequential addition of discs (2D) or spheres (3D).

    Centres are uniform in the box, radii uniform in [r_min, r_max] (a fixed
    radius when equal).  Objects are added until the porosity first drops to
    ``porosity`` or below.  With ``overlap=False`` a candidate that intersects
    an earlier object (centre distance < r_a + r_b) is rejected.  The lateral
    axes (all but x) wrap when ``lateral_periodic``; x never wraps.

    Returns ``(mask, PackInfo)``.
    """
    shape = tuple(int(s) for s in shape)
    ndim = len(shape)
    assert ndim in (2, 3)
    solid = np.zeros(shape, dtype=np.uint8)
    rng = SplitMix64(seed)
    periodic = set(range(ndim - 1)) if lateral_periodic else set()
    placed = []
    total = solid.size
    n_solid = 0
    attempts = 0
    while 1.0 - n_solid / total > porosity and attempts < max_attempts:
        attempts += 1
        # draw x first, then y (then z): coordinates in (x, y, z) order
        xyz = [rng.uniform() * shape[ndim - 1 - a] for a in range(ndim)]
        r = r_min if r_max == r_min else rng.uniform_range(r_min, r_max)
        centre = tuple(reversed(xyz))  # array axis order
        if not overlap:
            if any(_periodic_dist2(centre, c, shape, periodic) < (r + rc) ** 2
                   for c, rc in placed):
                continue
        placed.append((centre, r))
        n_solid += _stamp(solid, centre, r, periodic)
    phi = 1.0 - n_solid / total
    return solid, PackInfo(phi, len(placed), mask_sha256(solid))


def fibre_pack(n: int, porosity: float, diameter_vox: float, seed: int,
               max_fibres: int = 100000):
    """Random straight fibres of one diameter through an n^3 box (the fibrous
    electrodes of Sec. 5): each fibre's axis passes through a point uniform in
    the box along a direction uniform on the sphere and extends to the box
    faces; voxels whose centre lies within half the diameter of the axis are
    solid; fibres overlap freely; fibres are added until the porosity first
    drops to the target.  Returns ``(mask, PackInfo)`` with shape (n, n, n)."""
    rng = SplitMix64(seed)
    solid = np.zeros((n, n, n), dtype=np.uint8)        # (z, y, x)
    flat = solid.reshape(-1)
    r = 0.5 * diameter_vox
    h = int(np.ceil(r * np.sqrt(3.0))) + 1             # slice window half-width
    w = np.arange(-h, h + 1)
    total = solid.size
    n_solid = 0
    count = 0
    while 1.0 - n_solid / total > porosity and count < max_fibres:
        p = np.array([rng.uniform() * n for _ in range(3)])          # x, y, z
        cz = 2.0 * rng.uniform() - 1.0
        ph = 2.0 * np.pi * rng.uniform()
        s = np.sqrt(1.0 - cz * cz)
        d = np.array([s * np.cos(ph), s * np.sin(ph), cz])          # unit axis
        # walk the axis along its dominant direction: in each slice the
        # voxels within r of the axis lie within h of the crossing point
        m = int(np.argmax(np.abs(d)))
        a, b = [k for k in range(3) if k != m]
        cm = np.arange(n) + 0.5
        t = (cm - p[m]) / d[m]
        qa = p[a] + t * d[a]
        qb = p[b] + t * d[b]
        ia = np.floor(qa).astype(int)[:, None, None] + w[None, :, None]
        ib = np.floor(qb).astype(int)[:, None, None] + w[None, None, :]
        im = np.broadcast_to(np.arange(n)[:, None, None], (n, w.size, w.size))
        ia = np.broadcast_to(ia, im.shape)
        ib = np.broadcast_to(ib, im.shape)
        inside = (ia >= 0) & (ia < n) & (ib >= 0) & (ib < n)
        coords = [None, None, None]
        coords[m], coords[a], coords[b] = im[inside], ia[inside], ib[inside]
        vx = coords[0] + 0.5 - p[0]
        vy = coords[1] + 0.5 - p[1]
        vz = coords[2] + 0.5 - p[2]
        tt = vx * d[0] + vy * d[1] + vz * d[2]
        hit = vx * vx + vy * vy + vz * vz - tt * tt <= r * r
        idx = np.unique((coords[2][hit] * n + coords[1][hit]) * n + coords[0][hit])
        n_solid += int(np.count_nonzero(flat[idx] == 0))
        flat[idx] = 1
        count += 1
    phi = 1.0 - n_solid / total
    return solid, PackInfo(phi, count, mask_sha256(solid))


def mask_sha256(mask: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(mask, dtype=np.uint8).tobytes()).hexdigest()


def channel_2d(nx: int, ny: int) -> np.ndarray:
    """Open 2D channel (all pore); walls come from the lateral wall flag."""
    return np.zeros((ny, nx), dtype=np.uint8)


def crop(mask: np.ndarray, shape) -> np.ndarray:
    """Leading corner crop (x from the inlet side)."""
    sl = tuple(slice(0, s) for s in shape)
    return np.ascontiguousarray(mask[sl])


# Synthetic stand-ins for the paper's workloads (recipes written out in words
# in the design notes).  Sizes are (nx, ny[, nz]).
def disc_pack_128x64():
    """128x64 lattice, non-overlapping discs of radius 6, porosity 0.6, seed 0."""
    return grain_pack((64, 128), 0.6, 6.0, 6.0, seed=0, overlap=False)


def disc_pack_1024x512():
    """1024x512 lattice, polydisperse discs r~U[4,16] (overlap allowed),
    porosity 0.5, seed 1."""
    return grain_pack((512, 1024), 0.5, 4.0, 16.0, seed=1, overlap=True)


def sphere_pack_256():
    """256^3 pack of spheres r~U[6,12] (overlap allowed), porosity 0.45, seed 2."""
    return grain_pack((256, 256, 256), 0.45, 6.0, 12.0, seed=2, overlap=True)


def sweep_instance(seed: int):
    """One geometry of the batched parameter sweep: a 2D polydisperse disc
    pack (overlap allowed, r ~ U[4, 16]) whose size and porosity are drawn
    from the seed: nx = 32 k, k uniform in 8..32; ny = 32 j, j uniform in
    8..16 (256x256 to 1024x512); porosity ~ U[0.4, 0.7].  Returns
    ``(mask, PackInfo)``."""
    rng = SplitMix64(seed ^ 0x5EED5EED)
    nx = 32 * (8 + int(rng.uniform() * 25))
    ny = 32 * (8 + int(rng.uniform() * 9))
    phi = rng.uniform_range(0.4, 0.7)
    return grain_pack((ny, nx), phi, 4.0, 16.0, seed=seed)


def serve_instance(seed: int):
    """One request geometry of the serving workload: half are 2D 512x512 disc
    packs, half 3D n^3 sphere packs with n in {64, 96, 128, 160, 192};
    porosity ~ U[0.4, 0.6], r ~ U[4, 16] (2D) or U[6, 12] (3D); the applied
    potential ~ U[0.2, 1.2] V.  Returns ``(mask, applied_V)``."""
    rng = SplitMix64(seed ^ 0x5E11E)
    three_d = rng.uniform() < 0.5
    phi = rng.uniform_range(0.4, 0.6)
    V = rng.uniform_range(0.2, 1.2)
    if three_d:
        n = (64, 96, 128, 160, 192)[int(rng.uniform() * 5)]
        m, _ = grain_pack((n, n, n), phi, 6.0, 12.0, seed=seed)
    else:
        m, _ = grain_pack((512, 512), phi, 4.0, 16.0, seed=seed)
    return m, V


def random_mask(shape, solid_fraction: float, seed: int) -> np.ndarray:
    """I.i.d. voxel noise (for edge-case tests): each voxel solid with the
    given probability, drawn from numpy's seeded PCG64 generator."""
    rs = np.random.default_rng(seed)
    return (rs.random(shape) < solid_fraction).astype(np.uint8)
