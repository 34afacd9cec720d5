"""FP64 CPU oracle for the pore-scale CDI model of arXiv 2110.13055.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, the smoke check and the
benchmark's CPU-baseline leg may import this package.  The product path (the
CUDA library and its binding) never touches it, and it shares no code with
that path: the heavy loops live in ``cdi_oracle.c`` (plain C, FP64), built
here with gcc; the light post-processing below is plain numpy.

Every function cites the passage it follows (Sec./Eq. of the paper).  The
readings taken where the paper is silent are listed at the top of
``cdi_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cdi_oracle.c")
_HDR = os.path.join(_HERE, "cdi_oracle.h")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()

# Physical constants.  e and k_B are the values printed with Eq. 9-10.
E_CHARGE = 1.6e-19      # C
K_B = 1.38e-23          # J/K
FARADAY = 96485.0       # C/mol
EPS0 = 8.854e-12        # F/m
T_DEFAULT = 298.15      # K (the paper's temperature unit is garbled; kelvin)
EPS_R_DEFAULT = 78.5    # water (not stated in the paper)


def thermal_voltage(T=T_DEFAULT):
    """k_B T / e, the scale of psi in Eq. 3 and Eq. 9."""
    return K_B * T / E_CHARGE


def debye_length(c_bulk, T=T_DEFAULT, eps_r=EPS_R_DEFAULT):
    """The length in the exponent of Eq. 10: sqrt(eps_r eps0 k_B T / (2 C e F))."""
    return np.sqrt(eps_r * EPS0 * K_B * T / (2.0 * c_bulk * E_CHARGE * FARADAY))


def build(force: bool = False) -> str:
    """Compile ``cdi_oracle.c`` into ``_build/liboracle.so`` with gcc."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                       os.path.getmtime(_HDR))):
            return _LIB_PATH
        os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i, l, d = ctypes.c_int, ctypes.c_long, ctypes.c_double
        lib.orc_lbm.argtypes = [i, i, i, i, P, i, i, d, d, d, i, l, P, P, P]
        lib.orc_lbm.restype = i
        lib.orc_psi.argtypes = [i, i, i, i, P, i, d, d, d, i, P, P, P]
        lib.orc_psi.restype = i
        lib.orc_np_dt.argtypes = [i, i, i, i, P, i, P, P, i, P, P, d, d, d, d]
        lib.orc_np_dt.restype = d
        lib.orc_np_run.argtypes = [i, i, i, i, P, i, P, P, i, P, P, d, d, d, d,
                                   d, l, P, P, P, P]
        lib.orc_np_run.restype = i
        lib.orc_psi_src.argtypes = [i, i, i, i, P, i, d, d, P, d, i, P, P, P]
        lib.orc_psi_src.restype = i
        lib.orc_pnp_run.argtypes = [i, i, i, i, P, i, P, i, P, P, d, d, d, d, d, l, l, d, d,
                                    d, P, P, P, P, P]
        lib.orc_pnp_run.restype = i
        lib.orc_np_operator.argtypes = [i, i, i, i, P, i, P, P, i, d, d, d, d, d, P, P, P, P, P]
        lib.orc_np_operator.restype = i
        lib.orc_set_threads.argtypes = [i]
        lib.orc_set_threads.restype = None
        lib.orc_threads.argtypes = []
        lib.orc_threads.restype = i
        _lib = lib
    return _lib


def set_threads(n: int) -> None:
    """Host threads of the oracle's parallel loops (OpenMP).  Results do not
    depend on the count: parallel loops write disjoint outputs and sums are
    taken in a fixed order."""
    _load().orc_set_threads(int(n))


def threads() -> int:
    """Host threads the oracle's parallel loops use."""
    return int(_load().orc_threads())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(mask: np.ndarray):
    if mask.ndim == 2:
        ny, nx = mask.shape
        return 2, nx, ny, 1
    nz, ny, nx = mask.shape
    return 3, nx, ny, nz


def _mask(mask):
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    if m.min(initial=0) < 0 or m.max(initial=0) > 1:
        raise ValueError("mask values must be 0 (pore) or 1 (solid)")
    return m


# --------------------------------------------------------------------------
# Flow (Sec. 2, Eq. 1-2 solved by Eq. 7-8)
# --------------------------------------------------------------------------
def lbm(mask, *, mirror=True, lateral_walls=False, tau=1.0, force=1e-6,
        tol=1e-8, check_every=100, max_steps=2_000_000):
    """Steady Stokes flow by the lattice Boltzmann method (Eq. 7-8, bounce-back
    and body force of Sec. 2).

    Returns ``(u_flow, steps, residual, status)``; ``u_flow`` has shape
    ``(dim,) + flow_grid_shape`` in lattice units, where the flow grid is the
    mask followed by its mirror image along x when ``mirror``.  ``status`` is 0
    when converged (or when ``tol <= 0`` and ``max_steps`` were run), 1 when
    ``tol`` was not reached.
    """
    m = _mask(mask)
    dim, nx, ny, nz = _dims(m)
    NX = 2 * nx if mirror else nx
    shape = (ny, NX) if dim == 2 else (nz, ny, NX)
    u = np.zeros((dim,) + shape, dtype=np.float64)
    steps = ctypes.c_long(0)
    res = ctypes.c_double(0.0)
    st = _load().orc_lbm(dim, nx, ny, nz, _ptr(m), int(mirror), int(lateral_walls),
                         float(tau), float(force), float(tol), int(check_every),
                         int(max_steps), _ptr(u), ctypes.byref(steps),
                         ctypes.byref(res))
    if st < 0:
        raise ValueError("orc_lbm rejected its arguments")
    return u, steps.value, res.value, st


def velocity_export(mask, u_flow, U_target):
    """Scale the lattice velocity on the original (unmirrored) grid so that the
    pore-mean x velocity U = sum u / (N phi) of Sec. 4 equals ``U_target``
    (m/s).  Returns ``(u_phys, U_lattice)``; u_phys is 0 in solid cells."""
    m = _mask(mask)
    nx = m.shape[-1]
    u = np.array(u_flow[..., :nx], dtype=np.float64)
    pore = m == 0
    n_pore = int(pore.sum())
    U_lat = float(u[0][pore].sum() / n_pore) if n_pore else 0.0
    if U_target == 0.0:
        return np.zeros_like(u), U_lat
    if U_lat == 0.0:
        raise ValueError("no net flow through the pore space")
    u_phys = u * (U_target / U_lat)
    u_phys[:, ~pore] = 0.0
    return u_phys, U_lat


# --------------------------------------------------------------------------
# Potential (Eq. 4-5, Dirichlet at the solid surface)
# --------------------------------------------------------------------------
def psi(mask, psi_s, *, dx=1e-7, c_bulk=10.0, T=T_DEFAULT, eps_r=EPS_R_DEFAULT,
        mode="debye", lambda_D=None, lateral_walls=False, tol=1e-13,
        max_iter=200000):
    """Frozen potential field in volts (0 in solid cells).

    ``mode='debye'`` screens Eq. 4 with the Debye length of Eq. 10 (or
    ``lambda_D`` when given); ``mode='laplace'`` solves Eq. 4 with zero charge
    (the electroneutral initial state)."""
    m = _mask(mask)
    dim, nx, ny, nz = _dims(m)
    if mode == "laplace":
        kdx2 = 0.0
    else:
        lam = lambda_D if lambda_D else debye_length(c_bulk, T, eps_r)
        kdx2 = (dx / lam) ** 2
    out = np.zeros(m.shape, dtype=np.float64)
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = _load().orc_psi(dim, nx, ny, nz, _ptr(m), int(lateral_walls), float(psi_s),
                         float(kdx2), float(tol), int(max_iter), _ptr(out),
                         ctypes.byref(it), ctypes.byref(rel))
    if st < 0:
        raise ValueError("orc_psi rejected its arguments")
    return out, it.value, rel.value


def psi_operator(mask, psi_s, *, lateral_walls=False):
    """The potential's face rules of Eq. 4 (Sec. 2) as a sparse matrix over
    the pore cells: (A0 v)_P = sum_f T_f v_P - sum_{pore neighbours} v_nb with
    T = 1 towards a pore neighbour or the inlet feed (psi = 0), 2 towards a
    solid face (psi_s at half a cell), 0 at the outlet and at lateral walls;
    b_P = 2 psi_s per solid face.  Returns ``(A0, b, cells)`` (scipy CSR,
    right-hand side, lattice indices of the pore cells in order)."""
    import scipy.sparse as sp
    m = _mask(mask)
    dim, nx, ny, nz = _dims(m)
    m3 = m.reshape(nz, ny, nx)
    cells = np.flatnonzero(m3.reshape(-1) == 0)
    index = -np.ones(m3.size, dtype=np.int64)
    index[cells] = np.arange(len(cells))
    z, y, x = np.unravel_index(cells, (nz, ny, nx))
    diag = np.zeros(len(cells))
    b = np.zeros(len(cells))
    rows, cols = [], []
    for a, s in [(0, 1), (0, -1), (1, 1), (1, -1), (2, 1), (2, -1)][:2 * dim]:
        X, Y, Z = x.copy(), y.copy(), z.copy()
        if a == 0:
            X += s
            inlet, outlet = X < 0, X >= nx
            inside = ~(inlet | outlet)
            diag[inlet] += 1.0                   # the feed at psi = 0
            wall = np.zeros_like(inside)
        else:
            C = Y if a == 1 else Z
            ext = ny if a == 1 else nz
            C += s
            beyond = (C < 0) | (C >= ext)
            wall = beyond if lateral_walls else np.zeros_like(beyond)
            C %= ext
            inside = ~wall
        q = np.zeros(len(cells), dtype=np.int64)
        q[inside] = (Z[inside] * ny + Y[inside]) * nx + X[inside]
        solid = inside & (m3.reshape(-1)[q] == 1)
        pore = inside & ~solid
        diag[solid] += 2.0
        b[solid] += 2.0 * psi_s
        diag[pore] += 1.0
        rows.append(np.flatnonzero(pore))
        cols.append(index[q[pore]])
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    n = len(cells)
    A0 = sp.csr_matrix((np.concatenate([diag, -np.ones(len(r))]),
                        (np.concatenate([np.arange(n), r]), np.concatenate([np.arange(n), c]))),
                       shape=(n, n))
    return A0, b, cells


def psi_pb(mask, psi_s, *, dx=1e-7, c_bulk=10.0, T=T_DEFAULT, eps_r=EPS_R_DEFAULT,
           lambda_D=None, lateral_walls=False, tol=1e-12, max_newton=200):
    """Eq. 4 with the charge of Eq. 5 at Boltzmann equilibrium (Eq. 9) for a
    1:1 salt: the nonlinear Poisson-Boltzmann equation whose 1D solution is
    Eq. 10.  Per pore cell, with the face rules of ``psi_operator`` and
    kdx2 = (dx / lambda_D)^2,
        (A0 psi)_P - b_P + kdx2 V_T sinh(psi_P / V_T) = 0.
    Newton's method from psi = 0: each step solves
        (A0 + kdx2 cosh(psi / V_T)) psi' = b + kdx2 (psi cosh(psi / V_T) - V_T sinh(psi / V_T))
    with a sparse LU factorisation, until the residual is below ``tol``
    relative to |b|.  Returns ``(psi, newton_steps, relres)``; psi in volts on
    the lattice, 0 in solid cells."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    m = _mask(mask)
    lam = lambda_D if lambda_D else debye_length(c_bulk, T, eps_r)
    kdx2 = (dx / lam) ** 2
    vt = thermal_voltage(T)
    A0, b, cells = psi_operator(m, psi_s, lateral_walls=lateral_walls)
    bb = np.linalg.norm(b)
    psi = np.zeros(len(cells))
    rel, it = 0.0, 0
    while True:
        F = A0 @ psi - b + kdx2 * vt * np.sinh(psi / vt)
        rel = np.linalg.norm(F) / bb if bb > 0 else 0.0
        if rel < tol or it >= max_newton:
            break
        ch = np.cosh(psi / vt)
        J = (A0 + sp.diags(kdx2 * ch)).tocsc()
        psi = spl.spsolve(J, b + kdx2 * (psi * ch - vt * np.sinh(psi / vt)))
        it += 1
    out = np.zeros(m.size)
    out[cells] = psi
    return out.reshape(m.shape), it, rel


# --------------------------------------------------------------------------
# Transport (Eq. 3) with adsorption (Eq. 6)
# --------------------------------------------------------------------------
def _species(z, D):
    z = np.ascontiguousarray(np.atleast_1d(z), dtype=np.int32)
    D = np.ascontiguousarray(np.atleast_1d(D), dtype=np.float64)
    assert z.shape == D.shape
    return z, D


def np_dt(mask, u, psi_field, z, D, *, dx=1e-7, Ka=1e-6, T=T_DEFAULT,
          lateral_walls=False, safety=0.9):
    """Explicit step: ``safety`` over the largest outflow rate of any cell."""
    m = _mask(mask)
    dim, nx, ny, nz = _dims(m)
    z, D = _species(z, D)
    u = np.ascontiguousarray(u, dtype=np.float64)
    p = np.ascontiguousarray(psi_field, dtype=np.float64)
    return _load().orc_np_dt(dim, nx, ny, nz, _ptr(m), int(lateral_walls), _ptr(u),
                             _ptr(p), len(z), _ptr(z), _ptr(D), float(dx),
                             float(Ka), thermal_voltage(T), float(safety))


def np_run(mask, u, psi_field, z, D, *, c0, dt, n_steps, dx=1e-7, Ka=1e-6,
           T=T_DEFAULT, lateral_walls=False, C=None, acc=None):
    """Advance ``n_steps`` explicit Nernst-Planck steps.

    Starts from C = c0 in every pore cell (the saturated initial state of
    Sec. 4) unless ``C`` is given.  Returns ``(C, Gamma, In, Out)``; C has shape
    ``(ns,) + mask.shape`` (mol/m^3); Gamma, In, Out are per species (mol, or
    mol per metre of depth in 2D), accumulated onto ``acc`` when given."""
    m = _mask(mask)
    dim, nx, ny, nz = _dims(m)
    z, D = _species(z, D)
    ns = len(z)
    u = np.ascontiguousarray(u, dtype=np.float64)
    p = np.ascontiguousarray(psi_field, dtype=np.float64)
    if C is None:
        C = np.where(m[None] == 0, float(c0), 0.0) * np.ones((ns,) + m.shape)
    C = np.ascontiguousarray(C, dtype=np.float64).copy()
    if acc is None:
        acc = (np.zeros(ns), np.zeros(ns), np.zeros(ns))
    G, I, O = (np.ascontiguousarray(a, dtype=np.float64).copy() for a in acc)
    st = _load().orc_np_run(dim, nx, ny, nz, _ptr(m), int(lateral_walls), _ptr(u),
                            _ptr(p), ns, _ptr(z), _ptr(D), float(dx), float(Ka),
                            float(c0), thermal_voltage(T), float(dt),
                            int(n_steps), _ptr(C), _ptr(G), _ptr(I), _ptr(O))
    if st < 0:
        raise ValueError("orc_np_run rejected its arguments")
    return C, G, I, O


def np_operator(mask, u, psi_field, zi, Di, *, c0, dx=1e-7, Ka=1e-6, T=T_DEFAULT,
                lateral_walls=False):
    """The transport operator of one species (Eq. 3 with Eq. 6, the face rules
    of np_run): (1/dx) sum_f J_f(C) = A C - b.  Returns (A as a scipy CSR
    matrix, b)."""
    import scipy.sparse as sp
    m = _mask(mask)
    dim, nx, ny, nz = _dims(m)
    N = m.size
    u = np.ascontiguousarray(u, dtype=np.float64)
    p = np.ascontiguousarray(psi_field, dtype=np.float64)
    rows = np.zeros(7 * N, dtype=np.int64)
    cols = np.zeros(7 * N, dtype=np.int64)
    vals = np.zeros(7 * N)
    b = np.zeros(N)
    nnz = ctypes.c_long(0)
    st = _load().orc_np_operator(dim, nx, ny, nz, _ptr(m), int(lateral_walls), _ptr(u), _ptr(p),
                                 int(zi), float(Di), float(dx), float(Ka), float(c0),
                                 thermal_voltage(T), _ptr(rows), _ptr(cols), _ptr(vals),
                                 ctypes.byref(nnz), _ptr(b))
    if st < 0:
        raise ValueError("orc_np_operator rejected its arguments")
    k = nnz.value
    A = sp.csr_matrix((vals[:k], (rows[:k], cols[:k])), shape=(N, N))
    return A, b


def np_implicit_run(mask, u, psi_field, z, D, *, c0, dt, n_steps, dx=1e-7, Ka=1e-6,
                    T=T_DEFAULT, lateral_walls=False, C=None):
    """The implicit finite-volume transport of Sec. 2: backward Euler steps
    (I + dt A) C^{n+1} = C^n + dt b per species, solved by a sparse LU
    factorisation (a library primitive); the adsorbed, inflow and outflow
    accounts take the face fluxes at C^{n+1}, evaluated by np_run's face
    rules (one explicit evaluation of the fluxes, whose concentration update
    is discarded).  Starts from C = c0 in the pore cells unless C is given.
    Returns (C, Gamma, In, Out) like np_run."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    m = _mask(mask)
    z, D = _species(z, D)
    ns = len(z)
    N = m.size
    if C is None:
        C = np.where(m[None] == 0, float(c0), 0.0) * np.ones((ns,) + m.shape)
    C = np.array(C, dtype=np.float64).reshape(ns, N)
    solvers, rhs_b = [], []
    for k in range(ns):
        A, b = np_operator(m, u, psi_field, z[k], D[k], c0=c0, dx=dx, Ka=Ka, T=T,
                           lateral_walls=lateral_walls)
        M = (sp.identity(N, format="csr") + dt * A).tocsc()
        solvers.append(spla.splu(M))
        rhs_b.append(b)
    G, I, O = np.zeros(ns), np.zeros(ns), np.zeros(ns)
    for _ in range(n_steps):
        for k in range(ns):
            C[k] = solvers[k].solve(C[k] + dt * rhs_b[k])
        # the accounts of this step: the fluxes at C^{n+1}, times dt
        _, g, i, o = np_run(m, u, psi_field, z, D, c0=c0, dt=dt, n_steps=1, dx=dx, Ka=Ka, T=T,
                            lateral_walls=lateral_walls, C=C.reshape((ns,) + m.shape))
        G += g
        I += i
        O += o
    return C.reshape((ns,) + m.shape), G, I, O


def charge_coef(dx, eps_r=EPS_R_DEFAULT):
    """F dx^2 / (eps_r eps_0): turns sum_i z_i C_i (mol/m^3) into the charge
    term of the discrete Eq. 4 (volts)."""
    return FARADAY * dx * dx / (eps_r * EPS0)


def psi_src(mask, psi_s, src, *, lateral_walls=False, tol=1e-13, max_iter=1000000):
    """Eq. 4 with Dirichlet psi_s at solid faces, the inlet feed at 0 and the
    charge term ``src`` (volts, per cell: dx^2 rho_e / (eps_r eps_0)) on the
    right-hand side; Laplace operator."""
    m = _mask(mask)
    dim, nx, ny, nz = _dims(m)
    src = np.ascontiguousarray(src, dtype=np.float64)
    out = np.zeros(m.shape, dtype=np.float64)
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = _load().orc_psi_src(dim, nx, ny, nz, _ptr(m), int(lateral_walls), float(psi_s),
                             0.0, _ptr(src), float(tol), int(max_iter), _ptr(out),
                             ctypes.byref(it), ctypes.byref(rel))
    if st < 0:
        raise ValueError("orc_psi_src rejected its arguments")
    return out, it.value, rel.value


def pnp_run(mask, u, z, D, *, c0, dt, n_steps, K, psi_s, dx=1e-7, Ka=1e-6, T=T_DEFAULT,
            eps_r=EPS_R_DEFAULT, lateral_walls=False, psi_tol=1e-13, C=None):
    """Coupled Poisson-Nernst-Planck (Eq. 3-5): the potential is re-solved
    from the net charge of the current concentrations (Eq. 5) before every
    block of K explicit steps.  Starts from C = c0 in the pore cells unless C
    is given.  Returns ``(C, Gamma, In, Out, psi)`` with psi the last potential
    solved."""
    m = _mask(mask)
    dim, nx, ny, nz = _dims(m)
    z, D = _species(z, D)
    ns = len(z)
    u = np.ascontiguousarray(u, dtype=np.float64)
    if C is None:
        C = np.where(m[None] == 0, float(c0), 0.0) * np.ones((ns,) + m.shape)
    C = np.ascontiguousarray(C, dtype=np.float64).copy()
    G, I, O = np.zeros(ns), np.zeros(ns), np.zeros(ns)
    ps = np.zeros(m.shape, dtype=np.float64)
    st = _load().orc_pnp_run(dim, nx, ny, nz, _ptr(m), int(lateral_walls), _ptr(u), ns,
                             _ptr(z), _ptr(D), float(dx), float(Ka), float(c0),
                             thermal_voltage(T), float(dt), int(n_steps), int(K),
                             float(psi_s), charge_coef(dx, eps_r), float(psi_tol), _ptr(C),
                             _ptr(G), _ptr(I), _ptr(O), _ptr(ps))
    if st < 0:
        raise ValueError("orc_pnp_run rejected its arguments")
    return C, G, I, O, ps


# --------------------------------------------------------------------------
# Outputs (Sec. 4.1: outlet concentration, salt removal, averaged profiles)
# --------------------------------------------------------------------------
def outlet_concentration(mask, u, C):
    """Flux-weighted concentration over the pore cells of the outlet column:
    sum u_x C / sum u_x.  Falls back to the plain mean when sum u_x = 0."""
    m = _mask(mask)
    pore = m[..., -1] == 0
    ux = u[0][..., -1][pore]
    out = []
    for Ci in C:
        c = Ci[..., -1][pore]
        s = ux.sum()
        out.append(float((ux * c).sum() / s) if s != 0.0 else float(c.mean()))
    return np.array(out)


def salt_removal(c_in, c_out):
    """P_rm = (C_in - C_out) / C_in (Sec. 4.1)."""
    return (c_in - c_out) / c_in


def mass(mask, C, dx):
    """Dissolved amount per species: sum over pore cells of C dx^d (per metre
    of depth in 2D)."""
    m = _mask(mask)
    vol = dx ** m.ndim
    return np.array([float(Ci[m == 0].sum() * vol) for Ci in C])


def column_means(mask, C):
    """Mean over the pore cells of each x column (the vertically averaged
    profile of Fig. 6 and Fig. 9)."""
    m = _mask(mask)
    pore = (m == 0)
    axes = tuple(range(m.ndim - 1))
    cnt = pore.sum(axis=axes)
    out = []
    for Ci in C:
        s = np.where(pore, Ci, 0.0).sum(axis=axes)
        out.append(np.where(cnt > 0, s / np.maximum(cnt, 1), 0.0))
    return np.array(out)


def porosity(mask):
    """phi = pore cells / cells (Sec. 4)."""
    m = _mask(mask)
    return float(np.count_nonzero(m == 0)) / m.size


def interface_faces(mask, lateral_walls=False):
    """Voxel faces between a pore cell and a solid cell of the image (the
    staircase interface).  Faces across the inlet and outlet planes (x) are
    not interface; across the lateral image boundary the neighbour wraps
    periodically, unless the lateral boundary is a wall (then none)."""
    m = _mask(mask).astype(bool)
    total = 0
    for ax in range(m.ndim):
        x_axis = ax == m.ndim - 1
        n = m.shape[ax]
        for lo in range(n):
            hi = lo + 1
            if hi == n:
                if x_axis or lateral_walls:
                    continue
                hi = 0
            a = np.take(m, lo, axis=ax)
            b = np.take(m, hi, axis=ax)
            total += int(np.count_nonzero(a != b))
    return total


def specific_surface(mask, dx, lateral_walls=False):
    """s = pore-solid interface area / image volume (1/m; in 2D interface
    length / image area), the s of Sec. 4's l_c = pi / s."""
    m = _mask(mask)
    return interface_faces(m, lateral_walls) * dx ** (m.ndim - 1) / (m.size * dx ** m.ndim)


def derived(mask, u, C_out, *, c0, D, Ka, dx, dt, n_steps, lateral_walls=False):
    """The figures of Sec. 4 and Sec. 4.1 for a transport state: porosity phi,
    specific surface s, l_c = pi / s, the pore-mean velocity U = sum u_x /
    (N phi), elapsed time Delta t = n_steps dt, and per species Pe = U l_c / D,
    Da = Ka l_c / D, the salt removal P_rm = (C_in - C_out) / C_in (C_in the
    feed c0) and the adsorbed amount U A P_rm Delta t / (V_t phi) with A the
    inlet cross-section (ny dx per metre of depth in 2D, ny nz dx^2 in 3D) and
    V_t the electrode volume N dx^d."""
    m = _mask(mask)
    D = np.atleast_1d(np.asarray(D, dtype=np.float64))
    C_out = np.atleast_1d(np.asarray(C_out, dtype=np.float64))
    phi = porosity(m)
    s = specific_surface(m, dx, lateral_walls)
    l_c = np.pi / s
    U = float(np.asarray(u)[0][m == 0].sum()) / (m.size * phi)
    elapsed = n_steps * dt
    A = m.shape[0] * dx if m.ndim == 2 else m.shape[0] * m.shape[1] * dx * dx
    Vt = m.size * dx ** m.ndim
    P_rm = (c0 - C_out) / c0
    return dict(porosity=phi, specific_surface=s, l_c_m=l_c, U_mps=U, elapsed_s=elapsed,
                Pe=U * l_c / D, Da=Ka * l_c / D, removal=P_rm,
                amount=U * A * P_rm * elapsed / (Vt * phi))


def run_case(mask, *, mirror=True, lateral_walls=False, tau=1.0, force=1e-6,
             flow_tol=1e-8, check_every=100, max_flow_steps=2_000_000,
             U_target=1e-4, applied_V=1.0, c0=10.0, z=(1, -1),
             D=(1.33e-9, 2.03e-9), Ka=1e-6, dx=1e-7, T=T_DEFAULT,
             eps_r=EPS_R_DEFAULT, psi_mode="debye", lambda_D=None,
             psi_tol=1e-13, n_np_steps=2000, dt=None):
    """The whole path on one geometry: flow to steady state, velocity scaling,
    frozen potential (surface value -applied_V), time step, n_np_steps
    transport steps, then the outputs.  Returns a dict."""
    u_flow, steps, res, st = lbm(mask, mirror=mirror, lateral_walls=lateral_walls,
                                 tau=tau, force=force, tol=flow_tol,
                                 check_every=check_every, max_steps=max_flow_steps)
    u, U_lat = velocity_export(mask, u_flow, U_target)
    ps, it, rel = psi(mask, -applied_V, dx=dx, c_bulk=c0, T=T, eps_r=eps_r,
                      mode=psi_mode, lambda_D=lambda_D,
                      lateral_walls=lateral_walls, tol=psi_tol)
    if dt is None:
        dt = np_dt(mask, u, ps, z, D, dx=dx, Ka=Ka, T=T, lateral_walls=lateral_walls)
    C, G, I, O = np_run(mask, u, ps, z, D, c0=c0, dt=dt, n_steps=n_np_steps,
                        dx=dx, Ka=Ka, T=T, lateral_walls=lateral_walls)
    return dict(u_flow=u_flow, flow_steps=steps, flow_residual=res, flow_status=st,
                u=u, U_lattice=U_lat, psi=ps, psi_iters=it, psi_relres=rel, dt=dt,
                C=C, Gamma=G, In=I, Out=O,
                C_out=outlet_concentration(mask, u, C),
                M=mass(mask, C, dx), M0=mass(mask, np.where(np.asarray(mask)[None] == 0, c0, 0.0)
                                               * np.ones((len(z),) + np.asarray(mask).shape), dx))
