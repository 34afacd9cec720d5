"""Python binding of the C ABI in ``include/cdi.h`` (argument marshalling only).

Every function here has the name of the C entry point without its ``cdi_``
prefix and forwards to it through ctypes; all numerical work runs in the CUDA
kernels of ``libcdi.so``.  There is no CPU fallback: if the library is
missing, every call raises.  PyTorch, when present, provides the device
memory (its caching allocator) and the stream.

The ``Domain`` class wraps one ``cdi_domain`` handle for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

c_int, c_double, c_size_t, c_int64, c_void_p = (ctypes.c_int, ctypes.c_double,
                                                ctypes.c_size_t, ctypes.c_int64,
                                                ctypes.c_void_p)

FP64, FP32, FP32_SPLIT, BF16_POP, FP32_CPAIR = 0, 1, 2, 3, 4
FIELD_U_LATTICE, FIELD_U, FIELD_PSI, FIELD_C = 0, 1, 2, 3
STATUS = {0: "CDI_OK", 1: "CDI_ERR_INVALID_ARG", 2: "CDI_ERR_OOM", 3: "CDI_ERR_CUDA",
          4: "CDI_ERR_NOT_CONVERGED", 5: "CDI_ERR_TIMEOUT", 6: "CDI_ERR_STATE"}

ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_size_t, c_void_p)


class cdi_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", c_void_p)]


class cdi_domain_desc(ctypes.Structure):
    _fields_ = [("dim", c_int), ("nx", c_int), ("ny", c_int), ("nz", c_int),
                ("dx_m", c_double), ("lateral_walls", c_int), ("mirror_x", c_int),
                ("precision", c_int)]


class cdi_flow_params(ctypes.Structure):
    _fields_ = [("tau", c_double), ("force_lu", c_double), ("tol", c_double),
                ("check_every", c_int), ("max_steps", c_int64), ("U_target_mps", c_double)]


class cdi_elec_params(ctypes.Structure):
    _fields_ = [("T_K", c_double), ("eps_r", c_double), ("c_bulk_molm3", c_double),
                ("lambda_D_m", c_double), ("mode", c_int), ("tol", c_double),
                ("max_iter", c_int)]


class cdi_species(ctypes.Structure):
    _fields_ = [("z", c_int), ("D_m2s", c_double)]


class cdi_combo(ctypes.Structure):
    _fields_ = [("U_mps", c_double), ("applied_V", c_double)]


class cdi_derived(ctypes.Structure):
    _fields_ = [("porosity", c_double), ("specific_surface", c_double), ("l_c_m", c_double),
                ("U_mps", c_double), ("elapsed_s", c_double), ("Pe", c_double * 4),
                ("Da", c_double * 4), ("removal", c_double * 4), ("amount", c_double * 4)]


class cdi_timing(ctypes.Structure):
    _fields_ = [("flow_ms", c_double), ("flow_launches", c_int64),
                ("flow_check_ms", c_double), ("psi_ms", c_double), ("psi_iters", c_int64),
                ("np_ms", c_double), ("np_launches", c_int64), ("kernel_launches", c_int64),
                ("lbm_block", ctypes.c_int32), ("np_block", ctypes.c_int32),
                ("lbm_shape", ctypes.c_int32), ("np_shape", ctypes.c_int32)]


class CDIError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None

# (name, restype, argtypes) for every entry point of include/cdi.h
SIGNATURES = [
    ("cdi_create_domain", c_int, [ctypes.POINTER(cdi_domain_desc), c_void_p,
                                  ctypes.POINTER(cdi_allocator), c_void_p,
                                  ctypes.POINTER(c_void_p)]),
    ("cdi_solve_flow", c_int, [c_void_p, ctypes.POINTER(cdi_flow_params),
                               ctypes.POINTER(c_int64), ctypes.POINTER(c_double)]),
    ("cdi_solve_flow_batch", c_int, [c_void_p, c_int, ctypes.POINTER(cdi_flow_params),
                                     c_void_p, c_void_p, c_void_p]),
    ("cdi_set_velocity", c_int, [c_void_p, c_double]),
    ("cdi_set_potential", c_int, [c_void_p, c_double, ctypes.POINTER(cdi_elec_params),
                                  ctypes.POINTER(c_int), ctypes.POINTER(c_double)]),
    ("cdi_init_transport", c_int, [c_void_p, ctypes.POINTER(cdi_species), c_int, c_double,
                                   c_double, c_double, ctypes.POINTER(c_double)]),
    ("cdi_step_transport", c_int, [c_void_p, c_int64]),
    ("cdi_set_coupling", c_int, [c_void_p, c_int64]),
    ("cdi_set_implicit", c_int, [c_void_p, c_double, c_int]),
    ("cdi_set_launch_shapes", c_int, [c_void_p, c_int, c_int]),
    ("cdi_sweep_transport", c_int, [c_void_p, ctypes.POINTER(cdi_combo), c_int,
                                    ctypes.POINTER(cdi_elec_params),
                                    ctypes.POINTER(cdi_species), c_int, c_double, c_double,
                                    c_int64, c_void_p, c_void_p, c_void_p]),
    ("cdi_sweep_batch", c_int, [c_void_p, c_int, ctypes.POINTER(cdi_combo), c_int,
                                ctypes.POINTER(cdi_elec_params), ctypes.POINTER(cdi_species),
                                c_int, c_double, c_double, c_int64, c_void_p, c_void_p,
                                c_void_p]),
    ("cdi_query_adsorbed", c_int, [c_void_p, c_void_p]),
    ("cdi_query_outlet", c_int, [c_void_p, c_void_p]),
    ("cdi_query_mass_balance", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("cdi_query_column_means", c_int, [c_void_p, c_int, c_void_p]),
    ("cdi_query_derived", c_int, [c_void_p, ctypes.POINTER(cdi_derived)]),
    ("cdi_query_geometry", c_int, [c_void_p, ctypes.POINTER(c_double),
                                   ctypes.POINTER(c_double)]),
    ("cdi_copy_field", c_int, [c_void_p, c_int, c_void_p, c_size_t]),
    ("cdi_query_timing", c_int, [c_void_p, ctypes.POINTER(cdi_timing), c_int]),
    ("cdi_transport_sums_noalloc", c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int,
                                           c_int, c_int, c_double, c_void_p, c_void_p]),
    ("cdi_save_state", c_int, [c_void_p, c_void_p, ctypes.POINTER(c_size_t)]),
    ("cdi_load_state", c_int, [c_void_p, c_void_p, c_size_t]),
    ("cdi_last_error", ctypes.c_char_p, [c_void_p]),
    ("cdi_destroy_domain", None, [c_void_p]),
    ("cdi_version", c_int, []),
]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load ``libcdi.so`` (building it first only when asked)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built ({path}); run __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status, handle=None):
    if status != 0:
        msg = load().cdi_last_error(handle)
        raise CDIError(status, msg.decode() if msg else "")


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(c_void_p)


# ---------------------------------------------------------------------------
# one function per entry point
# ---------------------------------------------------------------------------
def version() -> int:
    return load().cdi_version()


def last_error(handle=None) -> str:
    m = load().cdi_last_error(handle)
    return m.decode() if m else ""


def create_domain(desc: cdi_domain_desc, mask: np.ndarray, allocator=None, stream=None):
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    out = c_void_p()
    st = load().cdi_create_domain(ctypes.byref(desc), _dptr(m),
                                  ctypes.byref(allocator) if allocator is not None else None,
                                  c_void_p(stream) if stream else None, ctypes.byref(out))
    _check(st, None)
    return out


def solve_flow(handle, params: cdi_flow_params, allow_not_converged=False):
    steps, res = c_int64(0), c_double(0.0)
    st = load().cdi_solve_flow(handle, ctypes.byref(params), ctypes.byref(steps),
                               ctypes.byref(res))
    if not (allow_not_converged and st == 4):
        _check(st, handle)
    return steps.value, res.value, st


def solve_flow_batch(handles, params: cdi_flow_params, allow_not_converged=False):
    """cdi_solve_flow_batch: returns (steps, residuals, statuses) per domain."""
    nd = len(handles)
    hs = (c_void_p * nd)(*[h.value if isinstance(h, c_void_p) else h for h in handles])
    steps, res = np.zeros(nd, np.int64), np.zeros(nd)
    st = np.zeros(nd, np.int32)
    rc = load().cdi_solve_flow_batch(hs, nd, ctypes.byref(params), _dptr(steps), _dptr(res),
                                     _dptr(st))
    if not (allow_not_converged and rc == 4):
        _check(rc, handles[0])
    return steps, res, st


def flow_batch(domains, *, tau=1.0, force=1e-6, tol=1e-8, check_every=100,
               max_steps=2_000_000, U_target=1e-4, allow_not_converged=False):
    """cdi_solve_flow_batch over Domain objects."""
    p = cdi_flow_params(float(tau), float(force), float(tol), int(check_every), int(max_steps),
                        float(U_target))
    return solve_flow_batch([d.handle for d in domains], p, allow_not_converged)


def set_velocity(handle, U_target: float):
    _check(load().cdi_set_velocity(handle, c_double(U_target)), handle)


def set_potential(handle, applied_V: float, params: cdi_elec_params):
    it, rel = c_int(0), c_double(0.0)
    _check(load().cdi_set_potential(handle, c_double(applied_V), ctypes.byref(params),
                                    ctypes.byref(it), ctypes.byref(rel)), handle)
    return it.value, rel.value


def init_transport(handle, z, D, c0, Ka, dt=0.0):
    n = len(z)
    sp = (cdi_species * n)(*[cdi_species(int(zz), float(dd)) for zz, dd in zip(z, D)])
    used = c_double(0.0)
    _check(load().cdi_init_transport(handle, sp, n, c_double(c0), c_double(Ka), c_double(dt),
                                     ctypes.byref(used)), handle)
    return used.value


def step_transport(handle, n_steps: int):
    _check(load().cdi_step_transport(handle, c_int64(n_steps)), handle)


def sweep_transport(handle, combos, params: cdi_elec_params, z, D, c0, Ka, n_steps):
    """combos: sequence of (U_mps, applied_V).  Returns (gamma, c_out, dt) with
    gamma and c_out of shape (n_combos, n_species)."""
    nc, ns = len(combos), len(z)
    cb = (cdi_combo * nc)(*[cdi_combo(float(U), float(V)) for U, V in combos])
    sp = (cdi_species * ns)(*[cdi_species(int(zz), float(dd)) for zz, dd in zip(z, D)])
    gam, cout, dt = np.zeros((nc, ns)), np.zeros((nc, ns)), np.zeros(nc)
    _check(load().cdi_sweep_transport(handle, cb, nc, ctypes.byref(params), sp, ns,
                                      c_double(c0), c_double(Ka), c_int64(n_steps), _dptr(gam),
                                      _dptr(cout), _dptr(dt)), handle)
    return gam, cout, dt


def sweep_batch(handles, combos, params: cdi_elec_params, z, D, c0, Ka, n_steps):
    """Every (domain, combination) member in one fused launch per step.
    Returns (gamma, c_out, dt) of shapes (n_doms, n_combos, n_species) and
    (n_doms, n_combos)."""
    nd, nc, ns = len(handles), len(combos), len(z)
    hs = (c_void_p * nd)(*[h.value if isinstance(h, c_void_p) else h for h in handles])
    cb = (cdi_combo * nc)(*[cdi_combo(float(U), float(V)) for U, V in combos])
    sp = (cdi_species * ns)(*[cdi_species(int(zz), float(dd)) for zz, dd in zip(z, D)])
    gam, cout, dt = np.zeros((nd, nc, ns)), np.zeros((nd, nc, ns)), np.zeros((nd, nc))
    _check(load().cdi_sweep_batch(hs, nd, cb, nc, ctypes.byref(params), sp, ns, c_double(c0),
                                  c_double(Ka), c_int64(n_steps), _dptr(gam), _dptr(cout),
                                  _dptr(dt)), handles[0])
    return gam, cout, dt


def batch(domains, combos, *, z=(1, -1), D=(1.33e-9, 2.03e-9), c0=10.0, Ka=1e-6, n_steps=5000,
          T=298.15, eps_r=78.5, c_bulk=None, lambda_D=0.0, mode="debye", tol=1e-12,
          max_iter=100000):
    """cdi_sweep_batch over Domain objects (each with a solved flow)."""
    p = cdi_elec_params(float(T), float(eps_r), float(c0 if c_bulk is None else c_bulk),
                        float(lambda_D or 0.0), 0 if mode == "debye" else 1, float(tol),
                        int(max_iter))
    for d in domains:
        d.ns = 0
    return sweep_batch([d.handle for d in domains], combos, p, z, D, c0, Ka, n_steps)


def set_implicit(handle, tol: float, max_iter: int = 1000):
    _check(load().cdi_set_implicit(handle, c_double(tol), c_int(max_iter)), handle)


def set_launch_shapes(handle, lbm_shape: int = -1, np_shape: int = -1):
    _check(load().cdi_set_launch_shapes(handle, c_int(lbm_shape), c_int(np_shape)), handle)


def set_coupling(handle, every_steps: int):
    _check(load().cdi_set_coupling(handle, c_int64(every_steps)), handle)


def save_state(handle) -> bytes:
    n = c_size_t(0)
    _check(load().cdi_save_state(handle, None, ctypes.byref(n)), handle)
    buf = ctypes.create_string_buffer(n.value)
    _check(load().cdi_save_state(handle, buf, ctypes.byref(n)), handle)
    return buf.raw[:n.value]


def load_state(handle, state: bytes):
    buf = ctypes.create_string_buffer(state, len(state))
    _check(load().cdi_load_state(handle, buf, c_size_t(len(state))), handle)


def query_adsorbed(handle, ns: int) -> np.ndarray:
    out = np.zeros(ns)
    _check(load().cdi_query_adsorbed(handle, _dptr(out)), handle)
    return out


def query_outlet(handle, ns: int) -> np.ndarray:
    out = np.zeros(ns)
    _check(load().cdi_query_outlet(handle, _dptr(out)), handle)
    return out


def query_mass_balance(handle, ns: int):
    M, G, I, O = (np.zeros(ns) for _ in range(4))
    _check(load().cdi_query_mass_balance(handle, _dptr(M), _dptr(G), _dptr(I), _dptr(O)),
           handle)
    return M, G, I, O


def query_geometry(handle):
    phi, s = c_double(0.0), c_double(0.0)
    _check(load().cdi_query_geometry(handle, ctypes.byref(phi), ctypes.byref(s)), handle)
    return phi.value, s.value


def query_derived(handle, ns: int) -> dict:
    """Pe, Da, l_c, U, salt removal and the adsorbed-amount figure of Sec. 4
    and 4.1 (per-species entries cut to the domain's species)."""
    d = cdi_derived()
    _check(load().cdi_query_derived(handle, ctypes.byref(d)), handle)
    out = {}
    for name, _ in cdi_derived._fields_:
        v = getattr(d, name)
        out[name] = np.array(v[:ns]) if not isinstance(v, float) else v
    return out


def query_column_means(handle, species: int, nx: int) -> np.ndarray:
    out = np.zeros(nx)
    _check(load().cdi_query_column_means(handle, species, _dptr(out)), handle)
    return out


def copy_field(handle, field: int, count: int) -> np.ndarray:
    out = np.zeros(count)
    _check(load().cdi_copy_field(handle, field, _dptr(out), c_size_t(count)), handle)
    return out


def query_timing(handle, reset=False) -> dict:
    t = cdi_timing()
    _check(load().cdi_query_timing(handle, ctypes.byref(t), int(bool(reset))), handle)
    return {name: getattr(t, name) for name, _ in cdi_timing._fields_}


def transport_sums_noalloc(C_ptr, ux_ptr, mask_ptr, dim, nx, ny, nz, n_species, dx, out_ptr,
                           stream=None):
    """Dissolved amount and outlet concentration of caller-owned device
    arrays (raw device pointers) without any allocation by the library; for
    callers that keep every device byte in their own memory pool.  See
    ``cdi_transport_sums_noalloc`` in include/cdi.h."""
    _check(load().cdi_transport_sums_noalloc(
        c_void_p(C_ptr), c_void_p(ux_ptr), c_void_p(mask_ptr), dim, nx, ny, nz, n_species,
        c_double(dx), c_void_p(out_ptr), c_void_p(stream) if stream else None), None)


def destroy_domain(handle):
    if handle:
        load().cdi_destroy_domain(handle)


# ---------------------------------------------------------------------------
# torch-backed device memory and stream
# ---------------------------------------------------------------------------
class TorchResources:
    """A torch CUDA stream plus an allocator table routing the library's
    device allocations to torch's caching allocator on that stream."""

    def __init__(self, device=0):
        import torch
        self.torch = torch
        self.device = device
        self.stream = torch.cuda.Stream(device=device)
        self._live = {}

        def _alloc(nbytes, ctx):
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                       self.stream)
            except Exception:  # out of memory: the library reports CDI_ERR_OOM
                return None
            self._live[p] = nbytes
            return p

        def _free(ptr, nbytes, ctx):
            if ptr in self._live:
                del self._live[ptr]
                torch.cuda.caching_allocator_delete(ptr)

        self._alloc_fn = ALLOC_FN(_alloc)
        self._free_fn = FREE_FN(_free)
        self.allocator = cdi_allocator(self._alloc_fn, self._free_fn, None)

    @property
    def stream_handle(self) -> int:
        return self.stream.cuda_stream


class Domain:
    """One voxel image: create, solve the flow, set the potential, run the
    transport, query.  Arrays follow the mask's (ny, nx) / (nz, ny, nx)."""

    def __init__(self, mask, *, dx=1e-7, precision=FP64, mirror=True, lateral_walls=False,
                 torch_resources: TorchResources | None = None, stream=None):
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        self.shape = m.shape
        self.dim = m.ndim
        nz = 1 if m.ndim == 2 else m.shape[0]
        ny, nx = m.shape[-2], m.shape[-1]
        self.nx, self.ny, self.nz = nx, ny, nz
        self.NX = 2 * nx if mirror else nx
        self.dx = dx
        self.precision = precision
        self.ns = 0
        self.res = torch_resources
        desc = cdi_domain_desc(self.dim, nx, ny, nz, float(dx), int(bool(lateral_walls)),
                               int(bool(mirror)), int(precision))
        alloc = torch_resources.allocator if torch_resources else None
        st = stream if stream is not None else (
            torch_resources.stream_handle if torch_resources else None)
        self.handle = create_domain(desc, m, alloc, st)

    def close(self):
        if self.handle:
            destroy_domain(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve_flow(self, *, tau=1.0, force=1e-6, tol=1e-8, check_every=100,
                   max_steps=2_000_000, U_target=1e-4, allow_not_converged=False):
        p = cdi_flow_params(float(tau), float(force), float(tol), int(check_every),
                            int(max_steps), float(U_target))
        return solve_flow(self.handle, p, allow_not_converged)

    def set_velocity(self, U_target):
        set_velocity(self.handle, U_target)

    def set_potential(self, applied_V, *, T=298.15, eps_r=78.5, c_bulk=10.0, lambda_D=0.0,
                      mode="debye", tol=1e-12, max_iter=100000):
        p = cdi_elec_params(float(T), float(eps_r), float(c_bulk), float(lambda_D or 0.0),
                            {"debye": 0, "laplace": 1, "pb": 2}[mode], float(tol),
                            int(max_iter))
        return set_potential(self.handle, applied_V, p)

    def init_transport(self, z=(1, -1), D=(1.33e-9, 2.03e-9), c0=10.0, Ka=1e-6, dt=0.0):
        self.ns = len(z)
        return init_transport(self.handle, z, D, c0, Ka, dt)

    def step(self, n):
        step_transport(self.handle, n)

    def sweep(self, combos, *, z=(1, -1), D=(1.33e-9, 2.03e-9), c0=10.0, Ka=1e-6,
              n_steps=5000, T=298.15, eps_r=78.5, c_bulk=None, lambda_D=0.0, mode="debye",
              tol=1e-12, max_iter=100000):
        """Batched transport over (U_mps, applied_V) combinations on the solved
        flow; see cdi_sweep_transport."""
        p = cdi_elec_params(float(T), float(eps_r), float(c0 if c_bulk is None else c_bulk),
                            float(lambda_D or 0.0), 0 if mode == "debye" else 1, float(tol),
                            int(max_iter))
        self.ns = 0
        return sweep_transport(self.handle, combos, p, z, D, c0, Ka, n_steps)

    def adsorbed(self):
        return query_adsorbed(self.handle, self.ns)

    def outlet(self):
        return query_outlet(self.handle, self.ns)

    def mass_balance(self):
        return query_mass_balance(self.handle, self.ns)

    def column_means(self, species):
        return query_column_means(self.handle, species, self.nx)

    def geometry(self):
        """(porosity, specific surface in 1/m)."""
        return query_geometry(self.handle)

    def derived(self):
        """Pe, Da, l_c, U, salt removal and adsorbed amount (Sec. 4, 4.1)."""
        return query_derived(self.handle, self.ns)

    def u_lattice(self):
        flow_shape = (self.NX,) if self.dim == 2 else (self.NX,)
        a = copy_field(self.handle, FIELD_U_LATTICE, self.dim * self.nz * self.ny * self.NX)
        return a.reshape((self.dim,) + self.shape[:-1] + flow_shape)

    def u(self):
        a = copy_field(self.handle, FIELD_U, self.dim * self.nz * self.ny * self.nx)
        return a.reshape((self.dim,) + self.shape)

    def psi(self):
        return copy_field(self.handle, FIELD_PSI, self.nz * self.ny * self.nx).reshape(self.shape)

    def C(self):
        n = self.nz * self.ny * self.nx
        return np.stack([copy_field(self.handle, FIELD_C + k, n).reshape(self.shape)
                         for k in range(self.ns)])

    def timing(self, reset=False):
        return query_timing(self.handle, reset)

    def set_implicit(self, tol: float = 1e-12, max_iter: int = 1000):
        """Backward Euler transport steps (Sec. 2's implicit finite volumes),
        solved to the relative residual tol; tol <= 0 returns to explicit
        steps."""
        set_implicit(self.handle, tol, max_iter)

    def set_launch_shapes(self, lbm_shape: int = -1, np_shape: int = -1):
        """Fix the launch shape of the LBM step (0-5) and of the transport
        step (0-9); -1 leaves it to the autotuner.  Every shape computes the
        same bits."""
        set_launch_shapes(self.handle, lbm_shape, np_shape)

    def set_coupling(self, every_steps: int):
        """Re-solve the potential from the net charge every ``every_steps``
        transport steps (Eq. 3-5); 0 freezes it."""
        set_coupling(self.handle, every_steps)

    def save_state(self) -> bytes:
        return save_state(self.handle)

    def load_state(self, state: bytes):
        load_state(self.handle, state)
        # species count from the state's header (int32 at byte 76)
        self.ns = int.from_bytes(state[76:80], "little", signed=True)
