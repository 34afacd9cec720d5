"""The allocation-free transport sums (``cdi_transport_sums_noalloc``).

Some callers cannot let a library allocate device memory: they keep every
device byte in their own pool or under a fixed budget, or they cannot afford
the device-wide synchronisation of a cudaMalloc/cudaFree in the middle of
their work.  This entry point computes the dissolved amount and the outlet
concentration of device arrays the caller owns, using only a fixed static
scratch array inside the library.  Its results must equal those of the
domain queries (which use the domain's allocated scratch), call after call.

This file is collected last so that a run stopping at the first failure has
run every other test first.
"""
import numpy as np
import pytest

from paper_2110_13055_gb300 import cdi, inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-11  # the FP64 tolerance of the parity tests


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def _noalloc(C, ux, mask, dx=1e-7):
    """Two calls in a row of the allocation-free sums on device copies of the
    host arrays; returns both results."""
    import torch
    ns = C.shape[0]
    dim = mask.ndim
    nz = 1 if dim == 2 else mask.shape[0]
    ny, nx = mask.shape[-2], mask.shape[-1]
    dev = torch.device("cuda", 0)
    Ct = torch.tensor(C, dtype=torch.float64, device=dev).contiguous()
    ut = torch.tensor(ux, dtype=torch.float64, device=dev).contiguous()
    mk = torch.tensor(mask, dtype=torch.uint8, device=dev).contiguous()
    out = torch.empty(2 * ns, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    got = []
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        out.fill_(float("nan"))
        cdi.transport_sums_noalloc(Ct.data_ptr(), ut.data_ptr(), mk.data_ptr(), dim, nx, ny,
                                   nz, ns, dx, out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        got.append(out.cpu().numpy())
    return got


def _domain_run(mask, U):
    with cdi.Domain(mask, precision=cdi.FP64) as d:
        d.solve_flow(tol=0.0, max_steps=400, U_target=U)
        d.set_potential(1.0, c_bulk=10.0, lambda_D=1.5e-7, tol=1e-13)
        d.init_transport(c0=10.0, Ka=1e-6)
        d.step(300)
        M_ref, _, _, _ = d.mass_balance()
        return d.C(), d.u(), M_ref, d.outlet()


@pytest.mark.parametrize("shape", [(23, 37), (9, 11, 13)])
def test_noalloc_sums_match_domain_queries_on_repeated_calls(shape):
    mask = inputs.grain_pack(shape, 0.62, 2.0, 4.5 if len(shape) == 2 else 3.0, seed=9)[0]
    C, u, M_ref, Cout_ref = _domain_run(mask, 1e-4)
    ns = C.shape[0]
    for got in _noalloc(C, u[0], mask):
        np.testing.assert_allclose(got[:ns], M_ref, rtol=TOL64)
        np.testing.assert_allclose(got[ns:], Cout_ref, rtol=TOL64)


def test_noalloc_plain_outlet_mean_without_flow():
    """With no flow the outlet concentration falls back to the plain mean
    over the outlet column's pore cells (checked against numpy)."""
    mask = inputs.grain_pack((23, 37), 0.62, 2.0, 4.5, seed=9)[0]
    C, u, M_ref, Cout_ref = _domain_run(mask, 0.0)
    assert np.all(u == 0.0)
    ns = C.shape[0]
    plain = [C[k][:, -1][mask[:, -1] == 0].mean() for k in range(ns)]
    for got in _noalloc(C, u[0], mask):
        np.testing.assert_allclose(got[:ns], M_ref, rtol=TOL64)
        np.testing.assert_allclose(got[ns:], plain, rtol=TOL64)
        np.testing.assert_allclose(got[ns:], Cout_ref, rtol=TOL64)


def test_noalloc_rejects_more_species_than_the_scratch_holds():
    import torch
    dev = torch.device("cuda", 0)
    buf = torch.zeros(64, dtype=torch.float64, device=dev)
    mk = torch.zeros(8, dtype=torch.uint8, device=dev)
    with pytest.raises(cdi.CDIError) as e:
        cdi.transport_sums_noalloc(buf.data_ptr(), buf.data_ptr(), mk.data_ptr(), 2, 4, 2, 1,
                                   5, 1e-7, buf.data_ptr())
    assert e.value.status == 1
    assert "n_species" in str(e.value)
