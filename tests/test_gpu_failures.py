"""Host-side failure handling (no GPU fault is made): an allocator that
returns NULL on its k-th call, for every k that create_domain reaches, gives
CDI_ERR_OOM and leaves nothing allocated; an allocation failure inside a
sweep fails the call alone, frees what it took, and the domain still works."""
import ctypes

import numpy as np
import pytest

from paper_2110_13055_gb300 import cdi, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


class FailingAllocator:
    """Device memory from torch's caching allocator; the fail_at-th call
    (1-based; 0 = never) and every later one return NULL."""

    def __init__(self, fail_at=0):
        import torch
        self.torch = torch
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}

        def _alloc(nbytes, ctx):
            self.calls += 1
            if self.fail_at and self.calls >= self.fail_at:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), 0)
            self.live[p] = nbytes
            return p

        def _free(ptr, nbytes, ctx):
            assert ptr in self.live, "freed a block it never allocated"
            assert self.live.pop(ptr) == nbytes
            torch.cuda.caching_allocator_delete(ptr)

        self._a = cdi.ALLOC_FN(_alloc)
        self._f = cdi.FREE_FN(_free)
        self.table = cdi.cdi_allocator(self._a, self._f, None)


def _create(mask, alloc, prec=cdi.FP32_CPAIR):
    m = np.ascontiguousarray(mask, np.uint8)
    nz = 1 if m.ndim == 2 else m.shape[0]
    desc = cdi.cdi_domain_desc(m.ndim, m.shape[-1], m.shape[-2], nz, 1e-7, 0, 1, prec)
    return cdi.create_domain(desc, m, alloc.table, None)


@pytest.mark.parametrize("shape", [(23, 37), (9, 11, 13)])
def test_create_fails_cleanly_at_every_allocation(shape):
    mask = inputs.grain_pack(shape, 0.6, 1.5, 3.0, seed=41)[0]
    probe = FailingAllocator()
    h = _create(mask, probe)
    n_calls = probe.calls
    cdi.destroy_domain(h)
    assert n_calls > 10 and not probe.live
    for k in range(1, n_calls + 1):
        a = FailingAllocator(fail_at=k)
        with pytest.raises(cdi.CDIError) as e:
            _create(mask, a)
        assert e.value.status == 2, (k, str(e.value))      # CDI_ERR_OOM
        assert not a.live, (k, len(a.live))                 # nothing leaked


def test_sweep_allocation_failure_fails_alone():
    mask = inputs.grain_pack((23, 37), 0.6, 1.5, 3.0, seed=41)[0]
    a = FailingAllocator()
    h = _create(mask, a, prec=cdi.FP32)
    try:
        p = cdi.cdi_flow_params(1.0, 1e-6, 0.0, 100, 400, 1e-4)
        cdi.solve_flow(h, p)
        ep = cdi.cdi_elec_params(298.15, 78.5, 10.0, 1.5e-7, 0, 1e-12, 100000)
        before = len(a.live)
        a.fail_at = a.calls + 5          # fail inside the sweep's member allocations
        with pytest.raises(cdi.CDIError) as e:
            cdi.sweep_transport(h, [(1e-4, 1.0)] * 4, ep, (1, -1), (1.33e-9, 2.03e-9), 10.0,
                                1e-6, 10)
        assert e.value.status == 2
        assert len(a.live) == before     # the sweep gave back what it took
        a.fail_at = 0
        cdi.set_potential(h, 1.0, ep)
        cdi.init_transport(h, (1, -1), (1.33e-9, 2.03e-9), 10.0, 1e-6)
        cdi.step_transport(h, 20)
        G = cdi.query_adsorbed(h, 2)
        assert np.all(np.isfinite(G)) and np.all(G > 0)
    finally:
        cdi.destroy_domain(h)
    assert not a.live
