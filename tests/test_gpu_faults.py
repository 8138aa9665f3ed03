"""Fault injection on the host side of a GPU context: an allocator callback
that refuses memory.  The failure comes from the callback; nothing faults on
the device."""
import ctypes as C

import pytest

from workloads import make_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_10487_gb300 import build
    build.build()
    import paper_2006_10487_gb300 as H
    return H


class CountingAllocator:
    """Device memory from torch's caching allocator; refuses every request
    after the first `grant` (None: never refuses)."""

    def __init__(self, H, grant=None):
        import torch
        self.torch, self.dev = torch, torch.cuda.current_device()
        self.grant, self.calls, self.live = grant, 0, {}
        self.fns = (H.ALLOC_FN(self._alloc), H.FREE_FN(self._free))

    def _alloc(self, size, _ctx):
        self.calls += 1
        if self.grant is not None and self.calls > self.grant:
            return None
        p = self.torch.cuda.caching_allocator_alloc(int(size), self.dev, self.torch.cuda.current_stream(self.dev))
        self.live[p] = size
        return p

    def _free(self, ptr, _ctx):
        self.torch.cuda.caching_allocator_delete(ptr)
        self.live.pop(ptr)


def _create(H, case, allocator):
    import torch
    lv, m, o, keep = H._marshal(case, precision="fp32", stream=torch.cuda.current_stream().cuda_stream,
                                allocator=allocator.fns)
    ctx = C.c_void_p()
    rc = H.lib().hlbm_create(lv, case.n_levels, C.byref(m), case.Re, case.Ma, case.aoa_deg, C.byref(o),
                             C.byref(ctx))
    return rc, ctx


def test_allocator_failure_is_reported_and_nothing_leaks(H):
    """A refusal at the first, a middle or the last device allocation of
    hlbm_create gives HLBM_ENOMEM and no context, and every block the
    callback did hand out is given back (hlbm_create itself gives back the
    tables of the finite-volume tiling its autotuner did not keep)."""
    case = make_case("hlbm_mini2")
    full = CountingAllocator(H)
    rc, ctx = _create(H, case, full)
    assert rc == H.HLBM_OK and ctx.value
    n = full.calls
    assert n > 3 and 0 < len(full.live) <= n
    H.lib().hlbm_destroy(ctx)
    assert not full.live
    for grant in (0, n // 2, n - 1):
        a = CountingAllocator(H, grant)
        rc, ctx = _create(H, case, a)
        assert rc == H.HLBM_ENOMEM and not ctx.value, grant
        assert "alloc" in H.hlbm_last_error(None)
        assert a.calls == grant + 1 and not a.live, grant
    # the device stays usable afterwards
    s = H.Solver(case, precision="fp32")
    s.step(2)
    assert len(s.forces()[0]) == 2
