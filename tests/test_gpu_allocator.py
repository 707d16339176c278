"""GPU: handles whose device memory comes from the caller's allocator (lbve_create_ex).

- PyTorch's caching allocator: the handle's buffers show up in torch's accounting while it lives, the results
  are those of a cudaMalloc handle (bitwise, same sweep launch shape), and everything is returned on destroy;
- allocation failures (host-side fault injection: the callback returns NULL) give ENOMEM, with every block
  handed out so far returned, at create and in a later call, and the handle stays usable;
- memory not aligned to 256 bytes is refused; alloc without free is refused.
"""
import numpy as np
import pytest

from paper_1504_06123_gb300 import lbve as L

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32, F64 = L.LBVE_F32, L.LBVE_F64


def _descs():
    return [L.make_desc(L.LBVE_D2Q9, 3, 12, tau_lb=0.8, G_inf=0.01, tau=30.0, gamma_c=0.1, g=(2e-5, 0, 0), C=8,
                        B=3, precision=F64, hist_storage=F32),
            L.make_desc(L.LBVE_D2Q9, 2, 20, tau_lb=0.9, G_inf=0.005, tau=40.0, gamma_c=0.2, g=(1e-5, 0, 0), C=8,
                        B=3, precision=F64, hist_storage=F32)]


class Counting:
    """torch caching allocator with a count of live blocks and an optional failure after `fail_after` calls."""

    def __init__(self, fail_after=None, offset=0):
        self.live, self.calls, self.fail_after, self.offset = {}, 0, fail_after, offset
        self.allocator = L.make_allocator(self.alloc, self.free)

    def alloc(self, n, stream):
        self.calls += 1
        if self.fail_after is not None and self.calls > self.fail_after:
            return 0
        p = torch.cuda.caching_allocator_alloc(n + self.offset, torch.cuda.current_device(), stream)
        self.live[p + self.offset] = p
        return p + self.offset

    def free(self, ptr, stream):
        torch.cuda.caching_allocator_delete(self.live.pop(ptr))


def test_torch_caching_allocator_matches_cudamalloc():
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    a = L.Channel(_descs(), allocator=L.torch_allocator())
    held = torch.cuda.memory_allocated() - base
    assert held >= L.lbve_memory_bytes(a.h)
    b = L.Channel(_descs())                       # cudaMalloc
    S, _, mode = L.lbve_sweep_config(a.h)
    L.lbve_set_sweep_config(b.h, S, mode)
    for ch in (a, b):
        L.lbve_set_probes(ch.h, [5, 40], 2, 64)   # probe buffers from the allocator too
        ch.step(50)
    fa, fb = a.fields(), b.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    ta, va, _ = L.lbve_probe_read(a.h, 2, 2, 64)
    tb, vb, _ = L.lbve_probe_read(b.h, 2, 2, 64)
    assert np.array_equal(ta, tb) and np.array_equal(va, vb)
    a.close()
    b.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base


@pytest.mark.parametrize("fail_after", [0, 1, 5, 12])
def test_allocation_failure_at_create_returns_everything(fail_after):
    al = Counting(fail_after=fail_after)
    with pytest.raises(L.LbveError) as e:
        L.lbve_create_ex(_descs(), None, al.allocator)
    assert e.value.status == L.LBVE_ENOMEM
    assert al.live == {}
    assert al.calls == fail_after + 1


def test_allocation_failure_in_a_later_call_leaves_the_handle_usable():
    al = Counting()
    ch = L.Channel(_descs(), allocator=al.allocator)
    n_created = len(al.live)
    al.fail_after = al.calls                       # every further allocation fails
    with pytest.raises(L.LbveError) as e:
        L.lbve_set_probes(ch.h, [1, 2, 3], 1, 1000)
    assert e.value.status == L.LBVE_ENOMEM
    assert len(al.live) == n_created
    al.fail_after = None
    ch.step(20)                                     # still steps
    assert np.all(np.isfinite(ch.fields()["u"]))
    ch.close()
    assert al.live == {}


def test_fields_staging_failure_reports_enomem():
    al = Counting()
    ch = L.Channel(_descs(), allocator=al.allocator)
    al.fail_after = al.calls
    with pytest.raises(L.LbveError) as e:
        ch.fields()                                 # the host copy needs its staging buffer
    assert e.value.status == L.LBVE_ENOMEM
    al.fail_after = None
    assert np.all(np.isfinite(ch.fields()["u"]))
    ch.close()
    assert al.live == {}


def test_misaligned_or_incomplete_allocators_are_refused():
    al = Counting(offset=16)
    with pytest.raises(L.LbveError) as e:
        L.lbve_create_ex(_descs(), None, al.allocator)
    assert e.value.status == L.LBVE_ENOMEM
    assert al.live == {}
    half = L.lbve_allocator(L.ALLOC_FN(lambda n, s, c: None), L.FREE_FN(), None)
    with pytest.raises(L.LbveError) as e:
        L.lbve_create_ex(_descs(), None, half)
    assert e.value.status == L.LBVE_EINVAL
