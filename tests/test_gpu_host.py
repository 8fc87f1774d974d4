"""Page-locked huge-page host buffers of the C ABI (psc_host_alloc /
psc_host_free): registration, copies in both directions, lifetime through
the binding, and errors."""
import numpy as np
import pytest

import paper_2509_05047_gb300 as psc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_05047_gb300 import build
    build.build()
    return torch


def test_host_tensor_is_pinned_and_round_trips(cuda):
    torch = cuda
    h = psc.host_tensor((3, 1000, 777), torch.float64)
    assert h.is_pinned() and h.shape == (3, 1000, 777)
    d = torch.randn(h.shape, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())   # d is written on the current stream
    with torch.cuda.stream(s):
        h.copy_(d, non_blocking=True)
    s.synchronize()
    assert torch.equal(h, d.cpu())
    back = torch.empty_like(d)
    back.copy_(h, non_blocking=True)
    torch.cuda.synchronize()
    assert torch.equal(back, d)


def test_host_alloc_rounds_to_huge_pages_and_frees(cuda):
    p = psc.psc_host_alloc(1)
    q = psc.psc_host_alloc(5 << 20)
    assert p != q and p % 4096 == 0 and q % 4096 == 0
    psc.psc_host_free(p)
    psc.psc_host_free(q)
    with pytest.raises(psc.PscError) as e:
        psc.psc_host_free(q)  # already freed
    assert e.value.code == psc.PSC_EINVAL


def test_host_alloc_rejects_bad_arguments(cuda):
    with pytest.raises(psc.PscError) as e:
        psc.psc_host_alloc(0)
    assert e.value.code == psc.PSC_EINVAL
    buf = np.zeros(16)
    with pytest.raises(psc.PscError) as e:
        psc.psc_host_free(buf.ctypes.data)  # not a buffer of psc_host_alloc
    assert e.value.code == psc.PSC_EINVAL
