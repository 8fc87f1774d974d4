"""The roofline measurement kernels (include/psc_peaks.h): every random
atomic add lands in the buffer, indices cover it uniformly, the gather runs,
and bad arguments are refused."""
import numpy as np
import pytest
from scipy import stats

import paper_2509_05047_gb300 as psc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_05047_gb300 import build
    build.build()
    return torch


def test_random_atomics_add_every_increment_uniformly(torch):
    buf = torch.zeros(1000, dtype=torch.int64, device="cuda")
    grid, block, k = 40, 128, 50
    psc.psc_peak_random_atomics(buf, grid, block, k, seed=3)
    torch.cuda.synchronize()
    h = buf.cpu().numpy()
    assert h.sum() == grid * block * k
    chi2 = ((h - h.mean()) ** 2 / h.mean()).sum()
    assert stats.chi2.sf(chi2, h.size - 1) > 1e-4


def test_random_gather_runs_and_leaves_the_sink(torch):
    table = torch.rand(1 << 20, device="cuda")
    sink = torch.full((1,), 7.0, device="cuda")
    psc.psc_peak_random_gather(table, sink, 64, 256, 64, seed=3)
    torch.cuda.synchronize()
    assert float(sink.item()) == 7.0


def test_peak_kernels_reject_bad_arguments(torch):
    buf = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(psc.PscError) as e:
        psc.psc_peak_random_atomics(buf, 1, 100, 1)  # block not a multiple of 32
    assert e.value.code == psc.PSC_EINVAL
    table = torch.rand(64, device="cuda")
    with pytest.raises(psc.PscError) as e:
        psc.psc_peak_random_gather(table, table[:1], 1, 32, 12)  # per_thread not a multiple of 8
    assert e.value.code == psc.PSC_EINVAL
