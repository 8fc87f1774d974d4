"""The transport kernel's Philox4x32-10 on the device: the published
known-answer vectors, the oracle's Philox on random counters and keys, and
cuRAND's Philox4_32_10 generator called on the device."""
import os

import numpy as np
import pytest

import oracle
import paper_2509_05047_gb300 as psc

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_05047_gb300 import build
    build.build()


def test_device_philox_known_answers(gpu):
    rows = [[int(x, 16) for x in l.split()] for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    a = np.array(rows, dtype=np.uint64).astype(np.uint32)
    np.testing.assert_array_equal(psc.psc_check_philox(a[:, :6]), a[:, 6:])


def test_device_philox_equals_oracle(gpu):
    rng = np.random.default_rng(5)
    a = rng.integers(0, 1 << 32, size=(2000, 6), dtype=np.uint64).astype(np.uint32)
    got = psc.psc_check_philox(a)
    for i in range(0, 2000, 97):
        assert list(got[i]) == list(oracle.philox4x32_10(list(a[i, :4]), list(a[i, 4:])))


@pytest.mark.parametrize("seed,sub", [(0, 0), (12345, 7), ((1 << 63) + 99, (1 << 40) + 3)])
def test_device_philox_equals_curand(gpu, seed, sub):
    """cuRAND keys Philox4_32_10 with the 64-bit seed and puts the 64-bit
    subsequence in counter words 2 and 3; draw b uses counter word 0 = b."""
    n = 5
    cur = psc.psc_check_curand_philox(seed, sub, n)
    rows = np.array([[b, 0, sub & 0xFFFFFFFF, sub >> 32, seed & 0xFFFFFFFF, seed >> 32] for b in range(n)],
                    dtype=np.uint64).astype(np.uint32)
    np.testing.assert_array_equal(psc.psc_check_philox(rows), cur)


def test_check_calls_reject_bad_arguments(gpu):
    with pytest.raises(psc.PscError):
        psc.psc_check_curand_philox(1, 0, 0)
