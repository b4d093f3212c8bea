"""The host-memory bandwidth probe (host only): it touches exactly its buffer, the copy op
copies, and bad arguments are refused (CPU only)."""
import numpy as np
import pytest

import paper_2604_22228_gb300 as mpt
from paper_2604_22228_gb300 import build


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def test_ops_and_rates():
    n = 8 << 20
    b = np.zeros(n + 128, dtype=np.uint8)
    body = b[64:64 + n]
    body[: n // 2] = np.arange(n // 2, dtype=np.uint64).astype(np.uint8)
    g = mpt.mpt_host_bandwidth(body.ctypes.data, n, 4, 2, 1)  # copy first half into second
    assert g > 0
    assert np.array_equal(body[n // 2:], body[: n // 2])
    assert (b[:64] == 0).all() and (b[64 + n:] == 0).all()  # nothing outside the buffer
    assert mpt.mpt_host_bandwidth(body.ctypes.data, n, 3, 1, 1) > 0  # write
    assert (b[:64] == 0).all() and (b[64 + n:] == 0).all()
    assert mpt.mpt_host_bandwidth(body.ctypes.data, n, 2, 0, 2) > 0  # read


@pytest.mark.parametrize("args", [(1, 9, 1), (0, 0, 1), (2000, 0, 1)])
def test_bad_arguments(args):
    b = np.zeros(1 << 20, dtype=np.uint8)
    threads, op, reps = args
    with pytest.raises(mpt.MptError) as e:
        mpt.mpt_host_bandwidth(b.ctypes.data, b.size, threads, op, reps)
    assert e.value.status == mpt.MPT_EINVAL


def test_too_small_for_the_threads():
    b = np.zeros(16 << 10, dtype=np.uint8)
    with pytest.raises(mpt.MptError):
        mpt.mpt_host_bandwidth(b.ctypes.data, b.size, 8, 0, 1)
