"""psfs_gather_rows, the measurement of the gather rate that bounds the
fusion kernels: every word of every indexed row is read exactly once, indices
outside the rows are skipped, and the XOR of all words read matches the XOR
computed on the host (bit-exact), for 32- and 64-byte rows, ragged counts and
a side stream."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1311_6811_gb300 import psfs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    psfs.load()


def _xor_rows(words: np.ndarray, idx: np.ndarray) -> int:
    keep = idx[(idx >= 0) & (idx < words.shape[0])]
    if keep.size == 0:
        return 0
    return int(np.bitwise_xor.reduce(words[keep].reshape(-1).view(np.uint32)))


@pytest.mark.parametrize("record_bytes", [32, 64])
@pytest.mark.parametrize("n", [0, 1, 31, 33, 1000, 250_007])
def test_checksum_equals_host_xor(record_bytes, n):
    rng = np.random.default_rng(7 + n + record_bytes)
    n_rows = 40_000
    words = rng.integers(0, 2**32, size=(n_rows, record_bytes // 4), dtype=np.uint64).astype(np.uint32)
    # rows repeat, and a few indices fall outside the rows on either side
    idx = rng.integers(-50, n_rows + 50, size=n).astype(np.int32)
    rows = torch.from_numpy(words.view(np.int32)).cuda()
    d_idx = torch.from_numpy(idx).cuda()
    ck = torch.zeros(1, dtype=torch.int32, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    psfs.psfs_gather_rows(rows, record_bytes, d_idx, ck, stream=side)
    side.synchronize()
    got = int(ck.item()) & 0xFFFFFFFF
    assert got == _xor_rows(words, idx)


def test_checksum_accumulates_across_calls():
    rng = np.random.default_rng(3)
    words = rng.integers(0, 2**32, size=(1000, 16), dtype=np.uint64).astype(np.uint32)
    idx = rng.integers(0, 1000, size=777).astype(np.int32)
    rows = torch.from_numpy(words.view(np.int32)).cuda()
    d_idx = torch.from_numpy(idx).cuda()
    ck = torch.zeros(1, dtype=torch.int32, device="cuda")
    psfs.psfs_gather_rows(rows, 64, d_idx, ck)
    psfs.psfs_gather_rows(rows, 64, d_idx, ck)   # the same rows again: the XOR returns to 0
    torch.cuda.synchronize()
    assert int(ck.item()) == 0
