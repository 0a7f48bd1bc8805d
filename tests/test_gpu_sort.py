"""The broad phase's radix sort (Section "Broad-Phase": boxes sorted by their
minimum; the cell sweep sorts (cell, minimum) keys of the box copies) against
numpy's stable sort, through the C ABI: keys and values bit for bit, over
several tiles of 4,096 keys and a ragged tail, with digits that are the same
for every key (passes skipped in pairs) and digits that are not, 4- and
8-byte keys, a count read from device memory, and the degenerate sizes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TILE = 4096


@pytest.fixture(scope="module")
def ctx():
    from paper_2112_06300_gb300 import build
    build.build()
    global ccd
    from paper_2112_06300_gb300 import ccd
    c = ccd.CCD(0)
    yield c
    c.close()


def run_sort(c, keys, key_bits, n_cap=None, skip_all=False):
    n = len(keys)
    vals = np.arange(n, dtype=np.uint32)[::-1].copy()          # values: a permutation, reversed
    kd = torch.from_numpy(keys.view(np.int64 if keys.dtype.itemsize == 8 else np.int32).copy()).cuda()
    vd = torch.from_numpy(vals.view(np.int32)).cuda()
    st = ccd.ccd_selftest_radix_sort(c.ctx, kd, vd, key_bits=key_bits, n_cap=n_cap, skip_all=skip_all)
    assert st == 0
    ko = kd.cpu().numpy().view(keys.dtype)
    vo = vd.cpu().numpy().view(np.uint32)
    bits = key_bits if key_bits else 8 * keys.dtype.itemsize
    mask = np.array((1 << bits) - 1 if bits < 64 else (1 << 64) - 1, dtype=np.uint64).astype(keys.dtype)
    order = np.argsort(keys & mask, kind="stable")
    np.testing.assert_array_equal(ko, keys[order])
    np.testing.assert_array_equal(vo, vals[order])


@pytest.mark.parametrize("n", [0, 1, 31, TILE - 1, TILE, 3 * TILE + 777])
def test_sizes(ctx, n):
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 1 << 56, n, dtype=np.uint64)
    run_sort(ctx, keys, 56)


@pytest.mark.parametrize("skip_all", [False, True])
@pytest.mark.parametrize("high", [20, 40, 48, 56, 64])
def test_constant_digits(ctx, high, skip_all):
    """Keys below 2^high: digits at and above high/8 are the same for every
    key (4, 2, 1, 0 and 0 of the 7 passes of a 56-bit sort, or of 8); those
    passes are skipped in pairs, or all of them (the cell sort's mode, the
    result's buffers then named on the device)."""
    rng = np.random.default_rng(high)
    n = 5 * TILE + 123
    keys = rng.integers(0, 1 << min(high, 63), n, dtype=np.uint64)
    if high == 64:
        keys = keys * np.uint64(2) + rng.integers(0, 2, n, dtype=np.uint64)
    run_sort(ctx, keys, 0 if high == 64 else 56, skip_all=skip_all)


def test_many_duplicates_cell_keys(ctx):
    """(cell << 32 | ordered minimum) keys as the cell sweep makes them:
    few cells, minima with many ties; stability decides the order of equal
    keys (values are the index, reversed)."""
    rng = np.random.default_rng(7)
    n = 200_000
    cell = rng.integers(0, 300, n, dtype=np.uint64)
    mn = rng.integers(0x3F000000, 0x3F000040, n, dtype=np.uint64)
    run_sort(ctx, (cell << np.uint64(32)) | mn, 56)
    run_sort(ctx, (cell << np.uint64(32)) | mn, 56, n_cap=n + 3 * TILE, skip_all=True)


@pytest.mark.parametrize("skip_all", [False, True])
def test_all_equal(ctx, skip_all):
    run_sort(ctx, np.full(2 * TILE + 5, 0x123456789A, dtype=np.uint64), 56, skip_all=skip_all)


@pytest.mark.parametrize("key_bits", [0, 24])
def test_four_byte_keys(ctx, key_bits):
    rng = np.random.default_rng(3)
    keys = rng.integers(0, 1 << 32, 4 * TILE + 99, dtype=np.uint64).astype(np.uint32)
    run_sort(ctx, keys, key_bits)


def test_count_from_device(ctx):
    """Launch sized for n_cap, count n read on the device (the cell-copy sort)."""
    rng = np.random.default_rng(11)
    keys = rng.integers(0, 1 << 56, 3 * TILE + 1, dtype=np.uint64)
    run_sort(ctx, keys, 56, n_cap=9 * TILE)


def test_large_lookback_chain(ctx):
    """About 730 tiles: the cross-tile walk-back over more tiles than are
    resident at once."""
    rng = np.random.default_rng(5)
    keys = rng.integers(0, 1 << 56, 3_000_000, dtype=np.uint64)
    run_sort(ctx, keys, 56)
