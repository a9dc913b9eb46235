"""The GPU radix sort (stage of the (tile, depth) sort) against numpy's stable argsort."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_06523_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def _keys(kind, n, rng):
    if kind == "uniform":
        return rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    if kind == "few":
        return rng.integers(0, 5, n).astype(np.uint32) * np.uint32(0x01010101)
    if kind == "equal":
        return np.full(n, 0xDEADBEEF, np.uint32)
    if kind == "sorted":
        return np.sort(rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32))
    if kind == "reversed":
        return np.sort(rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32))[::-1].copy()
    if kind == "floats":
        return rng.uniform(0.01, 300.0, n).astype(np.float32).view(np.uint32)
    raise ValueError(kind)


def _check(ctx, keys, begin, end):
    import torch
    n = len(keys)
    vals = np.arange(n, dtype=np.uint32) ^ np.uint32(0x5A5A5A5A)
    kd = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    vd = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    ctx.sort_pairs(kd, vd, begin, end)
    gk = kd.cpu().numpy().view(np.uint32)
    gv = vd.cpu().numpy().view(np.uint32)
    digit = (keys.astype(np.uint64) >> np.uint64(begin)) & np.uint64((1 << (end - begin)) - 1)
    o = np.argsort(digit, kind="stable")
    assert (gk == keys[o]).all()
    assert (gv == vals[o]).all()


@pytest.mark.parametrize("n", [1, 2, 31, 4095, 4096, 4097, 65536 + 3, 1_000_003])
@pytest.mark.parametrize("kind", ["uniform", "few", "equal", "sorted", "reversed", "floats"])
def test_sort_full_width(ctx, n, kind):
    rng = np.random.default_rng(n)
    _check(ctx, _keys(kind, n, rng), 0, 32)


@pytest.mark.parametrize("begin,end", [(0, 13), (0, 16), (8, 16), (3, 11), (16, 32), (0, 8)])
def test_sort_bit_ranges(ctx, begin, end):
    rng = np.random.default_rng(begin * 100 + end)
    _check(ctx, _keys("uniform", 300_001, rng), begin, end)


def test_sort_large(ctx):
    rng = np.random.default_rng(7)
    _check(ctx, _keys("floats", 20_000_017, rng), 0, 32)


def test_sort_empty(ctx):
    import torch
    k = torch.zeros(0, dtype=torch.int32, device="cuda")
    ctx.sort_pairs(k, k.clone(), 0, 32)
