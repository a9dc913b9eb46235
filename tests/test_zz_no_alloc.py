"""v3dg_sort_pairs_noalloc: the sort for callers that cannot allocate device memory.

Hosts that own every device allocation (an engine that reserves its pools at start-up, a
real-time loop where cudaMalloc would stall a frame) call this variant; it sorts with a fixed
scratch array inside the library instead of allocating.  Its output must equal that of
v3dg_sort_pairs, bit for bit, call after call.  This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_06523_gb300 import _native
    return _native


def _sorted_with_existing(keys, vals, begin, end):
    import torch
    from paper_2505_06523_gb300 import Context
    with Context(0) as ctx:
        k = torch.from_numpy(keys.view(np.int32).copy()).cuda()
        v = torch.from_numpy(vals.view(np.int32).copy()).cuda()
        ctx.sort_pairs(k, v, begin, end)
        return k.cpu().numpy().view(np.uint32), v.cpu().numpy().view(np.uint32)


def _sorted_noalloc(native, keys, vals, begin, end):
    import torch
    k = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    v = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    native.v3dg_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), k.numel(), begin, end,
                                   torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return k.cpu().numpy().view(np.uint32), v.cpu().numpy().view(np.uint32)


def test_noalloc_matches_existing_sort_twice(native):
    """Calls in a row, large after small and small after large: the shared scratch keeps the
    last call's look-back words, which must never leak into a later call's result."""
    rng = np.random.default_rng(11)
    for call, (n, begin, end) in enumerate([(300_001, 0, 32), (1 << 20, 0, 13), (70_000, 3, 29)]):
        keys = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
        vals = np.arange(n, dtype=np.uint32)
        want = _sorted_with_existing(keys, vals, begin, end)
        got = _sorted_noalloc(native, keys, vals, begin, end)
        assert (got[0] == want[0]).all() and (got[1] == want[1]).all(), f"call {call}"


def test_noalloc_allocates_nothing(native):
    """Free device memory is the same before and after calls made once the code is loaded."""
    import torch
    rng = np.random.default_rng(12)
    n = 200_003
    k = torch.from_numpy(rng.integers(0, 2 ** 31, n, dtype=np.int64).astype(np.int32)).cuda()
    v = torch.arange(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    native.v3dg_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), n, 0, 32, stream)   # code and scratch loaded
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        native.v3dg_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), n, 0, 32, stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    got = k.cpu().numpy()
    assert (np.diff(got.astype(np.int64)) >= 0).all()


def test_noalloc_rejects_beyond_its_scratch(native):
    import torch
    n = (1 << 20) + 1
    k = torch.zeros(n, dtype=torch.int32, device="cuda")
    v = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(native.V3dgError) as e:
        native.v3dg_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), n, 0, 32, torch.cuda.current_stream().cuda_stream)
    assert e.value.status == native.V3DG_EOVERFLOW


def test_noalloc_rejects_bad_bit_ranges(native):
    import torch
    k = torch.zeros(1000, dtype=torch.int32, device="cuda")
    v = torch.zeros(1000, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for begin, end in [(0, 33), (-1, 8), (12, 12), (20, 4)]:
        with pytest.raises(native.V3dgError) as e:
            native.v3dg_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), 1000, begin, end, stream)
        assert e.value.status == native.V3DG_EINVAL
