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
    rng = np.random.default_rng(11)
    for call, (n, begin, end) in enumerate([(300_001, 0, 32), (1 << 20, 0, 13)]):
        keys = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
        vals = np.arange(n, dtype=np.uint32)
        want = _sorted_with_existing(keys, vals, begin, end)
        got = _sorted_noalloc(native, keys, vals, begin, end)
        assert (got[0] == want[0]).all() and (got[1] == want[1]).all(), f"call {call}"


def test_noalloc_rejects_beyond_its_scratch(native):
    import torch
    n = (1 << 20) + 1
    k = torch.zeros(n, dtype=torch.int32, device="cuda")
    v = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(native.V3dgError) as e:
        native.v3dg_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), n, 0, 32, torch.cuda.current_stream().cuda_stream)
    assert e.value.status == native.V3DG_EOVERFLOW
