"""glisse_partition_device_noalloc: the partition for callers that cannot allocate.

Callers whose device memory is all owned by a framework or pool allocator, or
that fix their memory budget at start-up, cannot let a library call cudaMalloc.
This entry point takes its scratch from a fixed array in the library's device
image instead.  The test calls it through the C ABI and checks, on two calls
in a row with different data, that its output equals the allocating entry
point's exactly (a partition moves bytes; nothing may differ).  It lives in a
file of its own that pytest collects last, and passes alone in a fresh
process as well as after the other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_03484_gb300 as G

    G._build.build()
    G.load()
    return G


def _case(torch, n, seed):
    gen = torch.Generator().manual_seed(seed)
    ld = n + 3
    src = torch.randn(6, ld, dtype=torch.float64, generator=gen).cuda()
    ids = torch.randperm(n, generator=gen).to(torch.int32).cuda()
    # flags 0 (removed) and 1, 2, 255 (kept: any non-zero value keeps a slot)
    u = torch.rand(n, generator=gen)
    alive = torch.where(u < 0.4, 0, torch.where(u < 0.8, 1, torch.where(u < 0.9, 2, 255))).to(torch.uint8).cuda()
    return ld, src, ids, alive


def _outputs(torch, n, ld):
    dst = torch.full((6, ld), float("nan"), dtype=torch.float64, device="cuda")
    did = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    return dst, did, cnt


def test_noalloc_matches_allocating_partition_twice(G):
    import torch

    stream = torch.cuda.current_stream().cuda_stream
    for call, (n, seed) in enumerate([(300_001, 11), (4_099, 12)]):
        ld, src, ids, alive = _case(torch, n, seed)
        d_ref, id_ref, n_ref = _outputs(torch, n, ld)
        G.glisse_partition_device(n, ld, alive.data_ptr(), src.data_ptr(), ids.data_ptr(), d_ref.data_ptr(),
                                  id_ref.data_ptr(), n_ref.data_ptr(), stream)
        d_new, id_new, n_new = _outputs(torch, n, ld)
        G.glisse_partition_device_noalloc(n, ld, alive.data_ptr(), src.data_ptr(), ids.data_ptr(),
                                          d_new.data_ptr(), id_new.data_ptr(), n_new.data_ptr(), stream)
        m = int(n_ref.item())
        assert int(n_new.item()) == m, call
        assert m == int((alive != 0).sum().item())
        assert torch.equal(d_new[:, :m], d_ref[:, :m]), call
        assert torch.equal(id_new[:m], id_ref[:m]), call
        # and both equal the plain stable partition
        keep = alive != 0
        assert torch.equal(id_new[:m], ids[keep])
        assert torch.equal(d_new[:, :m], src[:, :n][:, keep])


def test_noalloc_at_its_maximum_size(G):
    """n = GLISSE_PARTITION_NOALLOC_MAX (67,108,864 slots, every scratch tile in use, ld = n):
    the result is the plain stable partition.  About 8 GB of device memory."""
    import torch

    n = G.GLISSE_PARTITION_NOALLOC_MAX
    gen = torch.Generator(device="cuda").manual_seed(21)
    src = torch.randn(6, n, dtype=torch.float64, device="cuda", generator=gen)
    ids = torch.arange(n, dtype=torch.int32, device="cuda")
    u = torch.rand(n, device="cuda", generator=gen)
    alive = torch.where(u < 0.5, 0, torch.where(u < 0.9, 1, 2)).to(torch.uint8)
    dst, did, cnt = _outputs(torch, n, n)
    stream = torch.cuda.current_stream().cuda_stream
    rc = G.glisse_partition_device_noalloc(n, n, alive.data_ptr(), src.data_ptr(), ids.data_ptr(), dst.data_ptr(),
                                           did.data_ptr(), cnt.data_ptr(), stream)
    assert rc in (None, 0)
    keep = alive != 0
    m = int(keep.sum().item())
    assert int(cnt.item()) == m
    assert torch.equal(did[:m], ids[keep])
    for c in range(6):
        assert torch.equal(dst[c, :m], src[c][keep]), c
    del src, ids, alive, dst, did, cnt, keep, u
    torch.cuda.empty_cache()


def test_noalloc_rejects_sizes_beyond_its_limit(G):
    L = G.load()
    n = G.GLISSE_PARTITION_NOALLOC_MAX + 1
    rc = L.glisse_partition_device_noalloc(n, n, 1, 1, 1, 1, 1, 1, None)
    assert rc == G.GLISSE_E_INVAL


def test_noalloc_zero_slots_is_the_set_up_call(G):
    """n = 0 does the per-device set-up only and reports no kept entries."""
    import torch

    cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    G.glisse_partition_device_noalloc(0, 0, None, None, None, None, None, cnt.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
    assert int(cnt.item()) == 0
