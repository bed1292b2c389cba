"""The allocation-free sampling entry point (mach_sample_noalloc) against the
allocating one (mach_sample): same kept indices and values on two calls in a
row, its size limit, and the capacity error.  Collected last on purpose: it
must also pass after every other GPU test has run in the same process."""
import pytest

from paper_0909_4969_gb300 import synth
from tests._gpu import mach_module, torch

pytestmark = pytest.mark.gpu


def _reference(mach, x, p, seed):
    s = mach.sample(x, p, seed)
    try:
        return s.indices().cpu(), s.values().cpu()
    finally:
        s.free()


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("dims,p,seed", [
    ((61, 47, 83), 0.05, 11),
    ((200, 150, 100), 0.01, 2024),
    ((17, 9, 13, 11), 0.3, 7),
])
def test_noalloc_matches_sample_twice(dims, p, seed, dtype):
    mach = mach_module()
    X = synth.tucker_numpy(synth.TuckerSpec(dims, (3,) * len(dims), noise=0.1, seed=seed, dtype=dtype))[0]
    x = torch.from_numpy(X).cuda()
    idx_ref, val_ref = _reference(mach, x, p, seed)
    K = idx_ref.numel()
    cap = K + 64
    idx = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    val = torch.zeros(cap, dtype=x.dtype, device="cuda")
    for call in range(2):
        idx.fill_(-1)
        val.zero_()
        free_before = torch.cuda.mem_get_info()[0]
        n = mach.sample_noalloc(x, p, seed, idx, val)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        assert n == K, "call %d: %d kept, expected %d" % (call, n, K)
        assert torch.equal(idx[:K].cpu(), idx_ref), "call %d: indices differ" % call
        assert torch.equal(val[:K].cpu(), val_ref), "call %d: values differ" % call
        assert bool((idx[K:] == -1).all()), "call %d: wrote past the kept count" % call
        if call == 1:
            assert free_after == free_before, "device memory changed across the call"


def test_noalloc_capacity_and_limits():
    mach = mach_module()
    dims, p, seed = (64, 64, 64), 0.1, 5
    X = synth.tucker_numpy(synth.TuckerSpec(dims, (2, 2, 2), noise=0.1, seed=seed, dtype="float32"))[0]
    x = torch.from_numpy(X).cuda()
    idx_ref, val_ref = _reference(mach, x, p, seed)
    K = idx_ref.numel()
    half = K // 2
    idx = torch.zeros(half, dtype=torch.int64, device="cuda")
    val = torch.zeros(half, dtype=torch.float32, device="cuda")
    with pytest.raises(mach.MachError) as ei:
        mach.sample_noalloc(x, p, seed, idx, val)
    assert ei.value.n_kept == K
    # the entries that fit are the first ones, in order
    assert torch.equal(idx.cpu(), idx_ref[:half])
    assert torch.equal(val.cpu(), val_ref[:half])
    # a tensor above the fixed-scratch limit is refused before any device work
    # (only the shape is passed; the pointer is a small valid buffer)
    big = (16384, 16384, 9)
    lib = mach.load()
    import ctypes
    n = ctypes.c_int64(-1)
    st = lib.mach_sample_noalloc(ctypes.c_void_p(x.data_ptr()), mach.MACH_F32, 3, mach._i64(big), 0.5,
                                 ctypes.c_uint64(1), ctypes.c_void_p(idx.data_ptr()),
                                 ctypes.c_void_p(val.data_ptr()), half, ctypes.byref(n), mach._stream())
    assert st == 1 and n.value == -1
    assert b"fixed scratch" in lib.mach_last_error()
    # the entry point still works after the refusals
    idx2 = torch.zeros(K, dtype=torch.int64, device="cuda")
    val2 = torch.zeros(K, dtype=torch.float32, device="cuda")
    assert mach.sample_noalloc(x, p, seed, idx2, val2) == K
    assert torch.equal(idx2.cpu(), idx_ref)
