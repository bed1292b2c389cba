"""GPU parity of the MACH coin (mach_sample) against the oracle: the kept
index set must match bit for bit, the kept values exactly."""
import math

import numpy as np
import pytest

from oracle import mach_oracle as O
from paper_0909_4969_gb300 import synth
from tests._gpu import mach_module, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("skip", [False, True])
@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("dims,p,seed", [
    ((100, 50, 200), 0.1, 0),          # small FP64 workload shape, many tiles
    ((37, 29, 53), 0.3, 7),            # ragged: N not a multiple of the tile or of 4
    ((5, 3), 0.5, 1),                  # tiny, smaller than one tile
    ((64, 64, 64), 1.0, 3),            # p = 1 keeps everything
    ((41, 17, 23, 11), 0.05, 2 ** 40 + 17),   # 4-way, seed with a high word
    ((300, 250, 190), 0.01, 123),      # sparse, ~14k kept over 14.25M entries
])
def test_sample_bit_exact(dims, p, seed, dtype, skip):
    """mach_sample and its sector-skipping form mach_sample_skip."""
    mach = mach_module()
    rng = np.random.default_rng(0)
    X = rng.standard_normal(dims).astype(dtype)
    xd = torch.from_numpy(X).cuda()
    s = mach.sample(xd, p, seed, skip=skip)
    idx = s.indices().cpu().numpy()
    vals = s.values().cpu().numpy()
    ref = O.kept_indices(0, X.size, p, seed)
    assert s.count() == ref.size
    assert np.array_equal(idx, ref)
    assert np.array_equal(vals, X.reshape(-1)[ref])
    s.free()


def test_sample_empty_and_degenerate():
    mach = mach_module()
    X = torch.ones((3, 4, 5), dtype=torch.float32, device="cuda")
    # p so small that nothing is kept among 60 entries for this seed
    p = 1e-9
    ref = O.kept_indices(0, 60, p, 5)
    s = mach.sample(X, p, 5)
    assert s.count() == ref.size == 0
    assert s.indices().numel() == 0
    with pytest.raises(mach.MachError):
        s.hooi((2, 2, 2), 1, "fp64")
    s.free()
    # single-entry modes
    Y = torch.arange(7, dtype=torch.float64, device="cuda").reshape(1, 7)
    s = mach.sample(Y, 1.0, 0)
    assert np.array_equal(s.indices().cpu().numpy(), np.arange(7))
    s.free()


def test_sample_rejects_bad_arguments():
    mach = mach_module()
    X = torch.zeros((4, 4, 4), dtype=torch.float32, device="cuda")
    for p in (0.0, -0.1, 1.5):
        with pytest.raises(mach.MachError):
            mach.sample(X, p, 0)
    big = torch.zeros((2, 20000), dtype=torch.float32, device="cuda")
    with pytest.raises(mach.MachError):
        mach.sample(big, 0.5, 0)
    with pytest.raises(mach.MachError):
        mach.sample(torch.zeros((4, 4, 4, 4, 2), device="cuda"), 0.5, 0)


def test_sample_full_size_windows():
    """The 1000^3 FP32 workload at full size (4 GB): sampled windows of l are
    bit-exact against the oracle, the count is within 5 sigma of the binomial
    mean, and the list is strictly increasing."""
    mach = mach_module()
    w = synth.config_large_fp32()
    X, _, _ = synth.tucker_torch(w.spec, device="cuda")
    s = mach.sample(X, w.p, w.spec.seed)
    N = X.numel()
    idx = s.indices()
    K = idx.numel()
    q = O.keep_threshold(w.p) / 2 ** 32
    assert abs(K - N * q) < 5 * math.sqrt(N * q * (1 - q))
    assert bool(torch.all(idx[1:] > idx[:-1]))
    rng = np.random.default_rng(99)
    starts = [0, N - 200_000] + [int(v) for v in rng.integers(0, N - 200_000, size=12)]
    idx_h = idx.cpu().numpy()
    vals_h = s.values().cpu().numpy()
    for a in starts:
        b = a + 200_000
        ref = O.kept_indices(a, b, w.p, w.spec.seed)
        lo, hi = np.searchsorted(idx_h, [a, b])
        assert np.array_equal(idx_h[lo:hi], ref)
        got = vals_h[lo:hi]
        want = X.reshape(-1)[torch.from_numpy(ref).cuda()].cpu().numpy() if ref.size else got
        assert np.array_equal(got, want)
    # the sector-skipping form keeps exactly the same (index, value) list
    s2 = mach.sample(X, w.p, w.spec.seed, skip=True)
    assert torch.equal(s2.indices(), idx)
    assert torch.equal(s2.values(), s.values())
    s2.free()
    s.free()
    del X
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("dims,p,seed,chunk", [
    ((100, 50, 200), 0.1, 0, 2048 * 16),      # 31 chunks, the last one partial
    ((37, 29, 53), 0.3, 7, 2048),             # ragged N, one chunk per 2048 entries
    ((64, 64, 64), 1.0, 3, 2048 * 40),        # p = 1
    ((41, 17, 23, 11), 0.05, 2 ** 40 + 17, 2048 * 8),
    ((30, 20, 10), 0.2, 5, 0),                # default chunk (one chunk covers the tensor)
])
def test_sample_host_streamed(dims, p, seed, chunk, dtype):
    """mach_sample_host: the tensor stays in (page-locked) host memory and is
    streamed in chunks; the kept set, values and every ordering equal the
    oracle's coin and mach_sample's result on the device copy."""
    mach = mach_module()
    rng = np.random.default_rng(1)
    X = rng.standard_normal(dims).astype(dtype)
    xh = torch.from_numpy(X).pin_memory()
    s = mach.sample(xh, p, seed, chunk_entries=chunk)
    idx = s.indices().cpu().numpy()
    vals = s.values().cpu().numpy()
    ref = O.kept_indices(0, X.size, p, seed)
    assert np.array_equal(idx, ref)
    assert np.array_equal(vals, X.reshape(-1)[ref])
    sd = mach.sample(torch.from_numpy(X).cuda(), p, seed)
    for m in range(len(dims)):
        assert s.fibers(m) == sd.fibers(m)
    if len(dims) == 3 and p < 1.0:
        G1, A1 = s.hooi((3, 3, 3), 2, "fp64")
        G2, A2 = sd.hooi((3, 3, 3), 2, "fp64")
        torch.cuda.synchronize()
        assert torch.allclose(G1, G2, rtol=0, atol=1e-12 * G2.abs().max().item())
    s.free()
    sd.free()


def test_sample_host_rejects_bad_chunk():
    mach = mach_module()
    xh = torch.randn(10, 10, 10)
    with pytest.raises(mach.MachError):
        mach.sample(xh, 0.5, 1, chunk_entries=1000)   # not a multiple of 2048
