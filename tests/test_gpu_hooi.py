"""GPU parity of MACH-HOOI / MACH-HOSVD (mach_hooi, mach_core, mach_error)
against the FP64 oracle: subspaces, core (after the sign convention) and
reconstruction error within 1e-10 for the FP64 path and 1e-5 for the FP32
path, on seeded synthetic tensors that span several tasks and tiles."""
import math

import numpy as np
import pytest

from oracle import mach_oracle as O
from paper_0909_4969_gb300 import synth
from tests._gpu import compare_decomposition, mach_module, torch

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


def run_both(X, ranks, p, seed, sweeps, prec):
    mach = mach_module()
    S, G_o, A_o = O.mach_hooi(X, ranks, p, seed, sweeps)
    xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    s = mach.sample(xd, p, seed)
    assert np.array_equal(s.indices().cpu().numpy(), S.idx)
    G, A = s.hooi(ranks, sweeps, prec)
    torch.cuda.synchronize()
    G_g = G.cpu().numpy()
    A_g = [a.cpu().numpy() for a in A]
    st = s.stats()
    assert st["flags"] == 0, st
    s.free()
    return S, G_o, A_o, G_g, A_g, xd


def test_plain_fp64_workload_full_size():
    """100 x 50 x 200 FP64, ranks 5, p = 0.1, 10 sweeps, seed 0 (full size)."""
    w = synth.config_plain_fp64()
    X, _, _ = synth.tucker_numpy(w.spec)
    S, G_o, A_o, G_g, A_g, xd = run_both(X, w.spec.ranks, w.p, w.spec.seed, w.sweeps, "fp64")
    compare_decomposition(O, X, G_o, A_o, G_g, A_g, TOL["fp64"], "fp64 100x50x200")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_large_workload_scaled(prec):
    """The 1000^3 / p = 0.01 / ranks 10 / 20 sweeps workload scaled to 120^3
    with p = 0.05 (same ranks, sweeps and noise)."""
    spec = synth.TuckerSpec((120, 120, 120), (10, 10, 10), "gaussian", 0.05, 0, "float32")
    X, _, _ = synth.tucker_numpy(spec)
    S, G_o, A_o, G_g, A_g, xd = run_both(X, spec.ranks, 0.05, 0, 20, prec)
    compare_decomposition(O, X.astype(np.float64), G_o, A_o, G_g, A_g, TOL[prec], prec + " 120^3")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_uneven_ranks_many_rows(prec):
    """Uneven ranks (6, 5, 7) on a 260 x 180 x 220 tensor: rows of ~2e3
    entries split over several TTM tasks (fix-up reduction) in every mode."""
    spec = synth.TuckerSpec((260, 180, 220), (6, 5, 7), "gaussian", 0.05, 3, "float32")
    X, _, _ = synth.tucker_numpy(spec)
    S, G_o, A_o, G_g, A_g, xd = run_both(X, spec.ranks, 0.05, 11, 6, prec)
    compare_decomposition(O, X.astype(np.float64), G_o, A_o, G_g, A_g, TOL[prec], prec + " uneven ranks, many rows")


def test_long_rows_fp32():
    """Rows of 6e3 - 1.2e4 entries (tasks split rows mid-fibre), FP32."""
    spec = synth.TuckerSpec((160, 200, 300), (4, 4, 4), "gaussian", 0.05, 5, "float32")
    X, _, _ = synth.tucker_numpy(spec)
    S, G_o, A_o, G_g, A_g, xd = run_both(X, spec.ranks, 0.2, 13, 3, "fp32")
    compare_decomposition(O, X.astype(np.float64), G_o, A_o, G_g, A_g, TOL["fp32"], "fp32 long rows")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_four_way_scaled(prec):
    spec = synth.TuckerSpec((30, 28, 26, 24), (4, 4, 4, 4), "lognormal_sign", 0.05, 1, "float32")
    X, _, _ = synth.tucker_numpy(spec)
    S, G_o, A_o, G_g, A_g, xd = run_both(X, spec.ranks, 0.2, 4, 8, prec)
    compare_decomposition(O, X.astype(np.float64), G_o, A_o, G_g, A_g, TOL[prec], prec + " 4-way")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_uneven_ranks_and_matrix(prec):
    spec = synth.TuckerSpec((70, 19, 300), (4, 4, 8), "gaussian", 0.10, 2, "float32")
    X, _, _ = synth.tucker_numpy(spec)
    S, G_o, A_o, G_g, A_g, xd = run_both(X, spec.ranks, 0.1, 9, 10, prec)
    compare_decomposition(O, X.astype(np.float64), G_o, A_o, G_g, A_g, TOL[prec], prec + " uneven")
    # d = 2: Tucker of a matrix is its truncated SVD
    M = synth.tucker_numpy(synth.TuckerSpec((90, 70), (3, 3), "gaussian", 0.05, 5, "float64"))[0]
    S, G_o, A_o, G_g, A_g, xd = run_both(M, (3, 3), 0.3, 1, 4, prec)
    compare_decomposition(O, M, G_o, A_o, G_g, A_g, TOL[prec], prec + " matrix")


@pytest.mark.parametrize("dims,ranks,core,p,sweeps", [
    ((30, 28, 26, 24), (4, 4, 4, 4), "lognormal_sign", 0.2, 8),
    ((120, 120, 120), (10, 10, 10), "gaussian", 0.05, 10),
])
def test_bf16_refine_matches_oracle(dims, ranks, core, p, sweeps):
    """BF16_REFINE: `sweeps` sweeps read BF16 copies of the sampled values,
    three more sweeps with the FP32 values refine every factor; against the
    FP64 oracle run for the same total number of sweeps, within 1e-5."""
    spec = synth.TuckerSpec(dims, ranks, core, 0.05, 2, "float32")
    X, _, _ = synth.tucker_numpy(spec)
    mach = mach_module()
    S, G_o, A_o = O.mach_hooi(X.astype(np.float64), ranks, p, 21, sweeps + 3)
    xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    s = mach.sample(xd, p, 21)
    G, A = s.hooi(ranks, sweeps, "bf16_refine")
    torch.cuda.synchronize()
    st = s.stats()
    assert st["flags"] == 0, st
    s.free()
    compare_decomposition(O, X.astype(np.float64), G_o, A_o, G.cpu().numpy(), [a.cpu().numpy() for a in A],
                          TOL["fp32"], "bf16_refine %s" % (dims,))


def test_exact_recovery_p_one():
    """Noise-free exact multilinear rank, p = 1: HOSVD is exact (Section 2.1)."""
    mach = mach_module()
    X, G, Us = synth.tucker_numpy(synth.TuckerSpec((40, 30, 50), (3, 4, 5), "gaussian", 0.0, 3, "float64"))
    xd = torch.from_numpy(X).cuda()
    s = mach.sample(xd, 1.0, 0)
    Gg, A = s.hooi((3, 4, 5), 0, "fp64")
    A_g = [a.cpu().numpy() for a in A]
    assert O.relative_error(X, Gg.cpu().numpy(), A_g) < 1e-12
    for k in range(3):
        assert O.subspace_distance(A_g[k], Us[k]) < 1e-12
    rel, xn = mach.error(xd, Gg, A)
    assert rel < 1e-6 and abs(xn - O.norm(X)) < 1e-10 * xn
    s.free()


def test_hosvd_only_matches_oracle():
    """sweeps = 0 is MACH-HOSVD (Algorithm 1); compared where the spectrum has a gap."""
    mach = mach_module()
    X = synth.tucker_numpy(synth.TuckerSpec((60, 40, 80), (3, 3, 3), "gaussian", 0.05, 6, "float64"))[0]
    S, G_o, A_o = O.mach_hosvd(X, (3, 3, 3), 0.5, 2)
    for k in range(3):
        w = np.sort(np.linalg.eigvalsh(S.gram(k)))[::-1]
        assert (w[2] - w[3]) / w[0] > 1e-3
    xd = torch.from_numpy(X).cuda()
    s = mach.sample(xd, 0.5, 2)
    G, A = s.hooi((3, 3, 3), 0, "fp64")
    compare_decomposition(O, X, G_o, A_o, G.cpu().numpy(), [a.cpu().numpy() for a in A], 1e-10, "hosvd")
    s.free()


def test_warm_start_continues_oracle_trajectory():
    mach = mach_module()
    X = synth.tucker_numpy(synth.TuckerSpec((50, 40, 60), (4, 4, 4), "gaussian", 0.1, 8, "float64"))[0]
    idx, vals = O.sample(X, 0.2, 3)
    S = O.SampledTensor(X.shape, idx, vals, 0.2)
    _, A3 = O.hooi(S, (4, 4, 4), 3)
    G_o, A_o = O.hooi(S, (4, 4, 4), 4, init=A3)
    xd = torch.from_numpy(X).cuda()
    s = mach.sample(xd, 0.2, 3)
    init = [torch.from_numpy(a).cuda() for a in A3]
    G, A = s.hooi((4, 4, 4), 4, "fp64", factors=init, warm=True)
    compare_decomposition(O, X, G_o, A_o, G.cpu().numpy(), [a.cpu().numpy() for a in A], 1e-10, "warm")
    s.free()


def test_core_and_error_entry_points():
    """mach_core with given (oracle) factors equals the oracle's core; mach_error
    equals the oracle's relative error."""
    mach = mach_module()
    X = synth.tucker_numpy(synth.TuckerSpec((45, 35, 55), (3, 4, 5), "gaussian", 0.1, 4, "float64"))[0]
    S, G_o, A_o = O.mach_hooi(X, (3, 4, 5), 0.3, 6, 2)
    xd = torch.from_numpy(X).cuda()
    s = mach.sample(xd, 0.3, 6)
    G = s.core((3, 4, 5), [torch.from_numpy(a).cuda() for a in A_o]).cpu().numpy()
    assert np.linalg.norm(G - G_o) <= 1e-12 * np.linalg.norm(G_o)
    rel, _ = mach.error(xd, torch.from_numpy(G_o).cuda(), [torch.from_numpy(a).cuda() for a in A_o])
    assert abs(rel - O.relative_error(X, G_o, A_o)) < 1e-10
    x32 = xd.float()
    rel32, _ = mach.error(x32, torch.from_numpy(G_o).cuda(), [torch.from_numpy(a).cuda() for a in A_o])
    assert abs(rel32 - O.relative_error(X.astype(np.float32).astype(np.float64), G_o, A_o)) < 1e-5
    s.free()


def test_rank_validation():
    mach = mach_module()
    xd = torch.randn((20, 10, 30), dtype=torch.float32, device="cuda")
    s = mach.sample(xd, 0.5, 1)
    for ranks in [(0, 2, 2), (21, 2, 2), (17, 2, 2), (2, 2, 5)]:   # r_3 = 5 > r_1 r_2 = 4
        with pytest.raises(mach.MachError):
            s.hooi(ranks, 1, "fp32")
    s.free()


def test_graph_replayed_sweeps_match_direct():
    """On a non-default stream the sweeps after the first run as replays of
    one captured CUDA graph.  From the same starting factors (warm start, so
    no atomically accumulated HOSVD Gram is involved) and the same fresh
    sample state, the replayed sweeps give the same result as direct launches
    on the default stream: the same kernels in the same order, every
    reduction in a fixed order."""
    mach = mach_module()
    spec = synth.TuckerSpec((90, 70, 110), (5, 4, 6), "gaussian", 0.05, 2, "float32")
    X, _, _ = synth.tucker_numpy(spec)
    xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    for prec in ("fp32", "fp64"):
        s0 = mach.sample(xd, 0.2, 5)
        _, A_start = s0.hooi(spec.ranks, 1, prec)
        torch.cuda.synchronize()
        s0.free()
        s1 = mach.sample(xd, 0.2, 5)
        G0, A0 = s1.hooi(spec.ranks, 8, prec, factors=[a.clone() for a in A_start], warm=True)
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            s2 = mach.sample(xd, 0.2, 5, stream=side)
            G1, A1 = s2.hooi(spec.ranks, 8, prec, factors=[a.clone() for a in A_start], warm=True, stream=side)
        side.synchronize()
        assert s1.stats()["flags"] == 0 and s2.stats()["flags"] == 0
        assert torch.equal(G0, G1), (prec, (G0 - G1).abs().max().item())
        for a0, a1 in zip(A0, A1):
            assert torch.equal(a0, a1), (prec, (a0 - a1).abs().max().item())
        s1.free()
        s2.free()
