"""Pins for the oracle's MACH-HOSVD / MACH-HOOI (Algorithm 1 / Algorithm 2)
against what the paper and the mathematics fix: the closed-form exactness of
HOSVD on noise-free data of exact multilinear rank (Section 2.1 "Tucker3
Algorithms"), the p = 1 special case (X^ = X) reducing to plain HOOI computed
by an independent brute-force route, orthonormal factors, the projection
bound ||G|| <= ||X^|| and HOOI's monotone fit, stationarity at convergence,
and the 1/p reweighing of Algorithm 2."""
import json
import math
import os

import numpy as np
import pytest

from oracle import mach_oracle as O
from paper_0909_4969_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_hooi(X, ranks, sweeps):
    """Plain HOOI written independently: Kronecker-form TTM chain
    Y_(n) = X_(n) (kron of the other factors) and dense SVDs."""
    d = X.ndim
    A = [O.leading_left_singular_vectors(O.unfold(X, k), ranks[k]) for k in range(d)]
    for _ in range(sweeps):
        for n in range(d):
            K = None
            for k in range(d):
                if k == n:
                    continue
                K = A[k] if K is None else np.kron(A[k], K)
            A[n] = O.leading_left_singular_vectors(O.unfold(X, n) @ K, ranks[n])
    G = X
    for k in range(d):
        G = O.mode_product(G, A[k].T, k)
    return G, A


def exact_rank_tensor(dims, ranks, seed):
    X, G, Us = synth.tucker_numpy(synth.TuckerSpec(dims, ranks, "gaussian", 0.0, seed, "float64"))
    return X, Us


@pytest.mark.parametrize("dims,ranks", [((8, 7, 9), (3, 2, 4)), ((6, 5, 7, 4), (2, 3, 2, 2))])
def test_hosvd_exact_on_exact_multilinear_rank(dims, ranks):
    X, Us = exact_rank_tensor(dims, ranks, 1)
    S, G, A = O.mach_hosvd(X, ranks, 1.0, 0)
    assert S.idx.size == X.size
    assert O.relative_error(X, G, A) < 1e-13
    for k in range(len(dims)):
        assert O.subspace_distance(A[k], Us[k]) < 1e-12


@pytest.mark.parametrize("dims,ranks", [((4, 3, 5), (2, 2, 3)), ((6, 5, 7, 3), (2, 3, 2, 2)), ((9, 8, 10), (3, 3, 3))])
def test_p_one_reduces_to_plain_hooi(dims, ranks):
    rng = np.random.default_rng(11)
    X = rng.standard_normal(dims)
    S, G, A = O.mach_hooi(X, ranks, 1.0, 5, sweeps=4)
    Gb, Ab = brute_hooi(X, list(ranks), 4)
    for k in range(len(dims)):
        assert O.subspace_distance(A[k], Ab[k]) < 1e-10
    Af = [O.fix_signs(a) for a in A]
    Abf = [O.fix_signs(a) for a in Ab]
    Gf = S.dense(scaled=True)
    Gbf = X
    for k in range(len(dims)):
        Gf = O.mode_product(Gf, Af[k].T, k)
        Gbf = O.mode_product(Gbf, Abf[k].T, k)
    np.testing.assert_allclose(Gf, Gbf, rtol=1e-9, atol=1e-10 * O.norm(X))


def _c1_small():
    spec = synth.TuckerSpec((30, 20, 40), (3, 3, 3), "gaussian", 0.1, 3, "float64")
    X, _, Us = synth.tucker_numpy(spec)
    return X, Us


def test_invariants_orthonormal_projection_monotone():
    X, _ = _c1_small()
    idx, vals = O.sample(X, 0.3, 4)
    S = O.SampledTensor(X.shape, idx, vals, 0.3)
    hist = []
    G, A = O.hooi(S, (3, 3, 3), 6, history=hist)
    for a in A:
        assert np.max(np.abs(a.T @ a - np.eye(a.shape[1]))) < 1e-13
    assert O.norm(G) <= O.norm(S.dense(scaled=True)) * (1 + 1e-14)
    for a, b in zip(hist, hist[1:]):
        assert b >= a * (1 - 1e-12)


def test_stationarity_at_convergence():
    X, _ = _c1_small()
    idx, vals = O.sample(X, 0.3, 4)
    S = O.SampledTensor(X.shape, idx, vals, 0.3)
    G, A = O.hooi(S, (3, 3, 3), 40)
    for n in range(3):
        Y = O.unfold(O.ttm_chain(S, A, skip=n), n)
        U = O.leading_left_singular_vectors(Y, 3)
        assert O.subspace_distance(U, A[n]) < 1e-10


def test_reweigh_once_matches_literal_algorithm():
    """Algorithm 2 reweighs kept entries by 1/p before HOOI; the oracle works on
    raw values and divides the core by p.  Both give the same factors and core."""
    X, _ = _c1_small()
    p = 0.3
    idx, vals = O.sample(X, p, 8)
    raw = O.SampledTensor(X.shape, idx, vals, p)
    literal = O.SampledTensor(X.shape, idx, vals / p, 1.0)
    G1, A1 = O.hooi(raw, (3, 3, 3), 3)
    G2, A2 = O.hooi(literal, (3, 3, 3), 3)
    for a, b in zip(A1, A2):
        assert O.subspace_distance(a, b) < 1e-12
    A1f = [O.fix_signs(a) for a in A1]
    A2f = [O.fix_signs(a) for a in A2]
    np.testing.assert_allclose(O.core(raw, A1f), O.core(literal, A2f), rtol=1e-10, atol=1e-12)


def test_hosvd_dense_and_sparse_routes_agree():
    X, _ = _c1_small()
    idx, vals = O.sample(X, 0.5, 2)
    S = O.SampledTensor(X.shape, idx, vals, 0.5)
    for k in range(3):
        a = O.leading_left_singular_vectors(O.unfold(S.dense(), k), 3)
        b = O.leading_eigenvectors(S.gram(k), 3)
        assert O.subspace_distance(a, b) < 1e-10


def test_error_decreases_towards_p_one():
    X, Us = synth.tucker_numpy(synth.TuckerSpec((40, 30, 50), (3, 3, 3), "gaussian", 0.0, 9, "float64"))[0], None
    errs = []
    for p in (0.1, 0.3, 1.0):
        S, G, A = O.mach_hooi(X, (3, 3, 3), p, 1, 2)
        errs.append(O.relative_error(X, G, A))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-12


def test_relative_error_slabs():
    X, _ = _c1_small()
    S, G, A = O.mach_hooi(X, (3, 3, 3), 0.5, 1, 1)
    assert abs(O.relative_error(X, G, A) - O.relative_error(X, G, A, slab=7)) < 1e-13


def test_synthetic_inverse_sum_loose():
    """Section 4's synthetic example at the paper's size n = 200: MACH-HOOI at
    p = 0.1 keeps the top principal component of every mode (the paper prints
    Pearson correlations 0.9955-0.9967); checked loosely (>= 0.98)."""
    gold = json.load(open(os.path.join(GOLDEN, "synthetic_inverse_sum.json")))
    assert min(gold["pearson_top_pc"]) > 0.99
    X = synth.inverse_sum_tensor(gold["n"])
    Se = O.SampledTensor(X.shape, np.arange(X.size), X.reshape(-1), 1.0)
    Ge, Ae = O.hooi(Se, gold["ranks"], 3)
    S, G, A = O.mach_hooi(X, gold["ranks"], gold["p"], 2009, 3)
    for k in range(3):
        assert abs(O.pearson(Ae[k][:, 0], A[k][:, 0])) >= 0.98


def test_tucker2_equals_tucker3_with_full_rank_in_the_kept_mode():
    """Tucker2 (mode c whole, Section 2.1 Tucker-n) is Tucker3 with r_c = I_c:
    a full orthonormal A_c only rotates the kept mode, so the compressed
    factors, the projection and the reconstruction error coincide.  The
    Tucker3 route computes its A_c by SVD and shares no Tucker2 branch."""
    X, _, _ = synth.tucker_numpy(synth.TuckerSpec((12, 9, 5), (3, 2, 3), "gaussian", 0.2, 4, "float64"))
    idx, vals = O.sample(X, 0.5, 21)
    S = O.SampledTensor(X.shape, idx, vals, 0.5)
    G2, A2 = O.hooi(S, (3, 2, 0), 6, keep=(2,))
    G3, A3 = O.hooi(S, (3, 2, 5), 6)
    assert np.allclose(A2[2], np.eye(5)) and G2.shape == (3, 2, 5)
    for k in (0, 1):
        assert O.subspace_distance(A2[k], A3[k]) < 1e-10
    assert abs(O.relative_error(X, G2, A2) - O.relative_error(X, G3, A3)) < 1e-12
    assert abs(O.norm(G2) - O.norm(G3)) < 1e-12 * O.norm(G3)


def test_tucker2_p_one_matches_brute_force_and_recovers_exact_rank():
    """At p = 1 the oracle's Tucker2 equals an independent Kronecker-form
    Tucker2 (identity for the kept mode), and a tensor of exact rank in the
    compressed modes is recovered to rounding."""
    rng = np.random.default_rng(5)
    U0 = np.linalg.qr(rng.standard_normal((10, 3)))[0]
    U2 = np.linalg.qr(rng.standard_normal((11, 2)))[0]
    C = rng.standard_normal((3, 6, 2))
    X = O.mode_product(O.mode_product(C, U0, 0), U2, 2)          # mode 1 (size 6) stays whole
    idx, vals = O.sample(X, 1.0, 1)
    S = O.SampledTensor(X.shape, idx, vals, 1.0)
    G, A = O.hooi(S, (3, 0, 2), 3, keep=(1,))
    assert O.relative_error(X, G, A) < 1e-13
    # brute force: Kronecker-form chain with A_1 = I, dense SVDs
    B = [O.leading_left_singular_vectors(O.unfold(X, 0), 3), np.eye(6),
         O.leading_left_singular_vectors(O.unfold(X, 2), 2)]
    for _ in range(3):
        for n in (0, 2):
            others = [k for k in range(3) if k != n]
            K = np.kron(B[others[1]], B[others[0]])
            B[n] = O.leading_left_singular_vectors(O.unfold(X, n) @ K, B[n].shape[1])
    for k in (0, 2):
        assert O.subspace_distance(A[k], B[k]) < 1e-12


@pytest.mark.parametrize("eps", [1e-3, 0.25, 2.0])
def test_relative_error_two_spike_closed_form(eps):
    """Section 4's accuracy measure is the unsquared norm ratio
    ||X - G x_1 A_1 .. x_d A_d|| / ||X||.  For X = e_111 + eps e_222 and the
    rank-(1,1,1) model G = [[[1]]], A_k = e_1 the residual is eps e_222, so
    the measure is eps / sqrt(1 + eps^2) (a squared form would give
    eps^2 / (1 + eps^2), a residual against X^ or a dropped core term
    something else).  HOOI at p = 1 finds that model exactly when eps < 1
    (the larger spike leads every unfolding); with eps > 1 it picks e_2."""
    X = np.zeros((2, 2, 2))
    X[0, 0, 0] = 1.0
    X[1, 1, 1] = eps
    e1 = np.array([[1.0], [0.0]])
    want = eps / math.sqrt(1.0 + eps * eps)
    assert abs(O.relative_error(X, np.ones((1, 1, 1)), [e1, e1, e1]) - want) < 1e-15
    assert abs(O.relative_error(X, np.ones((1, 1, 1)), [e1, e1, e1], slab=1) - want) < 1e-15
    S, G, A = O.mach_hooi(X, (1, 1, 1), 1.0, 3, 2)
    lead = max(1.0, eps)
    other = min(1.0, eps)
    assert abs(abs(G.item()) - lead) < 1e-14
    assert abs(O.relative_error(X, G, A) - other / math.sqrt(1.0 + eps * eps)) < 1e-14


def test_relative_error_orthogonal_residual_closed_form():
    """With orthonormal factors U_k and a residual E orthogonal to
    span(U_1) (E's mode-1 fibres are projected off U_1), X = G x U + E has
    ||X - G x U|| = ||E|| and ||X||^2 = ||G||^2 + ||E||^2 (orthonormal
    products preserve the norm, Section 2.1), so the measure is
    ||E|| / sqrt(||G||^2 + ||E||^2) exactly; a scale, a square or a
    transposed factor would break it."""
    rng = np.random.default_rng(5)
    dims, ranks = (9, 7, 8), (3, 2, 4)
    G = rng.standard_normal(ranks)
    Us = [np.linalg.qr(rng.standard_normal((n, r)))[0] for n, r in zip(dims, ranks)]
    E = rng.standard_normal(dims)
    E -= np.einsum("ia,ja,jkl->ikl", Us[0], Us[0], E)      # mode-1 fibres orthogonal to U_1
    X = np.einsum("abc,ia,jb,kc->ijk", G, *Us) + E
    nE, nG = np.linalg.norm(E), np.linalg.norm(G)
    want = nE / math.sqrt(nG ** 2 + nE ** 2)
    assert abs(O.relative_error(X, G, Us) - want) < 1e-14
    assert abs(O.relative_error(X, G, Us, slab=4) - want) < 1e-14
