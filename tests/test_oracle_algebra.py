"""Pins for the oracle's tensor algebra against the paper's definitions
(Section 2.1, "Tensor Concepts") written as brute-force loops on tiny
tensors, and against the algebraic identities the paper states."""
import itertools

import numpy as np
import pytest

from oracle import mach_oracle as O


def test_unfold_matches_column_major_formula():
    """(i_1..i_d) -> (i_k, j), j = 1 + sum_{q != k} (i_q - 1) J_q,
    J_q = prod_{m < q, m != k} I_m (1-based)."""
    rng = np.random.default_rng(0)
    dims = (3, 4, 2, 5)
    X = rng.standard_normal(dims)
    for k in range(len(dims)):
        M = O.unfold(X, k)
        assert M.shape == (dims[k], X.size // dims[k])
        for idx in itertools.product(*[range(1, n + 1) for n in dims]):
            j = 1
            for q in range(len(dims)):
                if q == k:
                    continue
                Jq = 1
                for m in range(q):
                    if m != k:
                        Jq *= dims[m]
                j += (idx[q] - 1) * Jq
            assert M[idx[k] - 1, j - 1] == X[tuple(i - 1 for i in idx)]
        assert np.array_equal(O.fold(M, k, dims), X)


def test_mode_product_matches_definition_loops():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((3, 4, 5))
    for n in range(3):
        Mt = rng.standard_normal((2, X.shape[n]))
        Y = O.mode_product(X, Mt, n)
        shp = list(X.shape)
        shp[n] = 2
        ref = np.zeros(shp)
        for out_idx in itertools.product(*[range(s) for s in shp]):
            s = 0.0
            for i in range(X.shape[n]):
                src = list(out_idx)
                src[n] = i
                s += X[tuple(src)] * Mt[out_idx[n], i]
            ref[out_idx] = s
        np.testing.assert_allclose(Y, ref, rtol=1e-14, atol=1e-14)


def test_mode_products_commute_and_compose():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((4, 5, 6))
    A = rng.standard_normal((3, 4))
    B = rng.standard_normal((2, 5))
    np.testing.assert_allclose(O.mode_product(O.mode_product(X, A, 0), B, 1),
                               O.mode_product(O.mode_product(X, B, 1), A, 0), rtol=1e-13, atol=1e-13)
    # X x_m A x_m B = X x_m (B A)
    A2 = rng.standard_normal((4, 6))
    B2 = rng.standard_normal((3, 4))
    np.testing.assert_allclose(O.mode_product(O.mode_product(X, A2, 2), B2, 2),
                               O.mode_product(X, B2 @ A2, 2), rtol=1e-13, atol=1e-13)


def test_orthonormal_product_preserves_norm():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((4, 5, 6))
    Q, _ = np.linalg.qr(rng.standard_normal((9, 5)))     # 9x5, Q^T Q = I
    assert abs(O.norm(O.mode_product(X, Q, 1)) - O.norm(X)) < 1e-12 * O.norm(X)
    Qs, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    assert abs(O.norm(O.mode_product(X, Qs, 2)) - O.norm(X)) < 1e-12 * O.norm(X)
    # a projection A A^T (A with orthonormal columns) can only shrink the norm
    A = np.linalg.qr(rng.standard_normal((5, 2)))[0]
    assert O.norm(O.mode_product(X, A @ A.T, 1)) <= O.norm(X) * (1 + 1e-14)


def test_norm_definition():
    X = np.arange(24, dtype=np.float64).reshape(2, 3, 4)
    assert O.norm(X) == pytest.approx(np.sqrt(sum(v * v for v in range(24))), rel=1e-15)


def test_sparse_products_match_dense():
    rng = np.random.default_rng(4)
    dims = (6, 5, 7)
    X = rng.standard_normal(dims)
    idx, vals = O.sample(X, 0.4, 9)
    S = O.SampledTensor(dims, idx, vals, 0.4)
    D = S.dense()
    for k in range(3):
        M = rng.standard_normal((3, dims[k]))
        np.testing.assert_allclose(S.mode_product_first(M, k), O.mode_product(D, M, k), rtol=1e-13, atol=1e-13)
        Uk = O.unfold(D, k)
        np.testing.assert_allclose(S.gram(k), Uk @ Uk.T, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(S.dense(scaled=True), O.sampled_dense(X, 0.4, 9), rtol=0, atol=0)


def test_ttm_chain_is_kronecker_form():
    """Independent route: Y_(n) = X_(n) (A_d kron ... kron A_1, skipping n),
    the Kronecker form of the column-major matricization."""
    rng = np.random.default_rng(5)
    dims = (5, 4, 6)
    X = rng.standard_normal(dims)
    S = O.SampledTensor(dims, np.arange(X.size), X.reshape(-1), 1.0)
    A = [np.linalg.qr(rng.standard_normal((n, 2)))[0] for n in dims]
    for n in range(3):
        Y = O.ttm_chain(S, A, skip=n)
        K = None
        for k in range(3):
            if k == n:
                continue
            K = A[k] if K is None else np.kron(A[k], K)
        np.testing.assert_allclose(O.unfold(Y, n), O.unfold(X, n) @ K, rtol=1e-12, atol=1e-12)


def test_leading_lsv_paths_agree():
    """Dense SVD of the matricization and eigenvectors of its Gram give the same subspace."""
    rng = np.random.default_rng(6)
    M = rng.standard_normal((30, 200)) * np.linspace(10, 1, 30)[:, None]
    A = O.leading_left_singular_vectors(M, 4)
    B = O.leading_eigenvectors(M @ M.T, 4)
    assert O.subspace_distance(A, B) < 1e-12
    # the leading vectors capture at least as much energy as any random 4-frame
    best = np.linalg.norm(A.T @ M)
    for _ in range(20):
        Q = np.linalg.qr(rng.standard_normal((30, 4)))[0]
        assert np.linalg.norm(Q.T @ M) <= best * (1 + 1e-14)


def test_fix_signs_and_subspace_distance():
    rng = np.random.default_rng(7)
    A = np.linalg.qr(rng.standard_normal((10, 3)))[0]
    B = A * np.array([-1.0, 1.0, -1.0])
    assert O.subspace_distance(A, B) < 1e-15
    np.testing.assert_allclose(O.fix_signs(A), O.fix_signs(B))
    C = np.linalg.qr(rng.standard_normal((10, 3)))[0]
    assert O.subspace_distance(A, C) > 0.1
