"""MACH oracle: a plain, slow, FP64 CPU implementation of MACH-HOSVD and
MACH-HOOI (Tsourakakis, "MACH: Fast Randomized Tensor Decompositions",
Section 3, Algorithm 1 and Algorithm 2).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  It shares no code with the CUDA path (no kernels, headers, helpers,
tables or pre/post-processing); the two meet only through the seeded input
generators in ``paper_0909_4969_gb300.synth``, which hold none of the
method's arithmetic.

Every step follows the paper's definitions written out, in the paper's order:

* coin toss per entry (Algorithm 1/2, Section 3 Remark 1, Theorem 1): the
  Philox4x32-10 coin of ``philox_ref.c`` decides each linear index; kept
  entries are reweighed by 1/p;
* matricization along mode k (Section 2.1, "Tensor Concepts"): column-major
  order of the remaining indices;
* n-mode product (Section 2.1): (X x_n M)[.., j, ..] = sum_i x[.., i, ..] m[j, i];
* HOSVD (Section 2.1, "Tucker3 Algorithms", Eq. eqcore): A_k = leading r_k
  left singular vectors of the mode-k matricization, G = X x_1 A_1^T ... ;
* HOOI / ALS (Section 2.1 and Algorithm 2): HOSVD initialisation, then for
  each mode i = 1..d in turn Y = X^ x_{k != i} A_k^T with the latest factors
  and A_i = leading r_i left singular vectors of Y_(i); finally
  G = X^ x_1 A_1^T ... x_d A_d^T;
* accuracy (Section 4, "Speedups & Synthetic Experiment"):
  1 - ||X - X^ x_1 A_1 A_1^T ... x_d A_d A_d^T|| / ||X|| against the ORIGINAL X.

Library primitives used as single steps: ``numpy.linalg.svd`` (the leading
left singular vectors of an explicit matricization), ``numpy.linalg.eigh``
(those same vectors from the Gram X_(k) X_(k)^T when the matricization is too
large to form densely), ``numpy.tensordot`` (one n-mode product),
``scipy.sparse`` matrix products (one n-mode product of the sparse sampled
tensor, or its Gram).

Readings of the paper that this oracle fixes (each is also listed in the
design notes):

* one coin per linear index, including zero-valued entries (Algorithm 1/2
  toss for every entry; Remark 1 says "non-zero"; the two agree on dense
  data);
* the 1/p reweighing is applied exactly once; leading singular vectors do
  not depend on a global scale, so ``hooi`` works on the raw kept values and
  multiplies the core by 1/p (identical to reweighing each entry first; a
  test checks the two agree);
* Gauss-Seidel order i = 1..d within a sweep, a fixed number of sweeps (the
  "maximum number of iterations" of Algorithm 2), no early stop;
* HOOI initialisation = HOSVD of the sampled tensor X^ (Algorithm 2; the
  statement of Theorem 1 names X, its proof and Algorithm 1 use X^).

Parity pins: see tests/test_oracle_*.py.  Nothing here is "parity unpinned"
except the Philox multipliers, which the tests can only check for oddness and
through statistical tests (no known-answer vectors are available offline).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_philox_ref.so")
_lib = None
_lib_lock = threading.Lock()


def build_oracle_lib(force: bool = False) -> str:
    """Compile philox_ref.c (plain C, no intrinsics) into a shared object."""
    src = os.path.join(_HERE, "philox_ref.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _clib():
    global _lib
    with _lib_lock:
        if _lib is None:
            lib = ctypes.CDLL(build_oracle_lib())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.oracle_philox4x32.argtypes = [u32p, u32p, ctypes.c_int, u32p]
            lib.oracle_philox4x32.restype = None
            lib.oracle_philox_batch.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p]
            lib.oracle_philox_batch.restype = None
            lib.oracle_keep.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64]
            lib.oracle_keep.restype = ctypes.c_int
            lib.oracle_kept_indices.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                                                ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int64]
            lib.oracle_kept_indices.restype = ctypes.c_int64
            lib.oracle_philox_constants.argtypes = [u32p]
            lib.oracle_philox_constants.restype = None
            _lib = lib
    return _lib


# ----------------------------------------------------------------------------
# The coin (Algorithm 1/2, first block; Theorem 1's sampling distribution)
# ----------------------------------------------------------------------------

def keep_threshold(p: float) -> int:
    """T = floor(p * 2^32) as an integer, computed in FP64; P(keep) = T / 2^32."""
    if not (0.0 < p <= 1.0):
        raise ValueError("p must lie in (0, 1]")
    return int(math.floor(p * 4294967296.0))


def philox4x32(ctr, key, rounds: int = 10):
    """Philox4x32 of one 4-word counter under a 2-word key (10 rounds = Philox4x32-10)."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    _clib().oracle_philox4x32(c, k, int(rounds), o)
    return [int(v) for v in o]


def philox_batch(q: np.ndarray, seed: int) -> np.ndarray:
    """Philox4x32-10 words for counters (q mod 2^32, q div 2^32, 0, 0): shape (n, 4) uint32."""
    q = np.ascontiguousarray(q, dtype=np.uint64)
    out = np.empty((q.size, 4), dtype=np.uint32)
    _clib().oracle_philox_batch(q.ctypes.data, q.size, int(seed), out.ctypes.data)
    return out


def philox_constants():
    o = (ctypes.c_uint32 * 4)()
    _clib().oracle_philox_constants(o)
    return [int(v) for v in o]


def keep(l: int, p: float, seed: int) -> bool:
    """The coin for linear index l."""
    return bool(_clib().oracle_keep(int(l), int(seed), keep_threshold(p)))


def kept_indices(l0: int, l1: int, p: float, seed: int) -> np.ndarray:
    """All kept linear indices in [l0, l1), increasing."""
    T = keep_threshold(p)
    cap = max(16, int((l1 - l0) * (T / 4294967296.0) * 1.2) + 64)
    while True:
        buf = np.empty(cap, dtype=np.int64)
        n = _clib().oracle_kept_indices(int(l0), int(l1), int(seed), T, buf.ctypes.data, cap)
        if n <= cap:
            return buf[:n].copy()
        cap = int(n)


def sample(X: np.ndarray, p: float, seed: int):
    """MACH sparsification of a dense tensor X (C-order linear indices).

    Returns (idx, vals): the kept linear indices in increasing order and the
    corresponding ORIGINAL values as FP64 (not yet multiplied by 1/p).
    """
    flat = np.ascontiguousarray(X).reshape(-1)
    idx = kept_indices(0, flat.size, p, seed)
    return idx, flat[idx].astype(np.float64)


def sampled_dense(X: np.ndarray, p: float, seed: int) -> np.ndarray:
    """X^ of Algorithm 1/2 written out densely: x/p where kept, 0 elsewhere."""
    idx, vals = sample(X, p, seed)
    Xh = np.zeros(X.size, dtype=np.float64)
    Xh[idx] = vals / p
    return Xh.reshape(X.shape)


# ----------------------------------------------------------------------------
# Tensor algebra (Section 2.1)
# ----------------------------------------------------------------------------

def unfold(X: np.ndarray, k: int) -> np.ndarray:
    """Mode-k matricization: (i_1..i_d) -> (i_k, j), j running over the other
    indices in column-major order (the first remaining index fastest)."""
    Ik = X.shape[k]
    return np.reshape(np.moveaxis(X, k, 0), (Ik, -1), order="F")


def fold(M: np.ndarray, k: int, shape) -> np.ndarray:
    """Inverse of ``unfold``."""
    shape = tuple(shape)
    rest = shape[:k] + shape[k + 1:]
    T = np.reshape(M, (shape[k],) + rest, order="F")
    return np.moveaxis(T, 0, k)


def mode_product(X: np.ndarray, M: np.ndarray, n: int) -> np.ndarray:
    """n-mode product X x_n M with M of shape (J, I_n)."""
    if M.shape[1] != X.shape[n]:
        raise ValueError("n-mode product: M must have I_n columns")
    return np.moveaxis(np.tensordot(M, X, axes=(1, n)), 0, n)


def norm(X) -> float:
    """Tensor norm: square root of the sum of squared entries (Eq. norm)."""
    return float(np.sqrt(np.sum(np.asarray(X, dtype=np.float64) ** 2)))


def leading_left_singular_vectors(M: np.ndarray, r: int) -> np.ndarray:
    """The r leading left singular vectors of a dense matrix (LAPACK SVD)."""
    U, _, _ = np.linalg.svd(M, full_matrices=False)
    return np.ascontiguousarray(U[:, :r])


def leading_eigenvectors(C: np.ndarray, r: int) -> np.ndarray:
    """The r eigenvectors of a symmetric PSD matrix with the largest eigenvalues."""
    w, V = np.linalg.eigh(C)
    order = np.argsort(w)[::-1][:r]
    return np.ascontiguousarray(V[:, order])


# ----------------------------------------------------------------------------
# Sparse sampled tensor: (idx, vals) with C-order linear indices
# ----------------------------------------------------------------------------

class SampledTensor:
    """The kept entries of X^ (raw values; scale 1/p applied by the caller)."""

    def __init__(self, dims, idx, vals, p):
        self.dims = tuple(int(v) for v in dims)
        self.idx = np.asarray(idx, dtype=np.int64)
        self.vals = np.asarray(vals, dtype=np.float64)
        self.p = float(p)
        self.coords = np.unravel_index(self.idx, self.dims) if self.idx.size else tuple(
            np.zeros(0, dtype=np.int64) for _ in self.dims)

    @property
    def d(self):
        return len(self.dims)

    def dense(self, scaled: bool = False) -> np.ndarray:
        out = np.zeros(int(np.prod(self.dims)), dtype=np.float64)
        out[self.idx] = self.vals / self.p if scaled else self.vals
        return out.reshape(self.dims)

    def _matrix(self, k: int):
        """The mode-k matricization as a scipy CSR matrix (rows i_k)."""
        import scipy.sparse as sp
        rest_dims = [self.dims[q] for q in range(self.d) if q != k]
        rest_coords = [self.coords[q] for q in range(self.d) if q != k]
        if rest_dims:
            col = np.ravel_multi_index(rest_coords, rest_dims, order="F")
        else:
            col = np.zeros(self.idx.size, dtype=np.int64)
        ncol = int(np.prod(rest_dims)) if rest_dims else 1
        return sp.csr_matrix((self.vals, (self.coords[k], col)), shape=(self.dims[k], ncol))

    def mode_product_first(self, M: np.ndarray, k: int) -> np.ndarray:
        """X^ x_k M (M of shape (J, I_k)) for the sparse X^; the result is dense.

        Written as one sparse-times-dense product: rows run over the other
        indices (C-order), columns over i_k.
        """
        import scipy.sparse as sp
        rest = [q for q in range(self.d) if q != k]
        rest_dims = [self.dims[q] for q in rest]
        row = np.ravel_multi_index([self.coords[q] for q in rest], rest_dims) if rest else \
            np.zeros(self.idx.size, dtype=np.int64)
        nrow = int(np.prod(rest_dims)) if rest else 1
        S = sp.csr_matrix((self.vals, (row, self.coords[k])), shape=(nrow, self.dims[k]))
        Z = np.asarray(S @ M.T)                              # (rest..., J)
        Z = Z.reshape(rest_dims + [M.shape[0]])
        return np.moveaxis(Z, -1, k)

    def gram(self, k: int) -> np.ndarray:
        """X^_(k) X^_(k)^T as a dense I_k x I_k matrix (raw values)."""
        S = self._matrix(k)
        return np.asarray((S @ S.T).toarray(), dtype=np.float64)


def ttm_chain(S: SampledTensor, factors, skip=None) -> np.ndarray:
    """Y = X^ x_1 A_1^T ... x_d A_d^T, omitting mode ``skip``, applied in
    increasing mode order exactly as Algorithm 2 writes it (raw values)."""
    modes = [k for k in range(S.d) if k != skip]
    Y = S.mode_product_first(factors[modes[0]].T, modes[0])
    for k in modes[1:]:
        Y = mode_product(Y, factors[k].T, k)
    return Y


# ----------------------------------------------------------------------------
# MACH-HOSVD (Algorithm 1) and MACH-HOOI (Algorithm 2)
# ----------------------------------------------------------------------------

DENSE_LIMIT = 4_000_000   # matricizations up to this many entries are formed explicitly


def hosvd_factor(S: SampledTensor, k: int, r: int) -> np.ndarray:
    """A_k = r leading left singular vectors of X^_(k)."""
    N = int(np.prod(S.dims))
    if N <= DENSE_LIMIT:
        return leading_left_singular_vectors(unfold(S.dense(), k), r)
    return leading_eigenvectors(S.gram(k), r)


def core(S: SampledTensor, factors) -> np.ndarray:
    """G = X^ x_1 A_1^T ... x_d A_d^T with X^ = kept values / p."""
    return ttm_chain(S, factors, skip=None) / S.p


def hosvd(S: SampledTensor, ranks):
    """Algorithm 1 after the coin: A_i for every mode, then the core."""
    A = [hosvd_factor(S, k, int(ranks[k])) for k in range(S.d)]
    return core(S, A), A


def hooi(S: SampledTensor, ranks, sweeps: int, init=None, history=None, keep=()):
    """Algorithm 2 after the coin: HOSVD initialisation (or the given factors),
    ``sweeps`` Gauss-Seidel sweeps over i = 1..d, then the core.

    ``keep``: modes left uncompressed (Section 2.1: compressing only some of
    the modes gives a Tucker-n decomposition, e.g. the Tucker2 of Section 4);
    their factor is the identity, never updated, and their rank is I_k.

    If ``history`` is a list, the norm of the core after every sweep is
    appended to it (HOOI never decreases it)."""
    keep = set(int(k) for k in keep)
    ranks = [int(S.dims[k]) if k in keep else int(r) for k, r in enumerate(ranks)]
    if init is None:
        A = [np.eye(S.dims[k]) if k in keep else hosvd_factor(S, k, ranks[k]) for k in range(S.d)]
    else:
        A = [np.eye(S.dims[k]) if k in keep else np.array(a, dtype=np.float64, copy=True)
             for k, a in enumerate(init)]
    for _ in range(int(sweeps)):
        for i in range(S.d):
            if i in keep:
                continue
            Y = ttm_chain(S, A, skip=i)
            A[i] = leading_left_singular_vectors(unfold(Y, i), ranks[i])
        if history is not None:
            history.append(norm(core(S, A)))
    return core(S, A), A


def mach_hooi(X: np.ndarray, ranks, p: float, seed: int, sweeps: int):
    """The whole of Algorithm 2: coin, HOSVD initialisation, sweeps, core."""
    idx, vals = sample(X, p, seed)
    S = SampledTensor(X.shape, idx, vals, p)
    G, A = hooi(S, ranks, sweeps)
    return S, G, A


def mach_tucker2(X: np.ndarray, ranks, keep: int, p: float, seed: int, sweeps: int):
    """Algorithm 2 as a Tucker2: mode ``keep`` stays whole (identity factor)."""
    idx, vals = sample(X, p, seed)
    S = SampledTensor(X.shape, idx, vals, p)
    G, A = hooi(S, ranks, sweeps, keep=(keep,))
    return S, G, A


def mach_hosvd(X: np.ndarray, ranks, p: float, seed: int):
    """The whole of Algorithm 1."""
    idx, vals = sample(X, p, seed)
    S = SampledTensor(X.shape, idx, vals, p)
    G, A = hosvd(S, ranks)
    return S, G, A


# ----------------------------------------------------------------------------
# Reporting quantities (Section 4)
# ----------------------------------------------------------------------------

def reconstruct(G: np.ndarray, factors) -> np.ndarray:
    """G x_1 A_1 ... x_d A_d."""
    Xr = G
    for k, A in enumerate(factors):
        Xr = mode_product(Xr, A, k)
    return Xr


def relative_error(X: np.ndarray, G: np.ndarray, factors, slab: int = 0) -> float:
    """||X - G x_1 A_1 ... x_d A_d|| / ||X|| (the paper's accuracy is 1 minus
    this), computed in slabs along mode 1 when ``slab`` > 0 to bound memory."""
    X = np.asarray(X)
    if slab <= 0 or slab >= X.shape[0]:
        return norm(X - reconstruct(G, factors)) / norm(X)
    num = 0.0
    den = 0.0
    for a in range(0, X.shape[0], slab):
        b = min(X.shape[0], a + slab)
        part = reconstruct(G, [factors[0][a:b]] + list(factors[1:]))
        diff = np.asarray(X[a:b], dtype=np.float64) - part
        num += float(np.sum(diff * diff))
        den += float(np.sum(np.asarray(X[a:b], dtype=np.float64) ** 2))
    return math.sqrt(num) / math.sqrt(den)


def subspace_distance(A: np.ndarray, B: np.ndarray) -> float:
    """||A A^T - B B^T||_F / sqrt(2 r) for orthonormal A, B with r columns."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    P = A @ A.T - B @ B.T
    return float(np.linalg.norm(P) / math.sqrt(2.0 * A.shape[1]))


def fix_signs(A: np.ndarray) -> np.ndarray:
    """Flip each column so that its largest-magnitude entry (lowest index on
    ties) is positive; Tucker factors are determined only up to such flips."""
    A = np.array(A, dtype=np.float64, copy=True)
    for j in range(A.shape[1]):
        i = int(np.argmax(np.abs(A[:, j])))
        if A[i, j] < 0:
            A[:, j] = -A[:, j]
    return A


def pearson(a: np.ndarray, b: np.ndarray) -> float:
    a = np.asarray(a, dtype=np.float64) - np.mean(a)
    b = np.asarray(b, dtype=np.float64) - np.mean(b)
    return float(np.dot(a, b) / math.sqrt(np.dot(a, a) * np.dot(b, b)))
