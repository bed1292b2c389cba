"""Shared helpers for the GPU parity tests (no method arithmetic here: the
expected values always come from oracle/)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def mach_module():
    need_gpu()
    import __graft_entry__ as ge
    ge.build()
    from paper_0909_4969_gb300 import mach
    mach.load()
    return mach


def signs(A):
    """+1/-1 per column making the largest-magnitude entry positive (lowest index on ties)."""
    A = np.asarray(A)
    s = np.ones(A.shape[1])
    for j in range(A.shape[1]):
        i = int(np.argmax(np.abs(A[:, j])))
        s[j] = -1.0 if A[i, j] < 0 else 1.0
    return s


def sign_fixed_core(G, factors):
    """Flip core slices consistently with the sign fix of every factor."""
    G = np.array(G, dtype=np.float64, copy=True)
    for k, A in enumerate(factors):
        s = signs(A)
        shape = [1] * G.ndim
        shape[k] = -1
        G = G * s.reshape(shape)
    return G


def compare_decomposition(O, X, G_o, A_o, G_g, A_g, tol, label=""):
    """Subspace distance per mode, core (after sign fix) and reconstruction
    error of the GPU decomposition against the oracle's, all within tol."""
    for k in range(len(A_o)):
        dist = O.subspace_distance(A_o[k], A_g[k])
        assert dist <= tol, "%s mode %d subspace distance %.3e > %.1e" % (label, k, dist, tol)
        ortho = np.max(np.abs(A_g[k].T @ A_g[k] - np.eye(A_g[k].shape[1])))
        assert ortho <= max(tol, 1e-12), "%s mode %d not orthonormal: %.3e" % (label, k, ortho)
    Go = sign_fixed_core(G_o, A_o)
    Gg = sign_fixed_core(G_g, A_g)
    rel = np.linalg.norm(Go - Gg) / np.linalg.norm(Go)
    assert rel <= tol, "%s core relative difference %.3e > %.1e" % (label, rel, tol)
    eo = O.relative_error(X, G_o, A_o)
    eg = O.relative_error(X, G_g, A_g)
    assert abs(eo - eg) <= tol * max(1.0, eo), "%s reconstruction error %.12f vs %.12f" % (label, eg, eo)
    return eo, eg
