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


def min_core_gap(G):
    """Smallest relative gap (s_j - s_{j+1}) / s_1 between consecutive
    singular values of the core unfoldings G_(k): the singular vectors inside
    each factor are determined only up to rotations of about rounding / gap."""
    G = np.asarray(G, dtype=np.float64)
    gaps = []
    for k in range(G.ndim):
        sv = np.linalg.svd(np.moveaxis(G, k, 0).reshape(G.shape[k], -1), compute_uv=False)
        if sv.size > 1 and sv[0] > 0:
            gaps.append(float(np.min(sv[:-1] - sv[1:]) / sv[0]))
    return min(gaps) if gaps else 1.0


def compare_decomposition(O, X, G_o, A_o, G_g, A_g, tol, label="", rounding=None):
    """Subspace distance per mode, core (after sign fix) and reconstruction
    error of the GPU decomposition against the oracle's, all within tol.
    With `rounding` (the unit roundoff of the path's arithmetic), the core is
    compared only when every core singular-value gap g satisfies
    rounding / g <= tol: below that, the individual singular vectors are not
    determined to tol by that arithmetic (degenerate singular values), and the
    subspaces and the reconstruction error carry the comparison."""
    for k in range(len(A_o)):
        dist = O.subspace_distance(A_o[k], A_g[k])
        assert dist <= tol, "%s mode %d subspace distance %.3e > %.1e" % (label, k, dist, tol)
        ortho = np.max(np.abs(A_g[k].T @ A_g[k] - np.eye(A_g[k].shape[1])))
        assert ortho <= max(tol, 1e-12), "%s mode %d not orthonormal: %.3e" % (label, k, ortho)
    gap = min_core_gap(G_o)
    core_compared = rounding is None or rounding / max(gap, 1e-300) <= tol
    Go = sign_fixed_core(G_o, A_o)
    Gg = sign_fixed_core(G_g, A_g)
    rel = float(np.linalg.norm(Go - Gg) / np.linalg.norm(Go))
    if core_compared:
        assert rel <= tol, "%s core relative difference %.3e > %.1e" % (label, rel, tol)
    eo = O.relative_error(X, G_o, A_o)
    eg = O.relative_error(X, G_g, A_g)
    assert abs(eo - eg) <= tol * max(1.0, eo), "%s reconstruction error %.12f vs %.12f" % (label, eg, eo)
    return {"eo": eo, "eg": eg, "core_compared": bool(core_compared), "core_rel": rel, "core_gap": gap}
