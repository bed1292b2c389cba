"""Seeded synthetic inputs shaped like the paper's monitoring workloads.

The paper's data are dense three-way monitoring tensors (machine id x type of
measurement x timeticks; Section 1, Table "density"; Section 4 datasets).
Those datasets are not available, so every input here is synthetic:

    X = G x_1 U_1 x_2 U_2 ... x_d U_d + E

with a seeded core G, orthonormal U_k (Q factor of a seeded Gaussian
I_k x r_k matrix) and i.i.d. Gaussian noise E scaled so that
||E||_F = eta * ||G x U||_F.  This module only synthesises data.  It holds
none of MACH's arithmetic (no coin, no HOOI) and is the one module that both
the oracle-based tests and the CUDA path's callers share.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

try:  # torch is optional for the CPU generators
    import torch
except Exception:  # pragma: no cover
    torch = None


@dataclasses.dataclass(frozen=True)
class TuckerSpec:
    dims: tuple
    ranks: tuple
    core: str = "gaussian"        # "gaussian" | "lognormal_sign"
    noise: float = 0.1            # ||E||_F / ||G x U||_F
    seed: int = 0
    dtype: str = "float64"        # storage dtype of X


def _core_np(rng: np.random.Generator, ranks, kind: str) -> np.ndarray:
    if kind == "gaussian":
        return rng.standard_normal(ranks)
    if kind == "lognormal_sign":
        mag = np.exp(rng.standard_normal(ranks))           # log-normal, sigma = 1
        sign = np.where(rng.random(ranks) < 0.5, -1.0, 1.0)
        return mag * sign
    raise ValueError("unknown core kind " + kind)


def orthonormal_np(rng: np.random.Generator, n: int, r: int) -> np.ndarray:
    q, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return q


def _expand(G: np.ndarray, Us: Sequence[np.ndarray]) -> np.ndarray:
    """Dense G x_1 U_1 ... x_d U_d for data synthesis (einsum, no MACH step)."""
    d = G.ndim
    letters = "abcdefgh"
    upper = "ABCDEFGH"
    expr = letters[:d] + "," + ",".join(upper[k] + letters[k] for k in range(d)) + "->" + upper[:d]
    return np.einsum(expr, G, *Us, optimize=True)


def tucker_numpy(spec: TuckerSpec):
    """CPU generator: returns (X, G, [U_k]) as numpy arrays (X in spec.dtype)."""
    rng = np.random.default_rng(spec.seed)
    G = _core_np(rng, spec.ranks, spec.core)
    Us = [orthonormal_np(rng, n, r) for n, r in zip(spec.dims, spec.ranks)]
    X = _expand(G, Us)
    if spec.noise > 0:
        E = rng.standard_normal(spec.dims)
        E *= spec.noise * np.linalg.norm(X) / np.linalg.norm(E)
        X = X + E
    return np.ascontiguousarray(X.astype(spec.dtype)), G, Us


def tucker_torch(spec: TuckerSpec, device="cuda", chunk_elems: int = 1 << 27):
    """Device generator for large inputs (not bit-identical to ``tucker_numpy``).

    Builds X in spec.dtype on ``device`` slab by slab along mode 1 so that no
    full-size FP64 temporary is needed.  Returns (X, G, [U_k]) with G and U_k
    as FP64 torch tensors on ``device``.
    """
    if torch is None:
        raise RuntimeError("torch is required for tucker_torch")
    gen = torch.Generator(device=device)
    gen.manual_seed(int(spec.seed))
    dt = getattr(torch, spec.dtype)
    ranks = list(spec.ranks)
    if spec.core == "gaussian":
        G = torch.randn(ranks, generator=gen, device=device, dtype=torch.float64)
    else:
        G = torch.exp(torch.randn(ranks, generator=gen, device=device, dtype=torch.float64))
        G = G * torch.where(torch.rand(ranks, generator=gen, device=device, dtype=torch.float64) < 0.5, -1.0, 1.0)
    Us = []
    for n, r in zip(spec.dims, ranks):
        # small QR on the host (keeps the device generator free of solver libraries)
        g = torch.randn(n, r, generator=gen, device=device, dtype=torch.float64).cpu().numpy()
        q, _ = np.linalg.qr(g)
        Us.append(torch.from_numpy(np.ascontiguousarray(q)).to(device))
    d = len(spec.dims)
    letters = "abcdefgh"
    upper = "ABCDEFGH"
    expr = letters[:d] + "," + ",".join(upper[k] + letters[k] for k in range(d)) + "->" + upper[:d]
    X = torch.empty(spec.dims, device=device, dtype=dt)
    rest = int(np.prod(spec.dims[1:]))
    slab = max(1, chunk_elems // max(1, rest))
    clean_sq = 0.0
    noise_sq = 0.0
    # pass 1: clean signal slabs and norms; pass 2 adds noise with the exact scale
    for a in range(0, spec.dims[0], slab):
        b = min(spec.dims[0], a + slab)
        part = torch.einsum(expr, G, Us[0][a:b], *Us[1:])
        clean_sq += float(torch.sum(part * part))
        X[a:b] = part.to(dt)
    if spec.noise > 0:
        gen2 = torch.Generator(device=device)
        gen2.manual_seed(int(spec.seed) + 0x5EED)
        for a in range(0, spec.dims[0], slab):
            b = min(spec.dims[0], a + slab)
            e = torch.randn((b - a,) + tuple(spec.dims[1:]), generator=gen2, device=device, dtype=torch.float32)
            noise_sq += float(torch.sum(e.double() * e.double()))
            del e
        scale = spec.noise * math.sqrt(clean_sq) / math.sqrt(noise_sq)
        gen2.manual_seed(int(spec.seed) + 0x5EED)
        for a in range(0, spec.dims[0], slab):
            b = min(spec.dims[0], a + slab)
            e = torch.randn((b - a,) + tuple(spec.dims[1:]), generator=gen2, device=device, dtype=torch.float32)
            X[a:b] += (e * scale).to(dt)
            del e
    return X, G, Us


# ----------------------------------------------------------------------------
# The five workloads (hosts x measurement types x timeticks families)
# ----------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    spec: TuckerSpec
    p: float
    sweeps: int
    precision: str          # "fp64" | "fp32" | "bf16_refine"


def config_plain_fp64() -> Workload:
    """100 x 50 x 200 FP64, Gaussian core 5^3, 10% noise, p = 0.1, ranks 5, 10 sweeps, seed 0."""
    return Workload("plain_fp64_100x50x200",
                    TuckerSpec((100, 50, 200), (5, 5, 5), "gaussian", 0.10, 0, "float64"),
                    0.1, 10, "fp64")


def config_tucker2_sensor() -> Workload:
    """Sensor-shaped tensor (sensors x measurement types x timeticks, the
    shape of the paper's sensor data): 54 x 4 x 5385 FP32, Tucker rank
    (5, 2, 8) plus 10% noise, p = 0.1, 10 sweeps; decomposed as a Tucker2
    with the time mode kept whole and ranks (5, 2) for the other two."""
    return Workload("tucker2_sensor_54x4x5385",
                    TuckerSpec((54, 4, 5385), (5, 2, 8), "gaussian", 0.10, 0, "float32"),
                    0.1, 10, "fp32")


def config_large_fp32(scale: int = 1000) -> Workload:
    """scale^3 FP32 (1000^3 = 4 GB at full size), core 10^3, 5% noise, p = 0.01, ranks 10, 20 sweeps."""
    return Workload("large_fp32_%dx%dx%d" % (scale, scale, scale),
                    TuckerSpec((scale, scale, scale), (10, 10, 10), "gaussian", 0.05, 0, "float32"),
                    0.01, 20, "fp32")


def config_mixed_4way(scale: int = 200) -> Workload:
    """scale^4 FP32 (200^4 = 6.4 GB at full size), log-normal x sign core 8^4, 5% noise, p = 0.05."""
    return Workload("mixed_4way_%d" % scale,
                    TuckerSpec((scale,) * 4, (8, 8, 8, 8), "lognormal_sign", 0.05, 0, "float32"),
                    0.05, 10, "bf16_refine")


def batched_dims(n: int = 512, seed: int = 0) -> List[tuple]:
    """Uneven window sizes: hosts ~ U{50..400}, types ~ U{8..32},
    timeticks = round(exp(U[ln 64, ln 2048]))."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        i1 = int(rng.integers(50, 401))
        i2 = int(rng.integers(8, 33))
        i3 = int(round(math.exp(rng.uniform(math.log(64), math.log(2048)))))
        out.append((i1, i2, i3))
    return out


def config_batched(n: int = 512, seed: int = 0) -> List[Workload]:
    """n independent FP32 tensors, ranks (4,4,8), 10% noise, p = 0.1, 10 sweeps, seed_b = b."""
    return [Workload("batched_%d" % b,
                     TuckerSpec(dims, (4, 4, 8), "gaussian", 0.10, b, "float32"), 0.1, 10, "fp32")
            for b, dims in enumerate(batched_dims(n, seed))]


@dataclasses.dataclass
class StreamWindow:
    stream: int
    window: int
    arrival_s: float
    dims: tuple
    resized: bool
    seed: int


def served_schedule(n_requests: int, n_streams: int = 64, rate_hz: float = 2000.0,
                    resize_frac: float = 0.10, seed: int = 0,
                    dims=(200, 16, 512), big_dims=(1000, 32, 4096)) -> List[StreamWindow]:
    """Poisson arrivals (seeded exponential gaps) over ``n_streams`` streams;
    ``resize_frac`` of the requests are resized to ``big_dims``."""
    rng = np.random.default_rng(seed)
    t = 0.0
    counters = [0] * n_streams
    out = []
    for k in range(n_requests):
        t += float(rng.exponential(1.0 / rate_hz))
        s = int(rng.integers(0, n_streams))
        big = bool(rng.random() < resize_frac)
        out.append(StreamWindow(s, counters[s], t, tuple(big_dims if big else dims), big,
                                seed * 1_000_003 + k))
        counters[s] += 1
    return out


def rotate_subspace(U: np.ndarray, theta: float, rng: np.random.Generator) -> np.ndarray:
    """Rotate span(U) by exactly theta: U + ((cos t - 1) U c + sin t w) c^T with
    c a random unit r-vector and w a random unit vector orthogonal to span(U)."""
    n, r = U.shape
    c = rng.standard_normal(r)
    c /= np.linalg.norm(c)
    w = rng.standard_normal(n)
    w -= U @ (U.T @ w)
    w /= np.linalg.norm(w)
    return U + np.outer((math.cos(theta) - 1.0) * (U @ c) + math.sin(theta) * w, c)


class StreamState:
    """Per-stream slowly rotating factors (theta rad per window) and a fixed core."""

    def __init__(self, stream: int, dims, ranks=(4, 4, 8), seed: int = 0):
        self.rng = np.random.default_rng(seed * 7919 + stream)
        self.dims = tuple(dims)
        self.ranks = tuple(ranks)
        self.G = self.rng.standard_normal(self.ranks)
        self.Us = [orthonormal_np(self.rng, n, r) for n, r in zip(self.dims, self.ranks)]

    def next_window(self, theta: float = 0.01, noise: float = 0.05, dtype="float32"):
        self.Us = [rotate_subspace(U, theta, self.rng) for U in self.Us]
        X = _expand(self.G, self.Us)
        E = self.rng.standard_normal(self.dims)
        E *= noise * np.linalg.norm(X) / np.linalg.norm(E)
        return np.ascontiguousarray((X + E).astype(dtype))


class StreamStateTorch:
    """Device variant of StreamState for large pools of windows: the small
    factors rotate on the host (same rotation as StreamState), the window is
    expanded and noised on the device."""

    def __init__(self, stream: int, dims, ranks=(4, 4, 8), seed: int = 0, device="cuda"):
        self.host = StreamState(stream, dims, ranks, seed)
        self.device = device
        self.gen = torch.Generator(device=device)
        self.gen.manual_seed(seed * 7919 + stream + 1)

    def next_window(self, theta: float = 0.01, noise: float = 0.05, dtype=None):
        h = self.host
        h.Us = [rotate_subspace(U, theta, h.rng) for U in h.Us]
        d = len(h.dims)
        letters, upper = "abcdefgh", "ABCDEFGH"
        expr = letters[:d] + "," + ",".join(upper[k] + letters[k] for k in range(d)) + "->" + upper[:d]
        G = torch.from_numpy(h.G).to(self.device)
        Us = [torch.from_numpy(np.ascontiguousarray(U)).to(self.device) for U in h.Us]
        X = torch.einsum(expr, G, *Us)
        E = torch.randn(X.shape, generator=self.gen, device=self.device, dtype=torch.float64)
        E *= noise * torch.linalg.vector_norm(X) / torch.linalg.vector_norm(E)
        return (X + E).to(dtype or torch.float32).contiguous()


def tucker_for_dims(dims, ranks, noise: float, seed: int, dtype="float32", core="gaussian"):
    """Convenience: one seeded Tucker tensor of the given dims (numpy)."""
    X, _, _ = tucker_numpy(TuckerSpec(tuple(dims), tuple(ranks), core, noise, seed, dtype))
    return X


def inverse_sum_tensor(n: int, dtype="float64") -> np.ndarray:
    """X_ijk = 1 / (i + j + k), i, j, k = 1..n (Section 4 synthetic example)."""
    i = np.arange(1, n + 1, dtype=np.float64)
    return (1.0 / (i[:, None, None] + i[None, :, None] + i[None, None, :])).astype(dtype)
