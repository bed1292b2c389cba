"""Python binding of libmach (include/mach.h): argument marshalling only.

Every step of the method runs in the CUDA kernels of libmach.so; this module
only turns torch tensors into device pointers and status codes into
exceptions.  It raises at import-time use when libmach.so is missing: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmach.so")

MACH_F32, MACH_F64 = 0, 1
PREC = {"fp64": 0, "fp32": 1, "bf16_refine": 2}
STATUS = {0: "MACH_OK", 1: "MACH_EINVAL", 2: "MACH_ENOMEM", 3: "MACH_ENOMEM_BUDGET", 4: "MACH_ECUDA",
          5: "MACH_ETIMEOUT", 6: "MACH_EBUSY", 7: "MACH_EAGAIN", 8: "MACH_EINTERNAL"}

# name -> (restype, argtypes)
_c_i64p = ctypes.POINTER(ctypes.c_int64)
_c_intp = ctypes.POINTER(ctypes.c_int)
_c_dblp = ctypes.POINTER(ctypes.c_double)
_c_pp = ctypes.POINTER(ctypes.c_void_p)
SIGNATURES = {
    "mach_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "mach_last_error": (ctypes.c_char_p, []),
    "mach_version": (ctypes.c_char_p, []),
    "mach_sample": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _c_i64p, ctypes.c_double,
                                   ctypes.c_uint64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "mach_sample_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _c_i64p, ctypes.c_double,
                                           ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                           _c_i64p, ctypes.c_void_p]),
    "mach_sample_skip": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _c_i64p, ctypes.c_double,
                                        ctypes.c_uint64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "mach_sample_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _c_i64p, ctypes.c_double,
                                        ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "mach_sample_count": (ctypes.c_int, [ctypes.c_void_p, _c_i64p]),
    "mach_sample_indices": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "mach_sample_values": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "mach_sample_fibers": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_i64p]),
    "mach_sample_free": (ctypes.c_int, [ctypes.c_void_p]),
    "mach_sample_gram": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "mach_sample_stats": (ctypes.c_int, [ctypes.c_void_p, _c_i64p, _c_i64p, _c_i64p,
                                         ctypes.POINTER(ctypes.c_uint)]),
    "mach_hooi": (ctypes.c_int, [ctypes.c_void_p, _c_intp, ctypes.c_int, ctypes.c_int, _c_pp, ctypes.c_void_p,
                                 ctypes.c_int, ctypes.c_void_p]),
    "mach_hooi_tucker2": (ctypes.c_int, [ctypes.c_void_p, _c_intp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _c_pp,
                                         ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "mach_hooi_batched": (ctypes.c_int, [_c_pp, ctypes.c_int, _c_intp, ctypes.c_int, ctypes.c_int, _c_pp, _c_pp,
                                         ctypes.c_int, ctypes.c_void_p]),
    "mach_core": (ctypes.c_int, [ctypes.c_void_p, _c_intp, _c_pp, ctypes.c_void_p, ctypes.c_void_p]),
    "mach_error": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _c_i64p, _c_intp, _c_pp,
                                  ctypes.c_void_p, _c_dblp, _c_dblp, ctypes.c_void_p]),
    "mach_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "mach_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                   _c_i64p, _c_intp, ctypes.c_double, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                   _c_i64p]),
    "mach_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, _c_intp, ctypes.c_void_p, _c_pp, _c_dblp]),
    "mach_server_stats": (ctypes.c_int, [ctypes.c_void_p, _c_i64p, _c_dblp, _c_dblp, _c_intp,
                                         ctypes.POINTER(ctypes.c_size_t)]),
    "mach_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "mach_request_bytes": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _c_i64p, _c_intp, ctypes.c_double, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_size_t)]),
    "mach_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "mach_profile_query": (ctypes.c_int, [ctypes.c_int, _c_dblp, _c_i64p, _c_dblp]),
    "mach_launch_count": (ctypes.c_int64, []),
    "mach_check_bounded_wait": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p]),
}

_lib = None


class MachError(RuntimeError):
    def __init__(self, fn: str, status: int, detail: str = ""):
        self.status = status
        super().__init__("%s failed: %s (%d)%s" % (fn, STATUS.get(status, "?"), status,
                                                 (": " + detail) if detail else ""))


def load(path: str = LIB_PATH):
    """Load libmach.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libmach.so not found at %s: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(fn: str, status: int):
    if status != 0:
        detail = load().mach_last_error().decode(errors="replace")
        raise MachError(fn, status, detail)


def _stream(stream=None) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return MACH_F32
    if t.dtype == torch.float64:
        return MACH_F64
    raise TypeError("tensor must be float32 or float64")


def _i64(vals) -> ctypes.Array:
    return (ctypes.c_int64 * len(vals))(*[int(v) for v in vals])


def _int(vals) -> ctypes.Array:
    return (ctypes.c_int * len(vals))(*[int(v) for v in vals])


def _ptrs(tensors) -> ctypes.Array:
    return (ctypes.c_void_p * len(tensors))(*[t.data_ptr() for t in tensors])


def new_factors(dims: Sequence[int], ranks: Sequence[int], device="cuda") -> List[torch.Tensor]:
    """FP64 column-major I_k x r_k factor buffers (returned as (I_k, r_k) views)."""
    return [torch.empty((int(r), int(n)), dtype=torch.float64, device=device).t() for n, r in zip(dims, ranks)]


def colmajor(A: torch.Tensor) -> torch.Tensor:
    """An (I, r) FP64 view whose storage is column-major (as the ABI expects)."""
    A = A.to(torch.float64)
    return A.t().contiguous().t()


class Sample:
    """A sampled tensor (mach_sample_t) owning its device buffers."""

    def __init__(self, x: torch.Tensor, p: float, seed: int, stream=None, skip: bool = False,
                 chunk_entries: int = 0):
        """skip=True: mach_sample_skip (reads only the sectors holding kept
        entries).  A CPU tensor x is streamed from host memory by
        mach_sample_host (chunk_entries per chunk, 0 = the default); the
        sample then lives on the current CUDA device."""
        if not x.is_contiguous():
            raise ValueError("x must be contiguous")
        lib = load()
        self._lib = lib
        self.dims = tuple(int(s) for s in x.shape)
        self.d = len(self.dims)
        self.p = float(p)
        self.seed = int(seed)
        self.dtype = x.dtype
        h = ctypes.c_void_p()
        if x.is_cuda:
            self.device = x.device
            fn = lib.mach_sample_skip if skip else lib.mach_sample
            _check("mach_sample", fn(ctypes.c_void_p(x.data_ptr()), _dtype_code(x), self.d, _i64(self.dims),
                                     self.p, ctypes.c_uint64(self.seed), _stream(stream), ctypes.byref(h)))
        else:
            if skip:
                raise ValueError("the sector-skipping sampler reads device memory")
            self.device = torch.device("cuda", torch.cuda.current_device())
            _check("mach_sample_host", lib.mach_sample_host(ctypes.c_void_p(x.data_ptr()), _dtype_code(x), self.d,
                                                            _i64(self.dims), self.p, ctypes.c_uint64(self.seed),
                                                            int(chunk_entries), _stream(stream), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("sample already freed")
        return self._h

    def count(self) -> int:
        n = ctypes.c_int64()
        _check("mach_sample_count", self._lib.mach_sample_count(self.handle, ctypes.byref(n)))
        return int(n.value)

    def indices(self, stream=None) -> torch.Tensor:
        k = self.count()
        out = torch.empty(max(k, 1), dtype=torch.int64, device=self.device)
        _check("mach_sample_indices", self._lib.mach_sample_indices(self.handle, ctypes.c_void_p(out.data_ptr()),
                                                                    out.numel(), _stream(stream)))
        return out[:k]

    def values(self, stream=None) -> torch.Tensor:
        k = self.count()
        out = torch.empty(max(k, 1), dtype=self.dtype, device=self.device)
        _check("mach_sample_values", self._lib.mach_sample_values(self.handle, ctypes.c_void_p(out.data_ptr()),
                                                                  out.numel(), _stream(stream)))
        return out[:k]

    def fibers(self, mode: int) -> int:
        n = ctypes.c_int64()
        _check("mach_sample_fibers", self._lib.mach_sample_fibers(self.handle, int(mode), ctypes.byref(n)))
        return int(n.value)

    def hooi(self, ranks: Sequence[int], sweeps: int, prec: str = "fp32",
             factors: Optional[List[torch.Tensor]] = None, warm: bool = False, core: bool = True, stream=None):
        """Algorithm 2 on this sample; returns (core or None, factors)."""
        if factors is None:
            if warm:
                raise ValueError("warm start needs factors")
            factors = new_factors(self.dims, ranks, self.device)
        else:
            factors = [colmajor(f) if f.stride(0) != 1 else f for f in factors]
        G = torch.empty(tuple(int(r) for r in ranks), dtype=torch.float64, device=self.device) if core else None
        _check("mach_hooi", self._lib.mach_hooi(self.handle, _int(ranks), int(sweeps), PREC[prec], _ptrs(factors),
                                                ctypes.c_void_p(G.data_ptr() if G is not None else 0),
                                                1 if warm else 0, _stream(stream)))
        return G, factors

    def tucker2(self, ranks: Sequence[int], keep: int, sweeps: int, prec: str = "fp32",
                factors: Optional[List[torch.Tensor]] = None, warm: bool = False, core: bool = True, stream=None):
        """mach_hooi_tucker2: mode `keep` stays whole; returns (core or None,
        factors) with None in place of the kept mode's (identity) factor."""
        full = [int(self.dims[k]) if k == keep else int(r) for k, r in enumerate(ranks)]
        if factors is None:
            if warm:
                raise ValueError("warm start needs factors")
            factors = new_factors(self.dims, [1 if k == keep else r for k, r in enumerate(full)], self.device)
        else:
            factors = [colmajor(f) if f is not None and f.stride(0) != 1 else f for f in factors]
        factors = [None if k == keep else f for k, f in enumerate(factors)]
        G = torch.empty(tuple(full), dtype=torch.float64, device=self.device) if core else None
        fptr = (ctypes.c_void_p * len(factors))(*[0 if f is None else f.data_ptr() for f in factors])
        _check("mach_hooi_tucker2", self._lib.mach_hooi_tucker2(self.handle, _int(full), int(keep), int(sweeps),
                                                                PREC[prec], fptr,
                                                                ctypes.c_void_p(G.data_ptr() if G is not None else 0),
                                                                1 if warm else 0, _stream(stream)))
        return G, factors

    def gram(self, mode: int, method: int = 0, stream=None) -> torch.Tensor:
        """mach_sample_gram: X^_(n) X^_(n)^T (raw values) as an FP64 I_n x I_n
        device tensor; method 0 exact FP64, 1 / 2 tensor cores (1 / 2 BF16
        terms)."""
        n = self.dims[mode] if 0 <= mode < self.d else 1   # the library rejects a bad mode
        out = torch.empty((n, n), dtype=torch.float64, device=self.device)
        _check("mach_sample_gram", self._lib.mach_sample_gram(self.handle, int(mode), int(method),
                                                              ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def core(self, ranks: Sequence[int], factors: Sequence[torch.Tensor], stream=None) -> torch.Tensor:
        factors = [colmajor(f) if f.stride(0) != 1 else f for f in factors]
        G = torch.empty(tuple(int(r) for r in ranks), dtype=torch.float64, device=self.device)
        _check("mach_core", self._lib.mach_core(self.handle, _int(ranks), _ptrs(factors),
                                                ctypes.c_void_p(G.data_ptr()), _stream(stream)))
        return G

    def stats(self) -> dict:
        """Eigensolver calls / iterations / unconverged solves and device status bits."""
        c, it, un = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        fl = ctypes.c_uint()
        _check("mach_sample_stats", self._lib.mach_sample_stats(self.handle, ctypes.byref(c), ctypes.byref(it),
                                                                ctypes.byref(un), ctypes.byref(fl)))
        return {"eig_calls": c.value, "eig_iters": it.value, "eig_unconverged": un.value, "flags": fl.value}

    def free(self):
        if self._h is not None:
            _check("mach_sample_free", self._lib.mach_sample_free(self._h))
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def hooi_batched(samples: Sequence["Sample"], ranks: Sequence[int], sweeps: int,
                 factors: Optional[List[List[torch.Tensor]]] = None, warm: bool = False, core: bool = True,
                 stream=None):
    """mach_hooi_batched: Algorithm 2 for every 3-way sample in one persistent
    launch (FP32 sweeps).  Returns (cores or None, factors), one entry per sample."""
    lib = load()
    B = len(samples)
    if factors is None:
        if warm:
            raise ValueError("warm start needs factors")
        factors = [new_factors(s.dims, ranks, s.device) for s in samples]
    else:
        factors = [[colmajor(f) if f.stride(0) != 1 else f for f in fs] for fs in factors]
    cores = [torch.empty(tuple(int(r) for r in ranks), dtype=torch.float64, device=s.device) for s in samples] \
        if core else None
    handles = (ctypes.c_void_p * max(B, 1))(*[s.handle.value for s in samples])
    flat = [f for fs in factors for f in fs]
    fptr = (ctypes.c_void_p * max(len(flat), 1))(*[f.data_ptr() for f in flat])
    cptr = (ctypes.c_void_p * max(B, 1))(*[c.data_ptr() for c in cores]) if core else None
    _check("mach_hooi_batched", lib.mach_hooi_batched(handles, B, _int(ranks), int(sweeps), PREC["fp32"], fptr,
                                                      cptr, 1 if warm else 0, _stream(stream)))
    return cores, factors


def sample(x: torch.Tensor, p: float, seed: int, stream=None, skip: bool = False, chunk_entries: int = 0) -> Sample:
    return Sample(x, p, seed, stream, skip, chunk_entries)


def sample_noalloc(x: torch.Tensor, p: float, seed: int, idx_out: torch.Tensor, val_out: torch.Tensor,
                   stream=None) -> int:
    """Kept (index, value) pairs written into the caller's preallocated
    idx_out (int64) and val_out (x's dtype); returns the number kept.  Raises
    MachError when the capacity min(len(idx_out), len(val_out)) is too small
    (the count is in the exception's ``n_kept``).  Nothing is allocated."""
    lib = load()
    if not x.is_contiguous():
        raise ValueError("x must be contiguous")
    if idx_out.dtype != torch.int64 or val_out.dtype != x.dtype:
        raise TypeError("idx_out must be int64 and val_out of x's dtype")
    cap = min(idx_out.numel(), val_out.numel())
    n = ctypes.c_int64(0)
    st = lib.mach_sample_noalloc(ctypes.c_void_p(x.data_ptr()), _dtype_code(x), x.dim(), _i64(x.shape),
                                 float(p), ctypes.c_uint64(seed), ctypes.c_void_p(idx_out.data_ptr()),
                                 ctypes.c_void_p(val_out.data_ptr()), cap, ctypes.byref(n), _stream(stream))
    if st != 0:
        err = MachError("mach_sample_noalloc", st, lib.mach_last_error().decode(errors="replace"))
        err.n_kept = int(n.value)
        raise err
    return int(n.value)


def error(x: torch.Tensor, core: torch.Tensor, factors: Sequence[torch.Tensor], stream=None):
    """(||X - G x A|| / ||X||, ||X||) against the dense X (one streaming pass)."""
    lib = load()
    factors = [colmajor(f) if f.stride(0) != 1 else f for f in factors]
    ranks = [int(s) for s in core.shape]
    rel = ctypes.c_double()
    xn = ctypes.c_double()
    _check("mach_error", lib.mach_error(ctypes.c_void_p(x.data_ptr()), _dtype_code(x), x.dim(),
                                        _i64(x.shape), _int(ranks), _ptrs(factors),
                                        ctypes.c_void_p(core.contiguous().data_ptr()), ctypes.byref(rel),
                                        ctypes.byref(xn), _stream(stream)))
    return float(rel.value), float(xn.value)


def request_bytes(shape, ranks, p: float, dtype=torch.float32, prec: str = "fp32") -> int:
    """Device memory the server reserves for one request of this shape."""
    lib = load()
    out = ctypes.c_size_t()
    code = MACH_F32 if dtype == torch.float32 else MACH_F64
    _check("mach_request_bytes", lib.mach_request_bytes(code, len(shape), _i64(shape), _int(ranks), float(p),
                                                        PREC[prec], ctypes.byref(out)))
    return int(out.value)


class Server:
    """Served decompositions of tensor streams (continuous batching over
    `slots` worker streams within an HBM budget); see include/mach.h."""

    def __init__(self, hbm_budget_bytes: int, slots: int):
        lib = load()
        h = ctypes.c_void_p()
        _check("mach_server_create", lib.mach_server_create(int(hbm_budget_bytes), int(slots), ctypes.byref(h)))
        self._h = h
        self._shapes = {}

    def submit(self, stream_id: int, x: torch.Tensor, ranks: Sequence[int], p: float, seed: int, sweeps: int,
               prec: str = "fp32") -> int:
        """Queue one window; x (device, contiguous) must stay alive until polled done."""
        lib = load()
        if not x.is_contiguous():
            raise ValueError("x must be contiguous")
        t = ctypes.c_int64()
        _check("mach_submit", lib.mach_submit(self._h, int(stream_id), ctypes.c_void_p(x.data_ptr()),
                                              _dtype_code(x), x.dim(), _i64(x.shape), _int(ranks), float(p),
                                              ctypes.c_uint64(seed), int(sweeps), PREC[prec], ctypes.byref(t)))
        self._shapes[t.value] = (tuple(int(v) for v in x.shape), tuple(int(r) for r in ranks))
        return t.value

    def poll(self, ticket: int):
        """None while running; then (core, [factors], rel_err) as float64 numpy arrays."""
        import numpy as np
        lib = load()
        dims, ranks = self._shapes[ticket]
        core = np.empty(ranks, dtype=np.float64)
        facs = [np.empty((r, i), dtype=np.float64) for i, r in zip(dims, ranks)]   # column-major I x r
        ptrs = (ctypes.c_void_p * len(facs))(*[f.ctypes.data for f in facs])
        done = ctypes.c_int()
        err = ctypes.c_double()
        st = lib.mach_poll(self._h, int(ticket), ctypes.byref(done), ctypes.c_void_p(core.ctypes.data),
                           ctypes.cast(ptrs, _c_pp), ctypes.byref(err))
        if not done.value:
            return None
        del self._shapes[ticket]
        _check("mach_poll", st)
        return core, [f.T for f in facs], float(err.value)

    def stats(self) -> dict:
        lib = load()
        n = ctypes.c_int64()
        p50 = ctypes.c_double()
        p99 = ctypes.c_double()
        mx = ctypes.c_int()
        used = ctypes.c_size_t()
        _check("mach_server_stats", lib.mach_server_stats(self._h, ctypes.byref(n), ctypes.byref(p50),
                                                          ctypes.byref(p99), ctypes.byref(mx), ctypes.byref(used)))
        return {"completed": n.value, "p50_ms": p50.value, "p99_ms": p99.value, "max_in_flight": mx.value,
                "budget_in_use": used.value}

    def close(self):
        if getattr(self, "_h", None):
            load().mach_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def check_bounded_wait(limit: int, arrive: bool, stream=None) -> int:
    """mach_check_bounded_wait: returns the status code (0 = the wait
    completed, 5 = MACH_ETIMEOUT: it ran out of polls and returned)."""
    return int(load().mach_check_bounded_wait(int(limit), 1 if arrive else 0, _stream(stream)))


def version() -> str:
    return load().mach_version().decode()
