"""Runs oracle decompositions of several tensors in parallel host processes
(spawned, so that no process forked after the first CUDA call holds a copy
of the CUDA context).  Test infrastructure only."""
import concurrent.futures as cf
import multiprocessing as mp
import os


def _oracle_hooi(job):
    import numpy as np
    from oracle import mach_oracle as O
    X, ranks, p, seed, sweeps = job
    S, G, A = O.mach_hooi(np.asarray(X, dtype=np.float64), ranks, p, seed, sweeps)
    return S.idx, G, A


def oracle_hooi_many(jobs, workers=None):
    """[(X, ranks, p, seed, sweeps)] -> [(kept indices, G, [A_k])] in order."""
    n = workers or max(1, min(len(jobs), (os.cpu_count() or 2)))
    with cf.ProcessPoolExecutor(n, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_oracle_hooi, jobs))
