"""Served decompositions (mach_server_* / mach_submit / mach_poll): each
window's result in the concurrent mix equals the same window decomposed
alone, warm starts chain window to window, resized windows start cold and
leave the stream state alone, admission respects the HBM budget, and a
served window matches the oracle."""
import time

import numpy as np
import pytest

from oracle import mach_oracle as O
from paper_0909_4969_gb300 import synth
from tests._gpu import compare_decomposition, mach_module, sign_fixed_core, torch

pytestmark = pytest.mark.gpu

RANKS = (4, 4, 8)
P = 0.3
SWEEPS = 3
TOL = 1e-5


def wait_all(srv, tickets, timeout_s=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t in out:
                continue
            r = srv.poll(t)
            if r is not None:
                out[t] = r
        assert time.time() - t0 < timeout_s, "served requests did not finish"
        time.sleep(0.001)
    return out


def make_streams():
    """3 streams x 4 windows of 60 x 16 x 128 (rotating by 0.01 rad per
    window), plus one resized 90 x 16 x 200 window in stream 1 after its
    second window."""
    seq = []
    for s in range(3):
        st = synth.StreamState(s, (60, 16, 128), RANKS, seed=17)
        for w in range(4):
            seq.append((s, w, st.next_window(0.01, 0.05, "float32"), False))
            if s == 1 and w == 1:
                big = synth.tucker_for_dims((90, 16, 200), RANKS, 0.05, 99, "float32")
                seq.append((s, 100, big, True))
    return seq


def alone(mach, seq):
    """The same windows one at a time, in each stream's order: the first
    window of a stream and resized windows start cold, the others warm-start
    from the stream's previous same-shape result."""
    res = {}
    prev = {}
    for s, w, X, resized in seq:
        x = torch.from_numpy(X).cuda()
        smp = mach.sample(x, P, 1000 * s + w)
        if resized or s not in prev:
            G, A = smp.hooi(RANKS, SWEEPS, "fp32")
        else:
            G, A = smp.hooi(RANKS, SWEEPS, "fp32", factors=[a.clone() for a in prev[s]], warm=True)
        err, _ = mach.error(x, G, A)
        if not resized:
            prev[s] = A
        res[(s, w)] = (G.cpu().numpy(), [a.cpu().numpy() for a in A], err)
        smp.free()
    return res


def test_mix_equals_alone_and_overlaps():
    mach = mach_module()
    seq = make_streams()
    ref = alone(mach, seq)
    srv = mach.Server(4 << 30, 3)
    xs = [torch.from_numpy(X).cuda() for _, _, X, _ in seq]
    tickets = {}
    for (s, w, X, resized), x in zip(seq, xs):
        tickets[srv.submit(s, x, RANKS, P, 1000 * s + w, SWEEPS, "fp32")] = (s, w)
    got = wait_all(srv, list(tickets))
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(seq)
    assert st["max_in_flight"] >= 2, st       # requests of different streams ran at the same time
    assert st["p99_ms"] >= st["p50_ms"] > 0.0
    for t, key in tickets.items():
        G_s, A_s, err_s = got[t]
        G_a, A_a, err_a = ref[key]
        for k in range(3):
            assert O.subspace_distance(A_s[k], A_a[k]) <= TOL, key
        Gs, Ga = sign_fixed_core(G_s, A_s), sign_fixed_core(G_a, A_a)
        assert np.linalg.norm(Gs - Ga) <= TOL * np.linalg.norm(Ga), key
        assert abs(err_s - err_a) <= TOL * max(1.0, err_a), key


def test_served_windows_match_oracle_chain():
    """One stream, three windows: the first cold (HOSVD), the next two warm
    from the previous window's factors, against the oracle run the same way."""
    mach = mach_module()
    st = synth.StreamState(7, (60, 16, 128), RANKS, seed=3)
    Xs = [st.next_window(0.01, 0.05, "float32") for _ in range(3)]
    srv = mach.Server(4 << 30, 2)
    xs = [torch.from_numpy(X).cuda() for X in Xs]
    tickets = [srv.submit(7, x, RANKS, P, 500 + w, SWEEPS, "fp32") for w, x in enumerate(xs)]
    got = wait_all(srv, tickets)
    srv.close()
    A_prev = None
    for w, (X, t) in enumerate(zip(Xs, tickets)):
        X64 = X.astype(np.float64)
        idx, vals = O.sample(X64, P, 500 + w)
        G_o, A_o = O.hooi(O.SampledTensor(X64.shape, idx, vals, P), RANKS, SWEEPS, init=A_prev)
        A_prev = A_o
        G_g, A_g, err = got[t]
        compare_decomposition(O, X.astype(np.float64), G_o, A_o, G_g, A_g, TOL, "served window %d" % w)


def test_budget_admission_and_errors():
    mach = mach_module()
    shape = (60, 16, 128)
    need = mach.request_bytes(shape, RANKS, P)
    assert need > 0
    # room for one request at a time: two slots, yet never two in flight
    srv = mach.Server(need + need // 2, 2)
    st0 = synth.StreamState(0, shape, RANKS, seed=5)
    xs = [torch.from_numpy(st0.next_window(0.01, 0.05, "float32")).cuda() for _ in range(2)]
    st1 = synth.StreamState(1, shape, RANKS, seed=5)
    xs += [torch.from_numpy(st1.next_window(0.01, 0.05, "float32")).cuda() for _ in range(2)]
    tickets = [srv.submit(i // 2, x, RANKS, P, i, SWEEPS, "fp32") for i, x in enumerate(xs)]
    wait_all(srv, tickets)
    assert srv.stats()["max_in_flight"] == 1
    # a window that can never fit the budget
    big = torch.zeros((400, 32, 2048), dtype=torch.float32, device="cuda")
    with pytest.raises(mach.MachError) as ei:
        srv.submit(3, big, RANKS, P, 1, SWEEPS, "fp32")
    assert ei.value.status == 3   # MACH_ENOMEM_BUDGET
    # invalid arguments and tickets
    with pytest.raises(mach.MachError):
        srv.submit(3, xs[0], (4, 4, 200), P, 1, SWEEPS, "fp32")
    lib = mach.load()
    import ctypes
    done = ctypes.c_int(-1)
    assert lib.mach_poll(srv._h, 987654321, ctypes.byref(done), None, None, None) == 1
    srv.close()
