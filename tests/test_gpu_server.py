"""The request server (continuous batching): served results equal direct
calls, each result is the same alone and in a mix, contractions run against
resident sketches, and admission, cancellation and bounded waits behave.
Failures are made on the host (oversized requests, unknown sketches, a
request that cannot be admitted in time); nothing faults or hangs the GPU.
Needs a GPU."""
from __future__ import annotations

import threading
import time

import numpy as np
import pytest
import torch

import synth
from gpu_common import CONTRACT_RTOL, SKETCH_RTOL, cuda, host, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fcs():
    import paper_2106_13062_gb300 as m
    m.build()
    return m


@pytest.fixture(scope="module")
def ctx(fcs):
    c = fcs.Context()
    yield c
    c.close()


def _shape(g):
    N = int(g.integers(3, 5))
    I = [int(g.integers(20, 400)) for _ in range(N)]
    J = [int(g.integers(64, 1500)) for _ in range(N)]
    return I, J, int(g.integers(1, 40)), int(g.integers(1, 8))


def _direct(fcs, ctx, U, lam, J, D, seed):
    h, s = fcs.fcs_make_hashes(ctx, seed, [u.shape[0] for u in U], J, D)
    out = fcs.fcs_sketch_cp(ctx, [cuda(u) for u in U], cuda(lam), J, h, s)
    return host(out), h, s


def _close(a, b, rtol):
    return all(rel_l2(a[d], b[d]) <= rtol for d in range(b.shape[0]))


def test_served_equals_direct(fcs, ctx):
    g = np.random.default_rng(1)
    srv = fcs.FcsServer(streams=3, max_inflight=16, max_batch=8)
    jobs = []
    for k in range(24):
        I, J, R, D = _shape(g)
        U, lam = synth.cp_factors(100 + k, I, R)
        out = np.zeros((D, sum(J) - len(J) + 1), dtype=np.float32)
        t = srv.submit_cp(U, lam, J, D, seed=500 + k, out=out)
        jobs.append((t, U, lam, J, D, 500 + k, out))
    for t, U, lam, J, D, seed, out in jobs:
        res = srv.wait(t, 60.0)
        assert res.state == 2 and res.status == 0 and res.latency_s > 0
        ref, _, _ = _direct(fcs, ctx, U, lam, J, D, seed)
        assert _close(out, ref, SKETCH_RTOL)
    st = srv.stats()
    assert st.completed == 24 and st.failed == 0
    assert st.rounds >= 1 and st.p99_latency_s >= st.p50_latency_s > 0
    srv.close()


def test_result_same_alone_and_in_mix(fcs):
    g = np.random.default_rng(2)
    I, J, R, D = [150, 220, 90], [700, 900, 400], 24, 6
    U, lam = synth.cp_factors(7, I, R)
    srv = fcs.FcsServer(streams=4, max_inflight=48, max_batch=16)
    alone = np.zeros((D, sum(J) - 2), dtype=np.float32)
    srv.wait(srv.submit_cp(U, lam, J, D, seed=77, out=alone), 60.0)
    # the same request submitted in the middle of a burst from two threads
    mixed = np.zeros_like(alone)
    tickets = []

    def burst(seed0):
        gg = np.random.default_rng(seed0)
        for k in range(20):
            I2, J2, R2, D2 = _shape(gg)
            U2, l2 = synth.cp_factors(seed0 * 100 + k, I2, R2)
            o2 = np.zeros((D2, sum(J2) - len(J2) + 1), dtype=np.float32)
            tickets.append(srv.submit_cp(U2, l2, J2, D2, seed=k, out=o2))
    th = threading.Thread(target=burst, args=(3,))
    th.start()
    mid = srv.submit_cp(U, lam, J, D, seed=77, out=mixed)
    burst(4)
    th.join()
    res = srv.wait(mid, 60.0)
    assert res.state == 2
    for t in tickets:
        assert srv.wait(t, 60.0).state == 2
    assert srv.stats().max_inflight_seen > 1       # it really ran in a mix
    assert _close(mixed, alone, SKETCH_RTOL)
    srv.close()


def _contract_refs(orc, sk, I, J, ho, so, u, m=0):
    """FP64 oracle contractions of the (FP32) sketch sk with u in every mode:
    per-sketch T(u,u,u) and its Cauchy-Schwarz scale ||FCS_d T|| ||FCS_d(u o u o u)||,
    and per-sketch T(I,u,u) with free mode m."""
    fT = sk.astype(np.float64)
    B, D = u.shape[0], sk.shape[0]
    ref, scale = np.zeros((B, D)), np.zeros((B, D))
    refs = np.zeros((B, D, I[m]))
    for b in range(B):
        vb = [u[b].astype(np.float64)] * len(I)
        ref[b] = orc.contract_all(fT, vb, J, ho, so)
        r1 = orc.fcs_cp([x[:, None] for x in vb], None, J, ho, so)
        scale[b] = np.linalg.norm(fT, axis=1) * np.linalg.norm(r1, axis=1)
        refs[b] = orc.contract_free(fT, vb, m, J, ho, so)
    return ref, scale, refs


def _assert_contract_close(orc, r_all, r_free, ref, scale, refs):
    """Medians within the contraction bar of the oracle's medians: T(u,u,u) on
    the Cauchy-Schwarz scale, T(I,u,u) in relative L2 of the largest sketch."""
    merr = np.abs(r_all - orc.median(ref.T)) / scale.max(axis=1)
    assert merr.max() <= CONTRACT_RTOL, f"T(u,u,u) median error {merr.max():.3e}"
    for b in range(refs.shape[0]):
        e = np.linalg.norm(r_free[b] - orc.median(refs[b]))
        assert e <= CONTRACT_RTOL * np.linalg.norm(refs[b], axis=1).max()


def test_contractions_on_resident_sketch(fcs, ctx, orc):
    """Served T(u,u,u) and T(I,u,u) against a resident sketch equal the
    oracle's contractions of that same sketch (copied out by the request that
    made it resident) and the direct library calls, at the contraction bar."""
    I, J, R, D, B = [60, 60, 60], [300, 300, 300], 8, 5, 7
    U, lam = synth.cp_factors(9, I, R)
    srv = fcs.FcsServer(streams=2)
    sk = np.zeros((D, sum(J) - 2), dtype=np.float32)
    t = srv.submit_cp(U, lam, J, D, seed=91, out=sk, keep_resident=True)
    res = srv.wait(t, 60.0)
    assert res.state == 2 and res.sketch_id > 0
    sid = res.sketch_id
    u = synth.unit_vectors(10, B, 60)
    r_all = np.zeros(B, dtype=np.float32)
    r_free = np.zeros((B, 60), dtype=np.float32)
    t1 = srv.submit_contract(sid, I, J, fcs.FCS_CONTRACT_ALL, [u, u, u], r_all)
    t2 = srv.submit_contract(sid, I, J, fcs.FCS_CONTRACT_FREE, [None, u, u], r_free)
    assert srv.wait(t1, 60.0).state == 2 and srv.wait(t2, 60.0).state == 2
    ho, so = orc.make_hashes(91, I, J, D)
    ref, scale, refs = _contract_refs(orc, sk, I, J, ho, so, u)
    _assert_contract_close(orc, r_all, r_free, ref, scale, refs)
    # the direct library calls on the same sketch
    ug, hg, sg = cuda(u), cuda(ho), cuda(so)
    a = host(fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_ALL, cuda(sk), [ug] * 3, I, J, hg, sg))
    b = host(fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_FREE, cuda(sk), [None, ug, ug], I, J,
                              hg, sg, free_mode=0))
    assert (np.abs(r_all - a) / scale.max(axis=1)).max() <= CONTRACT_RTOL
    for k in range(B):
        assert np.linalg.norm(r_free[k] - b[k]) <= CONTRACT_RTOL * np.linalg.norm(refs[k], axis=1).max()
    assert srv.release(sid) == 0
    with pytest.raises(fcs.FcsError) as e:        # released sketches are gone
        srv.submit_contract(sid, I, J, fcs.FCS_CONTRACT_ALL, [u, u, u], r_all)
    assert e.value.code == fcs.FCS_EINVAL
    srv.close()


def test_contractions_same_alone_and_in_mix(fcs, orc):
    """Both contraction kinds against a resident sketch give the same result
    when served alone on an idle server and when submitted in the middle of a
    burst of CP sketch requests from two threads (rounds overlapping on the
    device), within the contraction bar; both equal the oracle's."""
    I, J, R, D, B = [120, 120, 120], [900, 900, 900], 12, 6, 9
    U, lam = synth.cp_factors(21, I, R)
    srv = fcs.FcsServer(streams=4, max_inflight=48, max_batch=16)
    sk = np.zeros((D, sum(J) - 2), dtype=np.float32)
    res = srv.wait(srv.submit_cp(U, lam, J, D, seed=22, out=sk, keep_resident=True), 60.0)
    assert res.state == 2
    sid = res.sketch_id
    u = synth.unit_vectors(23, B, 120)

    def submit_both():
        ra = np.zeros(B, dtype=np.float32)
        rf = np.zeros((B, 120), dtype=np.float32)
        ta = srv.submit_contract(sid, I, J, fcs.FCS_CONTRACT_ALL, [u, u, u], ra)
        tf = srv.submit_contract(sid, I, J, fcs.FCS_CONTRACT_FREE, [None, u, u], rf)
        return ta, tf, ra, rf

    ta, tf, alone_a, alone_f = submit_both()
    assert srv.wait(ta, 60.0).state == 2 and srv.wait(tf, 60.0).state == 2
    tickets = []

    def burst(seed0):
        gg = np.random.default_rng(seed0)
        for k in range(20):
            I2, J2, R2, D2 = _shape(gg)
            U2, l2 = synth.cp_factors(seed0 * 100 + k, I2, R2)
            o2 = np.zeros((D2, sum(J2) - len(J2) + 1), dtype=np.float32)
            tickets.append(srv.submit_cp(U2, l2, J2, D2, seed=k, out=o2))
    th = threading.Thread(target=burst, args=(5,))
    th.start()
    ta, tf, mix_a, mix_f = submit_both()
    burst(6)
    th.join()
    assert srv.wait(ta, 60.0).state == 2 and srv.wait(tf, 60.0).state == 2
    for t in tickets:
        assert srv.wait(t, 60.0).state == 2
    assert srv.stats().max_inflight_seen > 1       # it really ran in a mix
    ho, so = orc.make_hashes(22, I, J, D)
    ref, scale, refs = _contract_refs(orc, sk, I, J, ho, so, u)
    assert (np.abs(mix_a - alone_a) / scale.max(axis=1)).max() <= CONTRACT_RTOL
    for k in range(B):
        assert np.linalg.norm(mix_f[k] - alone_f[k]) <= \
            CONTRACT_RTOL * np.linalg.norm(refs[k], axis=1).max()
    _assert_contract_close(orc, alone_a, alone_f, ref, scale, refs)
    _assert_contract_close(orc, mix_a, mix_f, ref, scale, refs)
    srv.close()


def test_admission_cancel_and_bounded_wait(fcs):
    I, J, R, D = [400, 400, 400], [2000, 2000, 2000], 64, 4
    U, lam = synth.cp_factors(11, I, R)
    need = 3 * 400 * 64 * 4 + 64 * 4 + D * 1200 * 5 + D * 5998 * 4
    # an arena that holds one request at a time: the second must wait
    srv = fcs.FcsServer(streams=2, max_inflight=1, max_batch=1,
                        arena_bytes=3 * need, staging_bytes=64 << 20)
    outs = [np.zeros((D, 5998), dtype=np.float32) for _ in range(3)]
    tk = [srv.submit_cp(U, lam, J, D, seed=k, out=outs[k]) for k in range(3)]
    # the last one is still queued behind the single slot: cancel it
    assert srv.cancel(tk[2]) in (0, 1)
    r0 = srv.wait(tk[0], 60.0)
    r1 = srv.wait(tk[1], 60.0)
    assert r0.state == 2 and r1.state == 2
    assert srv.stats().max_inflight_seen == 1
    # requests that can never fit are refused at submission
    big = [np.zeros((4000, 256), dtype=np.float32)] * 3
    with pytest.raises(fcs.FcsError) as e:
        srv.submit_cp(big, None, [2000] * 3, 4, seed=1,
                      out=np.zeros((4, 5998), dtype=np.float32))
    assert e.value.code == fcs.FCS_ENOMEM_BUDGET
    # malformed request
    with pytest.raises(fcs.FcsError) as e:
        srv.submit_cp(U, lam, J, 0, seed=1, out=outs[0])
    assert e.value.code == fcs.FCS_EINVAL
    # a contraction against a sketch that does not exist
    with pytest.raises(fcs.FcsError):
        srv.submit_contract(12345, I, J, fcs.FCS_CONTRACT_ALL,
                            [np.zeros((1, 400), np.float32)] * 3, np.zeros(1, np.float32))
    srv.close()


def test_wait_times_out_while_queue_is_held(fcs):
    """A producer that keeps the single slot busy: a waiter with a short limit
    gets FCS_ETIMEOUT and the server stays usable."""
    I, J, R, D = [1000, 1000, 1000], [5000] * 3, 100, 10
    U, lam = synth.cp_factors(12, I, R)
    srv = fcs.FcsServer(streams=1, max_inflight=1, max_batch=1)
    outs = [np.zeros((D, 14998), dtype=np.float32) for _ in range(6)]
    tk = [srv.submit_cp(U, lam, J, D, seed=k, out=outs[k]) for k in range(6)]
    res = srv.wait(tk[-1], 1e-4)
    assert res.state in (0, 1)                     # not finished within 0.1 ms
    for t in tk:
        assert srv.wait(t, 120.0).state == 2
    srv.close()


def test_destroy_with_queued_requests(fcs):
    I, J, R, D = [300, 300, 300], [1000] * 3, 50, 8
    U, lam = synth.cp_factors(13, I, R)
    srv = fcs.FcsServer(streams=1, max_inflight=1, max_batch=1)
    outs = [np.zeros((D, 2998), dtype=np.float32) for _ in range(10)]
    for k in range(10):
        srv.submit_cp(U, lam, J, D, seed=k, out=outs[k])
    t0 = time.time()
    srv.close()                                    # finishes in-flight, cancels the rest
    assert time.time() - t0 < 60.0
