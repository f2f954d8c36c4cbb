"""Batched CP-route sketches: a plan (one transpose launch, then one kernel per
FFT length, chained by programmatic dependent launch) over problems of uneven
order, sizes, rank and sketch length must give each problem's fcs_sketch_cp
result (and the oracle's) within the sketch tolerance.  Needs a GPU."""
from __future__ import annotations

import os

import numpy as np
import pytest
import torch

import synth
from gpu_common import assert_sketch_close, cuda, host

pytestmark = pytest.mark.gpu

# (I, J, R, D): orders 1..4, FFT lengths 16 .. 16384
SHAPES = [
    ([20, 20, 20], [8, 8, 8], 5, 1),
    ([300], [100], 4, 2),
    ([64, 80], [600, 700], 9, 3),
    ([10, 12, 9, 11], [50, 60, 70, 80], 3, 2),
    ([5, 6, 7], [2, 3, 4], 2, 1),
    ([200, 150, 300], [5000, 5000, 5000], 7, 4),
    ([90, 70, 80], [1500, 1200, 1000], 33, 5),
    ([1000, 700], [2000, 3000], 64, 10),
    ([100, 90, 80, 70], [1100, 1200, 1000, 1100], 6, 3),   # P = 8192, short hash ranges
    ([1500, 40], [5000, 1000], 5, 2),                 # P = 8192, long ranges, a mode > 4 x 256
]


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


def _make(fcs, ctx, orc=None, seed=0):
    probs, refs, keep = [], [], []
    for k, (I, J, R, D) in enumerate(SHAPES):
        U, lam = synth.cp_factors(seed + k, I, R)
        Ug = [cuda(u) for u in U]
        lamg = cuda(lam)
        h, s = fcs.fcs_make_hashes(ctx, 100 + seed + k, I, J, D)
        pr, out = fcs.cp_problem(Ug, lamg, J, h, s)
        probs.append(pr)
        refs.append(fcs.fcs_sketch_cp(ctx, Ug, lamg, J, h, s))
        keep.append((U, lam, Ug, lamg, h, s, out, I, J))
    return probs, refs, keep


@pytest.mark.parametrize("grain", [0, 1, 3, 64])
def test_batch_matches_single_problem_calls(fcs, ctx, grain):
    probs, refs, keep = _make(fcs, ctx)
    fcs.fcs_batch_sketch_cp(ctx, probs, grain=grain)
    for k, ref in enumerate(refs):
        assert_sketch_close(host(keep[k][6]), host(ref), what=f"problem {k}")


def test_batch_matches_oracle(fcs, ctx, orc):
    probs, refs, keep = _make(fcs, ctx, seed=7)
    fcs.fcs_batch_sketch_cp(ctx, probs)
    for k, (U, lam, Ug, lamg, h, s, out, I, J) in enumerate(keep):
        if np.prod(I) * U[0].shape[1] > 5e7:
            continue                       # the large ones are covered above
        ref = orc.fcs_cp([u.astype(np.float64) for u in U], lam.astype(np.float64), J,
                         host(h), host(s))
        assert_sketch_close(host(out), ref, what=f"problem {k}")


def test_plan_relaunch_and_graph_replay(fcs, ctx):
    probs, refs, keep = _make(fcs, ctx, seed=3)
    plan = fcs.BatchPlan(ctx, probs, grain=4)
    plan.launch()
    torch.cuda.synchronize()
    first = [host(k[6]).copy() for k in keep]
    for o in keep:
        o[6].zero_()
    plan.launch()                          # accumulators are cleared each launch
    torch.cuda.synchronize()
    for k, f in enumerate(first):
        assert_sketch_close(host(keep[k][6]), f, what=f"relaunch {k}")
    # capture one launch into a CUDA graph and replay it on new factor values
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        plan.launch()                      # warm the stream
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            plan.launch()
    for k, item in enumerate(keep):
        for u in item[2]:
            u.mul_(-1.0)                   # new inputs in the same buffers
        item[6].zero_()
    g.replay()
    torch.cuda.synchronize()
    for k, item in enumerate(keep):
        N = len(item[7])
        sign = -1.0 if N % 2 else 1.0      # every factor negated: (-1)^N
        assert_sketch_close(host(item[6]), sign * first[k], what=f"graph {k}")
    plan.close()


def test_autotune_and_cache_file(fcs, tmp_path):
    path = str(tmp_path / "fcs_tune.txt")
    os.environ["FCS_AUTOTUNE_CACHE"] = path
    try:
        c = fcs.Context()
        probs, refs, keep = _make(fcs, c, seed=11)
        g = fcs.fcs_batch_autotune(c, probs)
        assert g in (1, 2, 4, 8, 16, 32, 64)
        assert os.path.exists(path)
        line = open(path).read().split()
        assert int(line[1]) == g
        fcs.fcs_batch_sketch_cp(c, probs)   # uses the tuned grain
        for k, ref in enumerate(refs):
            assert_sketch_close(host(keep[k][6]), host(ref), what=f"tuned {k}")
        c.close()
    finally:
        del os.environ["FCS_AUTOTUNE_CACHE"]


def test_batch_rejects_bad_problem(fcs, ctx):
    probs, refs, keep = _make(fcs, ctx)
    probs[2].R = 0
    with pytest.raises(fcs.FcsError) as e:
        fcs.fcs_batch_sketch_cp(ctx, probs)
    assert e.value.code == fcs.FCS_EINVAL


def test_plan_outliving_its_context(fcs):
    """C-ABI order context-destroy-then-plan-destroy: the plan is detached from
    the context and its destruction must not touch the freed context (a long
    problem gives the plan its own scratch too)."""
    import ctypes as C
    L = fcs.lib()
    own = fcs.Context()
    probs, _, keep = _make(fcs, own, seed=7)
    U, lam = synth.cp_factors(99, [80, 90, 70], 3)
    Ug, lamg = [cuda(u) for u in U], cuda(lam)
    h, s = fcs.fcs_make_hashes(own, 98, [80, 90, 70], [9000, 8000, 7000], 2)   # P = 2^15
    pr, out = fcs.cp_problem(Ug, lamg, [9000, 8000, 7000], h, s)
    probs.append(pr)
    arr = fcs._problem_array(probs)
    ph = C.c_void_p()
    own.check(L.fcs_batch_plan_create(own.handle, len(probs), arr, 0, C.byref(ph)))
    own.check(L.fcs_batch_plan_launch(own.handle, ph))
    torch.cuda.synchronize()
    assert L.fcs_destroy(own.handle) == fcs.FCS_OK
    own._h = C.c_void_p()                        # already destroyed above
    assert L.fcs_batch_plan_destroy(ph) == fcs.FCS_OK
    # a Python plan closes before its context
    c2 = fcs.Context()
    probs2, _, keep2 = _make(fcs, c2, seed=8)
    plan = fcs.BatchPlan(c2, probs2)
    c2.close()
    assert not plan._h.value


# (engine for P = 8192, thread multiplier of the slot FFT, items per CTA)
CLASS_SHAPES = [(0, 1, 1), (0, 2, 1), (0, 1, 2), (0, 2, 2), (0, 1, 4), (0, 2, 4),
                (1, 1, 1), (1, 1, 2), (1, 1, 4)]


@pytest.mark.parametrize("eng,ntm,ipc", CLASS_SHAPES)
def test_every_class_shape_matches_single_calls(fcs, ctx, eng, ntm, ipc):
    """Each engine, thread multiplier and items-per-CTA count the autotuner
    may pick, applied to every FFT-length class of the batch (P = 16 ...
    16384: the warp-DIT engine is an option at P = 8192 and the only engine at
    P = 16384, the slot FFT runs the other sizes), gives each problem's
    fcs_sketch_cp result."""
    probs, refs, keep = _make(fcs, ctx, seed=21)
    lens = sorted({1 << max(4, (sum(J) - len(J)).bit_length()) for _, _, _, _, _, _, _, _, J
                   in keep}, reverse=True)
    assert 8192 in lens and 16384 in lens
    classes = []
    for P in lens:
        e = 1 if P == 16384 else (eng if P == 8192 else 0)
        classes.append((P, ntm if e == 0 else 1, ipc, e))
    plan = fcs.BatchPlan(ctx, probs, grain=2, classes=classes)
    grain, got = plan.config()
    assert grain == 2
    assert [(p, t, i, e) for p, t, i, _, e in got] == classes
    plan.launch()
    torch.cuda.synchronize()
    for k, ref in enumerate(refs):
        assert_sketch_close(host(keep[k][6]), host(ref), what=f"shape {ntm}x{ipc} problem {k}")
    plan.close()


def _uniform_batch(fcs, ctx, n, I, J, R, D, seed):
    probs, refs, keep = [], [], []
    for k in range(n):
        U, lam = synth.cp_factors(seed + k, I, R)
        Ug, lamg = [cuda(u) for u in U], cuda(lam)
        h, s = fcs.fcs_make_hashes(ctx, seed + 500 + k, I, J, D)
        pr, out = fcs.cp_problem(Ug, lamg, J, h, s)
        probs.append(pr)
        refs.append(fcs.fcs_sketch_cp(ctx, Ug, lamg, J, h, s))
        keep.append((Ug, lamg, h, s, out))
    return probs, refs, keep


def test_autotuner_picks_class_shapes(fcs, tmp_path):
    """Two batch shapes are autotuned: 400 tiny problems (P = 32, rank 1, one
    sketch: many light items, all resident at once) and two problems whose
    few items carry long columns (P = 2048, I_n = 2000, rank 2, two
    sketches: the Count Sketch of 2000 entries per column dominates, so twice
    the threads per transform should pay).  The plans created afterwards
    with grain 0 carry exactly the grain and class shapes the tuner stored
    (read back from the cache file), the two batch shapes get different
    class shapes, and every result equals fcs_sketch_cp's."""
    path = str(tmp_path / "fcs_tune_classes.txt")
    os.environ["FCS_AUTOTUNE_CACHE"] = path
    try:
        c = fcs.Context()
        chosen = []
        for n, I, J, R, D, seed in [(400, [6, 5, 7], [10, 11, 9], 1, 1, 1000),
                                    (2, [2000, 2000, 2000], [300, 400, 350], 2, 2, 2000)]:
            probs, refs, keep = _uniform_batch(fcs, c, n, I, J, R, D, seed)
            g = fcs.fcs_batch_autotune(c, probs)
            plan = fcs.BatchPlan(c, probs)               # grain 0: the tuned entry
            grain, cls = plan.config()
            assert grain == g and len(cls) == 1
            P, ntm, ipc, nt, eng = cls[0]
            assert ntm in (1, 2) and ipc in (1, 2, 4) and nt >= 32 and eng == 0
            # the cache file holds the same choice
            stored = {}
            for line in open(path):
                tok = line.split()
                stored[int(tok[1])] = stored.get(int(tok[1]), []) + [tuple(
                    int(x) for x in t.split(":")) for t in tok[2:]]
            assert any((P.bit_length() - 2, ntm, ipc, eng) in v for v in stored.values())
            plan.launch()
            torch.cuda.synchronize()
            for k, ref in enumerate(refs):
                assert_sketch_close(host(keep[k][4]), host(ref), what=f"tuned P={P} {k}")
            plan.close()
            chosen.append((P, ntm, ipc, grain))
        print(f"\nautotuned (P, threads x, items per CTA, grain): {chosen}")
        assert chosen[0][1:3] != chosen[1][1:3], chosen
        c.close()
    finally:
        del os.environ["FCS_AUTOTUNE_CACHE"]
