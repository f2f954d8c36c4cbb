"""Stream and graph ordering of the single-problem CP route and of batch
plans, against the FP64 oracle: back-to-back sketches through one
workspace, calls of different shapes one after another on a fresh
context, a sketch right after a batch chain (whose kernels release their
dependents early), inputs copied on another stream, CUDA-graph capture and
replay with the inputs changed in place between replays, and a graph that
reads every output of a batch plan right after the plan's launch, and
workspace growth while earlier calls are still queued.  Needs a GPU."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import synth
from gpu_common import assert_sketch_close, cuda, host

pytestmark = pytest.mark.gpu

I, J = [700, 600, 800], [5000, 4000, 6000]      # Jt = 14998, P = 16384 (warp-DIT kernel)
I2, J2 = [300, 200], [2000, 1500]               # Jt = 3499, P = 4096 (slot-FFT kernel)


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


def _ref(orc, U, lam, J_, seed, D):
    ho, so = orc.make_hashes(seed, [u.shape[0] for u in U], J_, D)
    return orc.fcs_cp([u.astype(np.float64) for u in U], lam.astype(np.float64), J_, ho, so)


@pytest.mark.parametrize("shape", [(I, J), (I2, J2)])
def test_back_to_back_sketches_share_the_workspace(fcs, ctx, orc, shape):
    """Call k + 1's prep overwrites the transposed factors and the spectrum
    accumulator that call k's sketch kernel reads: it must wait for it."""
    Is, Js = shape
    R, D = 40, 6
    outs, refs = [], []
    for k in range(4):
        U, lam = synth.cp_factors(200 + k, Is, R)
        h, s = fcs.fcs_make_hashes(ctx, 300 + k, Is, Js, D)
        outs.append(fcs.fcs_sketch_cp(ctx, [cuda(u) for u in U], cuda(lam), Js, h, s))
        refs.append(_ref(orc, U, lam, Js, 300 + k, D))
    for k in range(4):
        assert_sketch_close(host(outs[k]), refs[k], what=f"call {k}")


def test_calls_of_mixed_shapes_in_a_row(fcs, orc):
    """The spectrum accumulator and tickets must start every call at zero
    whatever the previous call's FFT length and sketch count: a sequence
    mixing them on a fresh context, each against the oracle."""
    c = fcs.Context()
    seq = [([700, 600, 800], [5000, 4000, 6000], 30, 16),    # P = 16384, D = 16
           ([20, 30], [10, 12], 3, 1),                        # P = 32
           ([300, 200], [2000, 1500], 12, 9),                 # P = 4096
           ([700, 600, 800], [5000, 4000, 6000], 7, 3),       # P = 16384 again
           ([40, 50, 60], [300, 200, 100], 5, 16)]            # P = 1024
    for k, (Is, Js, R, D) in enumerate(seq):
        U, lam = synth.cp_factors(250 + k, Is, R)
        h, s = fcs.fcs_make_hashes(c, 350 + k, Is, Js, D)
        got = fcs.fcs_sketch_cp(c, [cuda(u) for u in U], cuda(lam), Js, h, s)
        assert_sketch_close(host(got), _ref(orc, U, lam, Js, 350 + k, D), what=f"call {k}")
    c.close()


def test_sketch_right_after_a_batch_chain(fcs, ctx, orc):
    """The batch class kernels let their dependents launch early.  The batch
    writes its output straight into the factor matrix of a sketch queued
    right after the chain, whose prep kernel must wait for the chain."""
    R, D = 8, 3
    Ub, lamb = synth.cp_factors(210, [64, 48], 4)
    hb, sb = fcs.fcs_make_hashes(ctx, 310, [64, 48], [40, 60], 2)
    keep = [cuda(u) for u in Ub] + [cuda(lamb)]
    U, lam = synth.cp_factors(211, I, R)
    Ug = [cuda(u) for u in U]
    out_b = Ug[0].view(-1)[:2 * 99].view(2, 99)      # Jt = 40 + 60 - 1 = 99
    p, _ = fcs.cp_problem(keep[:2], keep[2], [40, 60], hb, sb, out=out_b)
    plan = fcs.BatchPlan(ctx, [p], grain=1)
    h, s = fcs.fcs_make_hashes(ctx, 311, I, J, D)
    lamg = cuda(lam)
    for _ in range(3):
        plan.launch()
        got = fcs.fcs_sketch_cp(ctx, Ug, lamg, J, h, s)
    ref_b = orc.fcs_cp([u.astype(np.float64) for u in Ub], lamb.astype(np.float64), [40, 60],
                       host(hb), host(sb))
    assert_sketch_close(host(out_b), ref_b, what="batch output")
    U0 = host(Ug[0]).copy()
    assert_sketch_close(host(got), _ref(orc, [U0, U[1], U[2]], lam, J, 311, D),
                        what="sketch after chain")
    plan.close()


def test_inputs_copied_on_another_stream(fcs, ctx, orc):
    """The factors arrive by a copy on a side stream that the main stream
    waits for; the hash kernel runs meanwhile, the prep kernel after both."""
    R, D = 60, 5
    U, lam = synth.cp_factors(220, I, R)
    hostbuf = torch.from_numpy(np.concatenate([u.reshape(-1) for u in U])).pin_memory()
    dev = torch.full(hostbuf.shape, float("nan"), device="cuda")
    offs = np.cumsum([0] + [u.size for u in U])
    Ud = [dev[offs[n]:offs[n + 1]].view(I[n], R) for n in range(3)]
    side = torch.cuda.Stream()
    main = torch.cuda.current_stream()
    side.wait_stream(main)
    with torch.cuda.stream(side):
        dev.copy_(hostbuf, non_blocking=True)
    h, s = fcs.fcs_make_hashes(ctx, 320, I, J, D)
    main.wait_stream(side)
    got = fcs.fcs_sketch_cp(ctx, Ud, cuda(lam), J, h, s)
    assert_sketch_close(host(got), _ref(orc, U, lam, J, 320, D), what="side-stream inputs")


def test_graph_capture_and_replay(fcs, ctx, orc):
    """make_hashes + sketch captured into one CUDA graph (programmatic edges)
    and replayed on new factor values in the same buffers."""
    R, D = 30, 4
    U, lam = synth.cp_factors(230, I, R)
    Ug = [cuda(u) for u in U]
    lamg = cuda(lam)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        h, s = fcs.fcs_make_hashes(ctx, 330, I, J, D)      # warm: workspace sized
        out = fcs.fcs_sketch_cp(ctx, Ug, lamg, J, h, s)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=st):
            h2, s2 = fcs.fcs_make_hashes(ctx, 331, I, J, D)
            fcs.fcs_sketch_cp(ctx, Ug, lamg, J, h2, s2, out=out)
    for u in Ug:
        u.mul_(-0.5)
    g.replay()
    torch.cuda.synchronize()
    Un = [u * -0.5 for u in U]
    assert_sketch_close(host(out), _ref(orc, Un, lam, J, 331, D), what="graph replay")
    for u in Ug:
        u.mul_(-2.0)                       # back to the original values
    g.replay()
    torch.cuda.synchronize()
    assert_sketch_close(host(out), _ref(orc, U, lam, J, 331, D), what="second replay")
    torch.cuda.current_stream().wait_stream(st)


@pytest.mark.parametrize("Is,Js,R,D", [
    (I, J, 30, 4),                                       # P = 16384
    ([500, 400, 600], [3000, 2500, 2000], 20, 5),        # P = 8192
    (I2, J2, 12, 6),                                     # P = 4096
])
def test_graph_replays_of_the_seeded_call(fcs, orc, Is, Js, R, D):
    """fcs_sketch_cp_seeded (prep launch, then the sketch kernel as its
    programmatic dependent) captured once and replayed four times, the factors
    changed in place before each replay: every replay must equal a direct call
    on the new values (and the first one the oracle), so the sketch kernel
    never reads what prep has not yet written."""
    c = fcs.Context()
    U, lam = synth.cp_factors(260, Is, R)
    Ug = [cuda(u) for u in U]
    lamg = cuda(lam)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        out, h, s = fcs.fcs_sketch_cp_seeded(c, Ug, lamg, Js, D, 360)   # buffers sized
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=st):
            fcs.fcs_sketch_cp_seeded(c, Ug, lamg, Js, D, 361, out=out, h=h, s=s)
    torch.cuda.current_stream().wait_stream(st)
    gen = torch.Generator(device="cuda").manual_seed(7)
    for k in range(4):
        for u in Ug:
            u.mul_(-1.3).add_(torch.randn(u.shape, device="cuda", generator=gen))
        g.replay()
        torch.cuda.synchronize()
        got = host(out).copy()
        if k == 0:
            Uh = [host(u).astype(np.float64) for u in Ug]
            assert_sketch_close(got, _ref(orc, Uh, lam, Js, 361, D), what="replay 0 vs oracle")
        ref, _, _ = fcs.fcs_sketch_cp_seeded(c, Ug, lamg, Js, D, 361)
        assert_sketch_close(got, host(ref).astype(np.float64), what=f"replay {k}")
    c.close()


def test_graph_reads_batch_outputs_after_the_chain(fcs, ctx, orc):
    """A graph that launches a batch plan (one class kernel per FFT size,
    chained) and then copies every output: the copies must see every class
    finished, not only the last one."""
    shapes = [([300, 200, 250], [5000, 4000, 6000], 40, 4),   # P = 16384 (longest class)
              ([100, 120], [2000, 1500], 8, 3),               # P = 4096
              ([50, 40], [300, 200], 4, 2)]                   # P = 512 (last, short)
    probs, refs, keep = [], [], []
    for k, (Is, Js, R, D) in enumerate(shapes):
        U, lam = synth.cp_factors(240 + k, Is, R)
        ho, so = orc.make_hashes(340 + k, Is, Js, D)
        kk = [cuda(u) for u in U] + [cuda(lam), cuda(ho), cuda(so)]
        p, out = fcs.cp_problem(kk[:len(U)], kk[-3], Js, kk[-2], kk[-1])
        probs.append(p)
        keep.append((kk, out))
        refs.append(orc.fcs_cp([u.astype(np.float64) for u in U], lam.astype(np.float64), Js,
                               ho, so))
    plan = fcs.BatchPlan(ctx, probs, grain=2)
    snaps = [torch.empty_like(out) for _, out in keep]
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        plan.launch()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=st):
            plan.launch()
            for snap, (_, out) in zip(snaps, keep):
                snap.copy_(out)
    torch.cuda.current_stream().wait_stream(st)
    for _ in range(3):
        for (_, out), snap in zip(keep, snaps):
            out.zero_()
            snap.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for k, (snap, ref) in enumerate(zip(snaps, refs)):
            assert_sketch_close(host(snap), ref, what=f"graph snapshot {k}")
    plan.close()


def test_persistent_accumulator_across_sketch_counts(fcs, orc):
    """Calls at P = 16384 with D = 16, 1 and 7 (and ranks fewer than the
    groups of a sketch) in a row on a fresh context reuse one workspace for
    the spectrum accumulator and tickets: each must start from zero."""
    c = fcs.Context()
    Is, Js = [60, 50, 40], [4000, 4000, 4000]            # Jt = 11998, P = 16384
    outs, refs = [], []
    for k, (R, D) in enumerate([(3, 16), (9, 1), (2, 7), (5, 16)]):
        U, lam = synth.cp_factors(600 + k, Is, R)
        h, s = fcs.fcs_make_hashes(c, 700 + k, Is, Js, D)
        outs.append(fcs.fcs_sketch_cp(c, [cuda(u) for u in U], cuda(lam), Js, h, s))
        refs.append(_ref(orc, U, lam, Js, 700 + k, D))
    for k in range(len(outs)):
        assert_sketch_close(host(outs[k]), refs[k], what=f"call {k}")
    c.close()


def test_workspace_grows_while_earlier_calls_are_queued(fcs, orc):
    """Calls of growing size queued back to back on a fresh context with no
    host synchronisation in between: every growth of the context's
    workspace is ordered on the stream (the old buffer is released only
    after the calls queued before have run), so each call still reads its
    own buffer.  Short, P = 16384, P = 32768 and two-pass (P = 2^17) routes;
    all results against the oracle at the end."""
    c = fcs.Context()
    seq = [([20, 30], [10, 12], 3, 1),                          # P = 32
           ([300, 200], [2000, 1500], 12, 9),                   # P = 4096
           ([700, 600, 800], [5000, 4000, 6000], 30, 16),       # P = 16384
           ([120, 100, 90], [9000, 8000, 7000], 6, 2),          # P = 32768
           ([60, 50, 40], [40000, 30000, 20000], 3, 2)]         # P = 2^17, two-pass route
    inputs = []
    for k, (Is, Js, R, D) in enumerate(seq):
        U, lam = synth.cp_factors(450 + k, Is, R)
        inputs.append((U, lam, [cuda(u) for u in U], cuda(lam)))
    torch.cuda.synchronize()
    outs = []
    for k, ((Is, Js, R, D), (_, _, Ug, lg)) in enumerate(zip(seq, inputs)):
        out, _, _ = fcs.fcs_sketch_cp_seeded(c, Ug, lg, Js, D, 550 + k)
        outs.append(out)
    torch.cuda.synchronize()
    for k, ((Is, Js, R, D), (U, lam, _, _)) in enumerate(zip(seq, inputs)):
        assert_sketch_close(host(outs[k]), _ref(orc, U, lam, Js, 550 + k, D), what=f"call {k}")
    c.close()
