"""Long sketches: the FFT-based calls for 16384 < P <= 2^20 (two-pass
global-memory FFT) against the FP64 oracle -- CP route (P = 2^15 .. 2^20,
including chunking under a small workspace budget), contractions (ALL and
FREE, with and without the spectrum cache), the outer combine, batches that
mix long and short problems, a long request through the server, and the
Jt > 2^20 limit.  Needs a GPU."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import synth
from gpu_common import CONTRACT_RTOL, assert_sketch_close, cuda, host, rel_l2

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


def _cp(fcs, ctx, orc, I, J, R, D, seed, budget_ctx=None):
    U, lam = synth.cp_factors(seed, I, R)
    ho, so = orc.make_hashes(seed + 100, I, J, D)
    ref = orc.fcs_cp([u.astype(np.float64) for u in U], lam.astype(np.float64), J, ho, so)
    c = budget_ctx or ctx
    got = fcs.fcs_sketch_cp(c, [cuda(u) for u in U], cuda(lam), J, cuda(ho), cuda(so))
    assert_sketch_close(host(got), ref)
    return got


@pytest.mark.parametrize("I,J,R,D", [
    ([200, 300, 250], [8192, 8192, 8192], 5, 3),      # Jt = 24574, P = 2^15 (fused kernel)
    ([20000], [20000], 3, 2),                         # one mode: its transform is also the last
    ([400, 300, 500, 200], [9000, 7000, 5000, 6000], 40, 10),   # 150 items of 2-3 ranks
    ([300, 400], [9000, 9000], 3, 2),                 # P = 2^15, two modes
    ([1500, 300, 200], [13700, 2000, 1500], 6, 3),    # P = 2^15 at the widest scatter buffer
    ([2500, 100, 100], [9000, 5000, 4000], 3, 2),     # P = 2^15, a mode longer than 4 x 512
    ([300, 200, 100], [14000, 2000, 1000], 4, 2),     # P = 2^15 past it: the block-FFT kernel
    ([300, 400], [20000, 15000], 3, 2),               # Jt = 34999, P = 2^16
    ([3000], [300000], 2, 2),                         # P = 2^19
    ([5000], [1 << 20], 2, 1),                        # Jt = 2^20 = P, the largest
])
def test_cp_long(fcs, ctx, orc, I, J, R, D):
    _cp(fcs, ctx, orc, I, J, R, D, 41)


def test_cp_long_chunked_small_budget(fcs, orc):
    """P = 2^16 under a 6 MiB budget: the chunked path (9 of 180 transforms at a time)."""
    small = fcs.Context(budget=6 << 20)
    _cp(fcs, None, orc, [150, 120, 100], [20000, 15000, 9000], 20, 3, 42, budget_ctx=small)
    small.close()


@pytest.mark.parametrize("budget", [6 << 20, 2 << 20])
def test_cp_p15_fused_small_budget(fcs, orc, budget):
    """P = 2^15 with room for 45 (6 MiB) or 12 (2 MiB) running-product slices:
    fewer CTAs than the 60 (sketch, rank group) items, each CTA taking several."""
    small = fcs.Context(budget=budget)
    _cp(fcs, None, orc, [150, 120, 100], [8000, 9000, 7000], 20, 3, 42, budget_ctx=small)
    small.close()


def test_cp_p15_invalid_hashes_dropped(fcs, ctx, orc):
    """Hash values outside [0, J_n) are skipped by the P = 2^15 kernel, as by
    the count-sketch kernel of the two-pass route: no access leaves the buffer."""
    I, J, R, D = [90, 80, 70], [9000, 8000, 7000], 4, 2
    U, lam = synth.cp_factors(47, I, R)
    ho, so = orc.make_hashes(48, I, J, D)
    bad = ho.copy()
    bad[:, 5] = -3                                   # mode 0, entry 5
    bad[:, I[0] + 7] = J[1]                          # mode 1, entry 7
    keep = np.ones_like(ho, dtype=bool)
    keep[:, 5] = keep[:, I[0] + 7] = False
    U0 = [u.astype(np.float64).copy() for u in U]
    U0[0][5] = 0.0                                   # the oracle sees those entries as zero
    U0[1][7] = 0.0
    ref = orc.fcs_cp(U0, lam.astype(np.float64), J, np.where(keep, ho, 0), so)
    got = fcs.fcs_sketch_cp(ctx, [cuda(u) for u in U], cuda(lam), J, cuda(bad), cuda(so))
    assert_sketch_close(host(got), ref)


def _contract_case(fcs, ctx, orc, cache: bool):
    I, J, D, B = [50, 60], [20000, 30000], 2, 2           # Jt = 49999, P = 2^16
    T = synth.gaussian(43, I)
    ho, so = orc.make_hashes(44, I, J, D)
    fT = orc.fcs_dense(T.astype(np.float64), J, ho, so)
    fTg = cuda(fT.astype(np.float32))
    fT = fT.astype(np.float32).astype(np.float64)
    u = [synth.unit_vectors(45 + n, B, I[n]) for n in range(2)]
    ug = [cuda(x) for x in u]
    hg, sg = cuda(ho), cuda(so)
    if cache:
        fcs.fcs_cache_spectra(ctx, True)
    for _ in range(2 if cache else 1):
        _, raw = fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_ALL, fTg, ug, I, J, hg, sg, raw=True)
        raw = host(raw)
        for b in range(B):
            vb = [x[b].astype(np.float64) for x in u]
            ref = orc.contract_all(fT, vb, J, ho, so)
            r1 = orc.fcs_cp([x[:, None] for x in vb], None, J, ho, so)
            scale = np.linalg.norm(fT, axis=1) * np.linalg.norm(r1, axis=1)
            assert np.max(np.abs(raw[b] - ref) / scale) <= CONTRACT_RTOL
        for m in (0, 1):
            vv = [None if n == m else ug[n] for n in range(2)]
            _, rawf = fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_FREE, fTg, vv, I, J, hg, sg,
                                       free_mode=m, raw=True)
            rawf = host(rawf)
            for b in range(B):
                vb = [x[b].astype(np.float64) for x in u]
                ref = orc.contract_free(fT, vb, m, J, ho, so)
                for d in range(D):
                    assert rel_l2(rawf[b, d], ref[d]) <= CONTRACT_RTOL
    if cache:
        fcs.fcs_cache_spectra(ctx, False)


def test_contract_long(fcs, ctx, orc):
    _contract_case(fcs, ctx, orc, cache=False)


def test_contract_long_cached(fcs, ctx, orc):
    _contract_case(fcs, ctx, orc, cache=True)


def test_outer_long(fcs, ctx, orc):
    nb, D, L = 2, 3, 20000                                 # Lo = 39999, P = 2^16
    g = np.random.default_rng(46)
    fa = g.standard_normal((nb, D, L)).astype(np.float32)
    fb = g.standard_normal((nb, D, L)).astype(np.float32)
    got = host(fcs.fcs_sketch_outer(ctx, cuda(fa), cuda(fb)))
    for b in range(nb):
        ref = orc.outer_combine(fa[b].astype(np.float64), fb[b].astype(np.float64))
        assert_sketch_close(got[b], ref)


def test_batch_mixes_long_and_short(fcs, ctx, orc):
    shapes = [([100, 120, 90], [3000, 2000, 1000], 7, 3),       # P = 8192
              ([80, 90, 70], [9000, 8000, 7000], 5, 2),         # P = 2^15
              ([60, 50], [700, 900], 4, 4)]                     # P = 2048
    probs, refs = [], []
    for k, (I, J, R, D) in enumerate(shapes):
        U, lam = synth.cp_factors(50 + k, I, R)
        ho, so = orc.make_hashes(60 + k, I, J, D)
        keep = [cuda(u) for u in U] + [cuda(lam), cuda(ho), cuda(so)]   # alive while the plan runs
        p, out = fcs.cp_problem(keep[:len(U)], keep[-3], J, keep[-2], keep[-1])
        probs.append((p, out, keep))
        refs.append(orc.fcs_cp([u.astype(np.float64) for u in U], lam.astype(np.float64), J,
                               ho, so))
    fcs.fcs_batch_sketch_cp(ctx, [p for p, _, _ in probs])
    for (p, out, _), ref in zip(probs, refs):
        assert_sketch_close(host(out), ref)


def test_batch_two_long_problems_linked_and_replayed(fcs, ctx, orc):
    """Two P = 2^15 problems in one plan with short ones: the first long
    problem is linked after the chain's last class (its CTAs start while the
    chain drains), the second follows it on the same scratch.  Both the plain
    launch and a captured replay after the factors change in place must give
    the oracle's sketches."""
    shapes = [([100, 120, 90], [3000, 2000, 1000], 7, 3),       # P = 8192
              ([80, 90, 70], [9000, 8000, 7000], 5, 2),         # P = 2^15, linked
              ([60, 70, 50], [8000, 9000, 6000], 3, 3),         # P = 2^15, after it
              ([60, 50], [700, 900], 4, 4)]                     # P = 2048
    probs, keep, host_in = [], [], []
    for k, (I, J, R, D) in enumerate(shapes):
        U, lam = synth.cp_factors(80 + k, I, R)
        ho, so = orc.make_hashes(90 + k, I, J, D)
        dev = [cuda(u) for u in U] + [cuda(lam), cuda(ho), cuda(so)]
        p, out = fcs.cp_problem(dev[:len(U)], dev[-3], J, dev[-2], dev[-1])
        probs.append(p)
        keep.append((dev, out))
        host_in.append((U, lam, J, ho, so))

    def refs(scale):
        return [orc.fcs_cp([u.astype(np.float64) * (scale if n == 0 else 1.0)
                            for n, u in enumerate(U)], lam.astype(np.float64), J, ho, so)
                for U, lam, J, ho, so in host_in]

    plan = fcs.BatchPlan(ctx, probs)
    plan.launch()
    torch.cuda.synchronize()
    for k, ((_, out), ref) in enumerate(zip(keep, refs(1.0))):
        assert_sketch_close(host(out), ref, what=f"plain launch, problem {k}")
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        plan.launch()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=st):
            plan.launch()
    torch.cuda.current_stream().wait_stream(st)
    for dev, out in keep:
        dev[0].mul_(-1.5)                                # mode-1 factor, in place
        out.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    for k, ((_, out), ref) in enumerate(zip(keep, refs(-1.5))):
        assert_sketch_close(host(out), ref, what=f"graph replay, problem {k}")
    plan.close()


def test_server_long_request(fcs, ctx, orc):
    I, J, R, D = [120, 100, 90], [9000, 8000, 7000], 6, 2       # P = 2^15
    U, lam = synth.cp_factors(70, I, R)
    srv = fcs.FcsServer(streams=2)
    out = np.zeros((D, sum(J) - 2), dtype=np.float32)
    res = srv.wait(srv.submit_cp(U, lam, J, D, seed=71, out=out), 120.0)
    assert res.state == 2 and res.status == 0
    h, s = fcs.fcs_make_hashes(ctx, 71, I, J, D)
    ref = host(fcs.fcs_sketch_cp(ctx, [cuda(u) for u in U], cuda(lam), J, h, s))
    assert_sketch_close(out, ref)
    srv.close()


def test_beyond_two_to_the_twenty(fcs, ctx):
    I, J = [10, 10], [600000, 600000]                           # Jt > 2^20
    U = [torch.zeros((10, 1), device="cuda")] * 2
    h = torch.zeros((1, 20), dtype=torch.int32, device="cuda")
    s = torch.ones((1, 20), dtype=torch.int8, device="cuda")
    with pytest.raises(fcs.FcsError) as e:
        fcs.fcs_sketch_cp(ctx, U, None, J, h, s)
    assert e.value.code == fcs.FCS_EUNSUPPORTED
