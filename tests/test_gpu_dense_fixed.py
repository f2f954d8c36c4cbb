"""The dense route's exact integer accumulation against the FP64 oracle: the
paths that leave the fixed-point fast path (outliers, int32 carries, the
rounding-error fallback, all-zero samples, extreme magnitudes, NaN) must give
the same sketch as the definition, eq. (FCS_asyn).  Needs a GPU."""
from __future__ import annotations

import numpy as np
import pytest

import synth
from gpu_common import SKETCH_RTOL, assert_sketch_close, cuda, host, rel_l2

pytestmark = pytest.mark.gpu

# 64 x 64 x 256: contiguous last mode with 256 entries, so every row is one
# warp unit of the row-chunk kernel and the 4096 rows spread over the CTAs.
SHAPE = (64, 64, 256)
J = [97, 131, 509]


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


def _run(fcs, ctx, T, J, ho, so):
    return host(fcs.fcs_sketch_dense(ctx, cuda(T), J, cuda(ho), cuda(so)))


def test_spikes_late_and_in_sample_rows(fcs, ctx, orc):
    """Huge entries far beyond the sampled range go through the FP32 outlier
    path; a huge entry inside a sampled row forces a coarse step, which the
    rounding-error test must catch (remainder pass).  Bins the spikes do not
    touch must keep their own relative accuracy."""
    T = synth.gaussian(31, SHAPE)
    spikes = {(63, 63, 17): 3.0e7, (40, 2, 255): -1.25e6, (0, 1, 5): 2.0e6}
    for (a, b, c), v in spikes.items():
        T[a, b, c] = np.float32(v)
    D = 3
    ho, so = orc.make_hashes(32, list(SHAPE), J, D)
    ref = orc.fcs_dense(T.astype(np.float64), J, ho, so)
    got = _run(fcs, ctx, T, J, ho, so)
    assert_sketch_close(got, ref)
    S = np.zeros_like(T)
    for (a, b, c), v in spikes.items():
        S[a, b, c] = np.float32(v)
    hit = orc.fcs_dense(S.astype(np.float64), J, ho, so) != 0
    for d in range(D):
        keep = ~hit[d]
        e = rel_l2(got[d][keep], ref[d][keep])
        assert e <= SKETCH_RTOL, f"bins without spikes, sketch {d}: {e:.3e}"


def test_int32_carries(fcs, ctx, orc):
    """All signs +1 and positive data: bin sums grow far past 2^31 steps, so
    the int32 bins wrap many times and the carries must land in the output."""
    T = synth.uniform(33, SHAPE, 1.0, 2.0)
    D = 2
    for Jc in ([1, 1, 1], [2, 3, 2]):
        ho, so = orc.make_hashes(34, list(SHAPE), Jc, D)
        so = np.ones_like(so)
        ref = orc.fcs_dense(T.astype(np.float64), Jc, ho, so)
        got = _run(fcs, ctx, T, Jc, ho, so)
        assert_sketch_close(got, ref)


def test_zero_sample_rows(fcs, ctx, orc):
    """The first rows are zero, so early CTAs sample nothing and fall back to
    FP32 accumulation; later CTAs use the integer path."""
    T = synth.gaussian(35, SHAPE)
    T.reshape(-1, SHAPE[-1])[:1200] = 0.0
    ho, so = orc.make_hashes(36, list(SHAPE), J, 4)
    ref = orc.fcs_dense(T.astype(np.float64), J, ho, so)
    assert_sketch_close(_run(fcs, ctx, T, J, ho, so), ref)


@pytest.mark.parametrize("scale", [1e-35, 1e-20, 1e20, 1e35])
def test_extreme_magnitudes(fcs, ctx, orc, scale):
    """Steps near the ends of the FP32 range (1e+-20) and magnitudes outside
    the integer path's range (1e+-35, FP32 accumulation)."""
    T = (synth.gaussian(37, SHAPE).astype(np.float64) * scale).astype(np.float32)
    assert np.all(np.isfinite(T))
    ho, so = orc.make_hashes(38, list(SHAPE), J, 2)
    ref = orc.fcs_dense(T.astype(np.float64), J, ho, so)
    assert_sketch_close(_run(fcs, ctx, T, J, ho, so), ref)


def test_nan_and_inf_propagate(fcs, ctx, orc):
    """A NaN and an Inf reach exactly the bins the oracle puts them in."""
    T = synth.gaussian(39, SHAPE)
    T[5, 60, 100] = np.nan
    T[50, 7, 3] = np.inf
    ho, so = orc.make_hashes(40, list(SHAPE), J, 2)
    ref = orc.fcs_dense(T.astype(np.float64), J, ho, so)
    got = _run(fcs, ctx, T, J, ho, so)
    bad = ~np.isfinite(ref)
    assert bad.any()
    assert np.array_equal(~np.isfinite(got), bad)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    for d in range(ref.shape[0]):
        ok = ~bad[d]
        assert rel_l2(got[d][ok], ref[d][ok]) <= SKETCH_RTOL


def test_repeat_calls_bitwise_stable_bins(fcs, ctx, orc):
    """Integer bins make each CTA's partial sums order-independent; two calls
    on the same input agree to FP32 rounding of the final adds."""
    T = synth.gaussian(41, SHAPE)
    ho, so = orc.make_hashes(42, list(SHAPE), J, 5)
    a = _run(fcs, ctx, T, J, ho, so)
    b = _run(fcs, ctx, T, J, ho, so)
    ref = orc.fcs_dense(T.astype(np.float64), J, ho, so)
    assert_sketch_close(a, ref)
    assert np.max(np.abs(a - b)) <= 1e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("strided", [False, True])
def test_invalid_hash_values_are_skipped(fcs, ctx, orc, strided):
    """Hash values outside [0, J_n) (in a leading mode and in the last mode)
    drop exactly the entries that use them, sketch by sketch; the rest
    matches the definition.  strided=True goes through the general-stride
    kernel."""
    T = synth.gaussian(43, SHAPE)
    D = 3
    ho, so = orc.make_hashes(44, list(SHAPE), J, D)
    bad = ho.copy()
    off = [0, SHAPE[0], SHAPE[0] + SHAPE[1]]
    bad[0, off[0] + 7] = J[0] + 5          # sketch 0, mode 0, index 7
    bad[1, off[2] + 100] = -3              # sketch 1, last mode, index 100
    bad[2, off[1] + 0] = 1 << 20           # sketch 2, mode 1, index 0
    ref = np.empty((D, sum(J) - 2))
    for d in range(D):
        Td = T.copy()
        hd = ho.copy()
        for n in range(3):
            sl = slice(off[n], off[n] + SHAPE[n])
            for i in np.nonzero((bad[d, sl] < 0) | (bad[d, sl] >= J[n]))[0]:
                idx = [slice(None)] * 3
                idx[n] = i
                Td[tuple(idx)] = 0.0
        ref[d] = orc.fcs_dense(Td.astype(np.float64), J, hd, so)[d]
    if strided:
        base = cuda(np.ascontiguousarray(T.transpose(2, 0, 1)))
        Tg = base.permute(1, 2, 0)
    else:
        Tg = cuda(T)
    got = host(fcs.fcs_sketch_dense(ctx, Tg, J, cuda(bad), cuda(so)))
    assert_sketch_close(got, ref)


@pytest.mark.parametrize("perm", [(2, 0, 1), (1, 2, 0), (0, 2, 1)])
def test_contiguous_mode_moved_last(fcs, ctx, orc, perm):
    """Views whose contiguous mode is not the last one: the modes are
    reordered internally (FCS does not depend on their order) so the
    integer-accumulating row kernel still runs; the sketch must equal the
    definition for the view's own mode order."""
    base = synth.gaussian(45, (48, 40, 64))
    Tv = np.ascontiguousarray(base.transpose(perm))
    I = list(Tv.shape)
    Jv = [37, 53, 29]
    ho, so = orc.make_hashes(46, I, Jv, 3)
    ref = orc.fcs_dense(Tv.astype(np.float64), Jv, ho, so)
    got = host(fcs.fcs_sketch_dense(ctx, cuda(base).permute(*perm), Jv, cuda(ho), cuda(so)))
    assert_sketch_close(got, ref)
