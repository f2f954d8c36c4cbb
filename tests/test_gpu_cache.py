"""The spectrum cache of fcs_contract (fcs_cache_spectra / fcs_forget):
cached contractions agree with the oracle, the library's own sketch calls
invalidate what they overwrite, fcs_forget drops a stale entry, and a cached
spectrum is safe to use from another stream.  Needs a GPU."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import synth
from gpu_common import CONTRACT_RTOL, cuda, host, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fcs():
    import paper_2106_13062_gb300 as m
    m.build()
    return m


def _ref_all(orc, fT, vecs, J, ho, so):
    B = vecs[0].shape[0]
    return np.stack([orc.contract_all(fT, [v[b].astype(np.float64) for v in vecs], J, ho, so)
                     for b in range(B)])


def _check(got, ref, fT, vecs, J, ho, so, orc):
    # Cauchy-Schwarz scale of each inner product (see gpu_common)
    B = vecs[0].shape[0]
    for b in range(B):
        r1 = orc.fcs_cp([v[b].astype(np.float64)[:, None] for v in vecs], None, J, ho, so)
        scale = np.linalg.norm(fT, axis=1) * np.linalg.norm(r1, axis=1)
        assert np.max(np.abs(got[b] - ref[b]) / scale) <= CONTRACT_RTOL


def test_cached_contractions(fcs, orc):
    ctx = fcs.Context()
    fcs.fcs_cache_spectra(ctx, True)
    I, J, D, B = [40, 40, 40], [300, 300, 300], 4, 5
    T = synth.gaussian(3, I)
    ho, so = orc.make_hashes(4, I, J, D)
    hg, sg = cuda(ho), cuda(so)
    fTg = fcs.fcs_sketch_dense(ctx, cuda(T), J, hg, sg)
    fT = host(fTg).astype(np.float64)
    u = synth.unit_vectors(5, B, 40)
    vecs = [u, u, u]
    ref = _ref_all(orc, fT, vecs, J, ho, so)
    for _ in range(3):                       # first call fills the cache, then hits
        _, raw = fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_ALL, fTg, [cuda(u)] * 3, I, J, hg, sg,
                                  raw=True)
        _check(host(raw), ref, fT, vecs, J, ho, so, orc)
    # FREE contractions share the cached spectrum
    _, rawf = fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_FREE, fTg, [None, cuda(u), cuda(u)], I, J,
                               hg, sg, free_mode=0, raw=True)
    rawf = host(rawf)
    for b in range(B):
        rf = orc.contract_free(fT, [u[b].astype(np.float64)] * 3, 0, J, ho, so)
        for d in range(D):
            assert rel_l2(rawf[b, d], rf[d]) <= CONTRACT_RTOL
    ctx.close()


def test_library_writes_invalidate(fcs, orc):
    """A new dense sketch written into the same buffer must not reuse the old
    spectrum."""
    ctx = fcs.Context()
    fcs.fcs_cache_spectra(ctx, True)
    I, J, D, B = [30, 30, 30], [200, 200, 200], 3, 4
    ho, so = orc.make_hashes(6, I, J, D)
    hg, sg = cuda(ho), cuda(so)
    u = synth.unit_vectors(7, B, 30)
    out = torch.empty((D, sum(J) - 2), dtype=torch.float32, device="cuda")
    for seed in (8, 9):
        T = synth.gaussian(seed, I)
        fcs.fcs_sketch_dense(ctx, cuda(T), J, hg, sg, out=out)
        fT = host(out).astype(np.float64)
        _, raw = fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_ALL, out, [cuda(u)] * 3, I, J, hg, sg,
                                  raw=True)
        _check(host(raw), _ref_all(orc, fT, [u] * 3, J, ho, so), fT, [u] * 3, J, ho, so, orc)
    ctx.close()


def test_forget_and_disable(fcs, orc):
    """An in-place change made outside the library is invisible to the cache
    until fcs_forget (the documented contract); disabling drops everything."""
    ctx = fcs.Context()
    fcs.fcs_cache_spectra(ctx, True)
    I, J, D, B = [25, 25, 25], [150, 150, 150], 2, 3
    ho, so = orc.make_hashes(10, I, J, D)
    hg, sg = cuda(ho), cuda(so)
    u = cuda(synth.unit_vectors(11, B, 25))
    fTg = fcs.fcs_sketch_dense(ctx, cuda(synth.gaussian(12, I)), J, hg, sg)
    a = fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_ALL, fTg, [u] * 3, I, J, hg, sg)
    a = host(a).copy()
    fTg.mul_(2.0)
    stale = fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_ALL, fTg, [u] * 3, I, J, hg, sg)
    np.testing.assert_allclose(host(stale), a, rtol=1e-5, atol=1e-6 * np.abs(a).max())
    fcs.fcs_forget(ctx, fTg)
    fresh = fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_ALL, fTg, [u] * 3, I, J, hg, sg)
    np.testing.assert_allclose(host(fresh), 2.0 * a, rtol=1e-5, atol=1e-6 * np.abs(a).max())
    fTg.mul_(0.5)
    fcs.fcs_cache_spectra(ctx, False)
    off = fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_ALL, fTg, [u] * 3, I, J, hg, sg)
    np.testing.assert_allclose(host(off), a, rtol=1e-5, atol=1e-6 * np.abs(a).max())
    ctx.close()


def test_cached_spectrum_on_another_stream(fcs, orc):
    ctx = fcs.Context()
    fcs.fcs_cache_spectra(ctx, True)
    I, J, D, B = [50, 50, 50], [400, 400, 400], 3, 6
    ho, so = orc.make_hashes(13, I, J, D)
    hg, sg = cuda(ho), cuda(so)
    T = synth.gaussian(14, I)
    u = synth.unit_vectors(15, B, 50)
    ug = cuda(u)
    fTg = fcs.fcs_sketch_dense(ctx, cuda(T), J, hg, sg)
    fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_ALL, fTg, [ug] * 3, I, J, hg, sg)   # fills
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        _, raw = fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_ALL, fTg, [ug] * 3, I, J, hg, sg,
                                  raw=True)
    side.synchronize()
    fT = host(fTg).astype(np.float64)
    _check(host(raw), _ref_all(orc, fT, [u] * 3, J, ho, so), fT, [u] * 3, J, ho, so, orc)
    ctx.close()
