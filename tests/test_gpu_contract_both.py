"""fcs_contract_both: T(v_1..v_N) and T(v_1, .., I, .., v_N) from one set of
transforms (eqs. T_uvw and T_Ivw) against the FP64 oracle, and against the
two separate fcs_contract calls.  Needs a GPU."""
from __future__ import annotations

import numpy as np
import pytest

import synth
from gpu_common import CONTRACT_RTOL, cuda, host, rel_l2

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


def _case(fcs, ctx, orc, I, J, D, B, m, seed, same):
    T = synth.gaussian(seed, I)
    ho, so = orc.make_hashes(seed + 1, I, J, D)
    fT = orc.fcs_dense(T.astype(np.float64), J, ho, so).astype(np.float32)
    if same:
        u = synth.unit_vectors(seed + 2, B, I[0])
        vecs = [u] * len(I)
    else:
        vecs = [synth.unit_vectors(seed + 2 + n, B, I[n]) for n in range(len(I))]
    fTg, hg, sg = cuda(fT), cuda(ho), cuda(so)
    vg = [cuda(v) for v in vecs]
    ma, mf, ra, rf = (host(x) for x in fcs.fcs_contract_both(ctx, fTg, vg, I, J, hg, sg,
                                                             free_mode=m, raw=True))
    fT64 = fT.astype(np.float64)
    scales = np.zeros(B)
    for b in range(B):
        vb = [v[b].astype(np.float64) for v in vecs]
        ref_all = orc.contract_all(fT64, vb, J, ho, so)
        r1 = orc.fcs_cp([x[:, None] for x in vb], None, J, ho, so)
        scale = np.linalg.norm(fT64, axis=1) * np.linalg.norm(r1, axis=1)
        scales[b] = scale.max()
        err = np.abs(ra[b] - ref_all) / scale
        assert err.max() <= CONTRACT_RTOL, f"T(v..v) b={b}: {err.max():.3e}"
        assert abs(ma[b] - orc.median(ref_all[:, None])[0]) <= CONTRACT_RTOL * scale.max()
        ref_free = orc.contract_free(fT64, vb, m, J, ho, so)
        for d in range(D):
            e = rel_l2(rf[b, d], ref_free[d])
            assert e <= CONTRACT_RTOL, f"T(..I..) b={b} d={d}: {e:.3e}"
        mref = orc.median(ref_free)
        assert np.linalg.norm(mf[b] - mref) <= CONTRACT_RTOL * np.linalg.norm(ref_free, axis=1).max()
    # the separate calls give the same estimates to FP32 rounding
    sa = host(fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_ALL, fTg, vg, I, J, hg, sg))
    sf = host(fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_FREE, fTg,
                               [v if n != m else None for n, v in enumerate(vg)], I, J,
                               hg, sg, free_mode=m))
    assert np.array_equal(sf, mf) or rel_l2(mf, sf) <= 1e-6
    assert np.all(np.abs(ma - sa) <= CONTRACT_RTOL * scales)


@pytest.mark.parametrize("m", [0, 1, 2])
def test_both_every_free_mode(fcs, ctx, orc, m):
    _case(fcs, ctx, orc, [30, 25, 40], [37, 23, 51], 5, 4, m, 61, same=False)


def test_both_rtpm_shape(fcs, ctx, orc):
    """Symmetric use (the same u in every mode), J_n = 2000 (P = 8192), D = 5."""
    _case(fcs, ctx, orc, [60, 60, 60], [2000, 2000, 2000], 5, 6, 0, 71, same=True)


def test_both_order4_even_D(fcs, ctx, orc):
    _case(fcs, ctx, orc, [9, 8, 7, 6], [20, 30, 25, 15], 10, 3, 2, 81, same=False)


def test_both_long_transform(fcs, ctx, orc):
    """P = 2^16: the long-FFT route runs the two contractions in turn."""
    _case(fcs, ctx, orc, [12, 10, 9], [20000, 20000, 3000], 2, 2, 1, 91, same=False)
