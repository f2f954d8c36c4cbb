"""Entry recovery (decompressing rule of the Kronecker / tensor-contraction
compression subsections) on every kernel the library dispatches to, and the
NaN results promised for out-of-range indices and gather bins.  Needs a GPU.

fcs_recover picks one of three kernels:
  * packed 16-bit tables, sketches staged in shared memory: Jt < 8192,
    N <= 7, sketches + tables <= 220 KiB;
  * 32-bit tables and sketches staged in shared memory: every J_n <= 32767 and
    sketches + tables <= 220 KiB (Jt >= 8192, or N = 8);
  * the generic kernel: sketches gathered from global memory, tables staged
    in shared memory when D * sum(I_n) * 4 <= 96 KiB, else read from global
    memory (D = 16 with Jt = 4000, D = 10 with Jt = 8998, J_n > 32767).
The cases below reach each branch; raw gathers must equal the oracle's
bit for bit and medians the oracle's median within FP32 rounding."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import synth
from gpu_common import cuda, host

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


def _jt(J):
    return sum(J) - len(J) + 1


def _smem_bytes(I, J, D):
    """Shared memory of the two staged kernels (sketches + packed tables)."""
    return ((D * _jt(J) * 4 + 15) // 16) * 16 + sum(I) * ((D + 1) // 2) * 4


# (I, J, D, branch) -- the branch is what the dispatch rule above selects
PATHS = [
    ([50, 60, 70], [100] * 3, 4, "packed"),
    ([300, 200, 100], [3000] * 3, 5, "staged32"),                 # Jt = 8998
    ([5, 6, 7, 3, 4, 5, 6, 7], [4, 5, 3, 6, 2, 4, 5, 3], 3, "staged32"),  # N = 8
    ([100, 100, 100], [1334] * 3, 16, "generic_smem_tables"),     # Jt = 4000, D = 16
    ([400, 300, 200], [3000] * 3, 10, "generic_smem_tables"),     # Jt = 8998, D = 10
    ([1000, 600, 400], [1334] * 3, 16, "generic_global_tables"),  # tables 128 KB
    ([100, 50], [40000, 7], 2, "generic_smem_tables"),            # J_1 > 32767
]


def _branch(I, J, D):
    sm2 = _smem_bytes(I, J, D)
    if _jt(J) < 8192 and len(I) <= 7 and sm2 <= 220 * 1024:
        return "packed"
    if all(j <= 32767 for j in J) and sm2 <= 220 * 1024:
        return "staged32"
    return "generic_smem_tables" if D * sum(I) * 4 <= 96 * 1024 else "generic_global_tables"


@pytest.mark.parametrize("I,J,D,branch", PATHS)
def test_recover_every_kernel(fcs, ctx, orc, I, J, D, branch):
    assert _branch(I, J, D) == branch          # the case reaches the intended kernel
    M = 200_003                                 # several CTAs' shares and a ragged tail
    sk = synth.gaussian(900 + D, (D, _jt(J)))
    ho, so = orc.make_hashes(901 + D, I, J, D)
    idx = synth.sample_indices(902 + D, M, I)
    out, raw = fcs.fcs_recover(ctx, cuda(sk), I, J, cuda(ho), cuda(so), cuda(idx), raw=True)
    ref, rref = orc.recover(sk.astype(np.float64), I, J, ho, so, idx, return_raw=True)
    assert np.array_equal(host(raw).astype(np.float64), rref)
    np.testing.assert_allclose(host(out), ref, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("I,J,D,branch", [PATHS[3], PATHS[5], PATHS[1]])
def test_recover_every_kernel_batched(fcs, ctx, orc, I, J, D, branch):
    nb, M = 3, 40_001
    sk = synth.gaussian(910, (nb, D, _jt(J)))
    ho, so = orc.make_hashes(911, I, J, D)
    idx = np.stack([synth.sample_indices(912 + b, M, I) for b in range(nb)])
    got = host(fcs.fcs_recover(ctx, cuda(sk), I, J, cuda(ho), cuda(so), cuda(idx)))
    for b in range(nb):
        ref = orc.recover(sk[b].astype(np.float64), I, J, ho, so, idx[b])
        np.testing.assert_allclose(got[b], ref, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("I,J,D,branch", PATHS)
def test_recover_out_of_range_index_is_nan(fcs, ctx, orc, I, J, D, branch):
    """An index outside [0, I_n) gives NaN in the median and in every raw
    value of its sample; the kernels test the index before any load, so the
    other samples are unaffected."""
    M = 5000
    sk = synth.gaussian(920, (D, _jt(J)))
    ho, so = orc.make_hashes(921, I, J, D)
    idx = synth.sample_indices(922, M, I)
    bad = np.arange(7, M, 97)
    g = np.random.default_rng(923)
    for k, q in enumerate(bad):
        n = int(g.integers(0, len(I)))
        idx[q, n] = [I[n], -1, 2**31 - 1, -2**31][k % 4]
    out, raw = fcs.fcs_recover(ctx, cuda(sk), I, J, cuda(ho), cuda(so), cuda(idx), raw=True)
    out, raw = host(out), host(raw)
    good = np.setdiff1d(np.arange(M), bad)
    assert np.isnan(out[bad]).all()
    assert np.isnan(raw[:, bad]).all()
    ref, rref = orc.recover(sk.astype(np.float64), I, J, ho, so, idx[good], return_raw=True)
    assert np.array_equal(raw[:, good].astype(np.float64), rref)
    np.testing.assert_allclose(out[good], ref, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("J", [[40, 50, 60], [6000, 6000, 6000]])
def test_contract_free_gather_out_of_range_is_nan(fcs, ctx, J):
    """The free-mode gather of T(.., I, ..) reads z_d at h_m(i); a table value
    outside [0, P) (P the FFT length) gives NaN for that i, both on the
    in-CTA route (P <= 16384) and on the two-pass route (P = 32768); the
    other entries are those of the call with valid tables."""
    I = [300, 200, 100]
    D, B = 3, 4
    Jt = _jt(J)
    P = 1 << max(4, (Jt - 1).bit_length())
    sk = cuda(synth.gaussian(930, (D, Jt)))
    h, s = fcs.fcs_make_hashes(ctx, 931, I, J, D)
    v = [cuda(synth.unit_vectors(932 + n, B, I[n])) for n in range(3)]
    vecs = [None, v[1], v[2]]
    ok_med, ok_raw = fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_FREE, sk, vecs, I, J, h, s,
                                      free_mode=0, raw=True)
    hb = h.clone()
    bad = [3, 77, 150, 299]
    for k, i in enumerate(bad):
        hb[k % D, i] = [-1, P, P + 7, 2**31 - 1][k]
    med, raw = fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_FREE, sk, vecs, I, J, hb, s,
                                free_mode=0, raw=True)
    raw, ok_raw = host(raw), host(ok_raw)
    for d in range(D):
        mine = [i for k, i in enumerate(bad) if k % D == d]
        assert np.isnan(raw[:, d, mine]).all()
        mask = np.ones(I[0], bool)
        mask[mine] = False
        np.testing.assert_allclose(raw[:, d, mask], ok_raw[:, d, mask], rtol=1e-6, atol=1e-6)
    # the median over D of values one of which is NaN is not specified
    _ = (med, ok_med)
