"""Parity of every C-ABI entry point (CUDA path, called through the binding)
against the FP64 oracle on identical seeded FP32 inputs.  Needs a GPU."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import synth
from gpu_common import (CONTRACT_RTOL, SKETCH_RTOL, assert_sketch_close, cuda,
                        host, rel_l2)

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


# ------------------------------------------------------------------ hashes
HASH_CASES = [
    (1, [20, 20, 20], [8, 8, 8], 1),
    (2, [1000, 1000, 1000], [5000, 5000, 5000], 10),
    (3, [500, 500, 500], [2000, 2000, 2000], 5),
    (4, [512, 512, 512, 512], [1024, 1024, 1024, 1024], 10),
    (5, [1], [1], 1),
    (6, [7, 1, 13, 2, 5, 3, 11, 4], [3, 1, 7, 2, 9, 1, 4, 8], 16),
    (7, [100000], [65537], 2),
    (2**64 - 1, [333, 77], [1 << 20, 3], 3),
]


@pytest.mark.parametrize("seed,I,J,D", HASH_CASES)
def test_hashes_bit_exact(fcs, ctx, orc, seed, I, J, D):
    h, s = fcs.fcs_make_hashes(ctx, seed, I, J, D)
    ho, so = orc.make_hashes(seed, I, J, D)
    assert np.array_equal(host(h), ho)
    assert np.array_equal(host(s), so)


# ------------------------------------------------------------------ dense
def _dense_case(fcs, ctx, orc, T, J, D, seed, Tdev=None):
    I = list(T.shape)
    ho, so = orc.make_hashes(seed, I, J, D)
    ref = orc.fcs_dense(T.astype(np.float64), J, ho, so)
    Tg = cuda(T) if Tdev is None else Tdev
    got = fcs.fcs_sketch_dense(ctx, Tg, J, cuda(ho), cuda(so))
    assert_sketch_close(host(got), ref)
    return ref


def test_dense_tiny_cp_tensor(fcs, ctx, orc):
    """20^3 rank-5 CP tensor, J_n = 8 (Jt = 22), D = 1, hash seed 1."""
    U, lam = synth.cp_factors(0, [20, 20, 20], 5)
    _dense_case(fcs, ctx, orc, synth.cp_dense(U, lam), [8, 8, 8], 1, 1)


@pytest.mark.parametrize("shape,J,D", [
    ([37, 41, 53], [13, 29, 7], 3),        # last dim not a multiple of 4
    ([30, 50, 100], [64, 64, 64], 4),      # vector path, ragged 128-chunk
    ([3, 5, 7, 9], [4, 6, 3, 8], 2),       # order 4
    ([1000], [97], 5),                     # order 1 (plain Count Sketch)
    ([16, 16, 16], [1, 1, 1], 2),          # Jt = 1
    ([24, 20, 12], [31, 17, 5], 16),       # D = 16
    ([1, 1, 4], [3, 2, 2], 1),             # degenerate modes
])
def test_dense_shapes(fcs, ctx, orc, shape, J, D):
    T = synth.gaussian(11, shape)
    _dense_case(fcs, ctx, orc, T, J, D, 12)


def test_dense_strided_views(fcs, ctx, orc):
    """A permuted view and a sliced view go through the element strides."""
    base = synth.gaussian(13, (40, 30, 20))
    J = [9, 21, 14]
    Tdev = cuda(base)
    _dense_case(fcs, ctx, orc, np.ascontiguousarray(base.transpose(2, 0, 1)), J, 2, 14,
                Tdev=Tdev.permute(2, 0, 1))
    _dense_case(fcs, ctx, orc, np.ascontiguousarray(base[:, ::2, 1:17]), J, 2, 14,
                Tdev=Tdev[:, ::2, 1:17])


def test_dense_batched_with_table_slice(fcs, ctx, orc):
    """Five order-2 sketches in one launch, with the hash pairs of modes 3..4
    of an order-4 table."""
    I4, J4, D = [48, 40, 36, 64], [31, 17, 29, 23], 4
    ho, so = orc.make_hashes(15, I4, J4, D)
    mats = synth.gaussian(16, (5, 36, 64))
    off = I4[0] + I4[1]
    h2, s2 = ho[:, off:].copy(), so[:, off:].copy()
    got = host(fcs.fcs_sketch_dense(ctx, cuda(mats), J4[2:], cuda(h2), cuda(s2),
                                    batched=True))
    for b in range(5):
        ref = orc.fcs_dense(mats[b].astype(np.float64), J4[2:], h2, s2)
        assert_sketch_close(got[b], ref)


def test_dense_ldh_on_wide_table(fcs, ctx, orc):
    """ldh lets a call read a run of modes from a wider table in place."""
    import ctypes as C
    I4, J4, D = [48, 40, 36, 64], [31, 17, 29, 23], 3
    ho, so = orc.make_hashes(17, I4, J4, D)
    hg, sg = cuda(ho), cuda(so)
    off = I4[0] + I4[1]
    A = synth.gaussian(18, (36, 64))
    Ag = cuda(A)
    Jt = sum(J4[2:]) - 1
    out = torch.empty((D, Jt), dtype=torch.float32, device="cuda")
    L = fcs.lib()
    rc = L.fcs_sketch_dense(ctx.handle, 2, fcs._arr(C.c_int64, [36, 64]), None,
                            fcs._arr(C.c_int32, J4[2:]), D, C.c_void_p(Ag.data_ptr()),
                            C.c_void_p(hg.data_ptr() + 4 * off),
                            C.c_void_p(sg.data_ptr() + off), sum(I4),
                            C.c_void_p(out.data_ptr()), 1, 0, 0)
    ctx.check(rc)
    ref = orc.fcs_dense(A.astype(np.float64), J4[2:], ho[:, off:], so[:, off:])
    assert_sketch_close(host(out), ref)


# ------------------------------------------------------------------ CP
def _cp_case(fcs, ctx, orc, I, J, R, D, seed, lam_none=False, ld_pad=0):
    U, lam = synth.cp_factors(seed, I, R)
    if lam_none:
        lam = None
    ho, so = orc.make_hashes(seed + 100, I, J, D)
    ref = orc.fcs_cp([u.astype(np.float64) for u in U],
                     None if lam is None else lam.astype(np.float64), J, ho, so)
    Ug = []
    for u in U:
        w = np.zeros((u.shape[0], R + ld_pad), dtype=np.float32)
        w[:, :R] = u
        Ug.append(cuda(w)[:, :R])
    got = fcs.fcs_sketch_cp(ctx, Ug, None if lam is None else cuda(lam), J,
                            cuda(ho), cuda(so))
    assert_sketch_close(host(got), ref)
    return U, lam, ho, so, ref


def test_cp_tiny_and_dense_agree(fcs, ctx, orc):
    """20^3 rank 5, J_n = 8: CP route == dense route on the same tensor."""
    U, lam, ho, so, ref = _cp_case(fcs, ctx, orc, [20, 20, 20], [8, 8, 8], 5, 1, 0)
    T = synth.cp_dense(U, lam)
    dense_gpu = host(fcs.fcs_sketch_dense(ctx, cuda(T), [8, 8, 8], cuda(ho), cuda(so)))
    assert_sketch_close(dense_gpu, ref, rtol=1e-5)


@pytest.mark.parametrize("I,J,R,D,kw", [
    ([37, 50, 23], [11, 29, 5], 7, 3, {}),               # P = 64
    ([300], [100], 4, 2, {}),                            # order 1, P = 128
    ([64, 80], [600, 700], 9, 2, {"lam_none": True}),    # P = 2048
    ([10, 12, 9, 11], [50, 60, 70, 80], 3, 2, {"ld_pad": 5}),  # P = 512
    ([5, 6, 7], [2, 3, 4], 2, 1, {}),                    # Jt = 7, P = 16
    ([200, 200, 200], [5000, 5000, 5000], 5, 2, {}),     # P = 16384
    ([90, 70, 80], [1500, 1200, 1000], 33, 4, {}),       # P = 4096, many ranks
    # P = 16384 (warp-DIT engine): order 1 with a tail beyond the prefetch,
    # uneven orders 2 and 4, few ranks with D = 16, and the full-width
    # scatter buffer (J = P)
    ([3000], [12000], 3, 2, {}),
    ([700, 900], [9000, 7000], 6, 3, {"lam_none": True}),
    ([40, 700, 30, 1200], [4000, 3000, 2000, 5000], 4, 2, {"ld_pad": 3}),
    ([50, 60, 70], [8192, 4096, 2048], 2, 16, {}),
    ([100], [16384], 2, 1, {}),
    ([200, 150, 100, 120], [4000, 4000, 4000, 4000], 3, 2, {}),   # 4-row scatter buffer
    # P = 8192 (warp-DIT engine of 256 threads, 8-row scatter buffer): order 1
    # with a tail beyond the prefetch, orders 2 and 4, D = 16 with few ranks,
    # J = P, and the shortest scatter-buffer rows
    ([3000], [6000], 3, 2, {}),
    ([700, 900], [4000, 3000], 6, 3, {"lam_none": True}),
    ([40, 700, 30, 1200], [2000, 2000, 1000, 2000], 4, 2, {"ld_pad": 3}),
    ([50, 60, 70], [4096, 2048, 1024], 2, 16, {}),
    ([100], [8192], 2, 1, {}),
    ([200, 150, 100, 120], [1500, 1500, 1500, 1500], 5, 2, {}),
])
def test_cp_shapes(fcs, ctx, orc, I, J, R, D, kw):
    _cp_case(fcs, ctx, orc, I, J, R, D, 21, **kw)


def test_cp_full_size_sampled_sketches(fcs, ctx, orc):
    """Order 3, I_n = 1000, R = 100, J_n = 5000 (Jt = 14998, P = 16384),
    D = 10, in the launch configuration the benchmark times; the oracle
    computes sketches d = 0 and d = 9 in full."""
    I, J, R, D = [1000] * 3, [5000] * 3, 100, 10
    U, lam = synth.cp_factors(2, I, R)
    hg, sg = fcs.fcs_make_hashes(ctx, 2, I, J, D)
    got = host(fcs.fcs_sketch_cp(ctx, [cuda(u) for u in U], cuda(lam), J, hg, sg))
    ho, so = orc.make_hashes(2, I, J, D)
    pick = [0, 9]
    ref = orc.fcs_cp([u.astype(np.float64) for u in U], lam.astype(np.float64), J,
                     ho[pick], so[pick])
    assert_sketch_close(got[pick], ref)


# ------------------------------------------------------------------ contractions
def _contract_setup(orc, I, J, D, B, seed, same=True):
    T = synth.gaussian(seed, I)
    ho, so = orc.make_hashes(seed + 1, I, J, D)
    fT = orc.fcs_dense(T.astype(np.float64), J, ho, so)
    if same:
        u = synth.unit_vectors(seed + 2, B, I[0])
        vecs = [u] * len(I)
    else:
        vecs = [synth.unit_vectors(seed + 2 + n, B, I[n]) for n in range(len(I))]
    return T, ho, so, fT, vecs


def _check_all(fcs, ctx, orc, I, J, ho, so, fT, vecs, fT_dev=None):
    D, B = fT.shape[0], vecs[0].shape[0]
    fTg = cuda(fT.astype(np.float32)) if fT_dev is None else fT_dev
    fT_in = fT.astype(np.float32).astype(np.float64) if fT_dev is None else fT
    med, raw = fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_ALL, fTg,
                                [cuda(v) for v in vecs], I, J, cuda(ho), cuda(so),
                                raw=True)
    med, raw = host(med), host(raw)
    ref = np.zeros((B, D))
    scale = np.zeros((B, D))
    for b in range(B):
        vb = [v[b].astype(np.float64) for v in vecs]
        ref[b] = orc.contract_all(fT_in, vb, J, ho, so)
        # ||FCS_d(v_1 o ... o v_N)|| via the oracle's rank-1 CP sketch
        r1 = orc.fcs_cp([x[:, None] for x in vb], None, J, ho, so)
        scale[b] = np.linalg.norm(fT_in, axis=1) * np.linalg.norm(r1, axis=1)
    err = np.abs(raw - ref) / scale
    assert err.max() <= CONTRACT_RTOL, f"T(v..v) error {err.max():.3e}"
    mref = orc.median(ref.T)
    merr = np.abs(med - mref) / scale.max(axis=1)
    assert merr.max() <= CONTRACT_RTOL, f"median error {merr.max():.3e}"


def _check_free(fcs, ctx, orc, I, J, ho, so, fT, vecs, m, fT_dev=None, rtol=CONTRACT_RTOL):
    D, B = fT.shape[0], vecs[0].shape[0]
    fTg = cuda(fT.astype(np.float32)) if fT_dev is None else fT_dev
    fT_in = fT.astype(np.float32).astype(np.float64) if fT_dev is None else fT
    vv = [cuda(v) if n != m else None for n, v in enumerate(vecs)]
    med, raw = fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_FREE, fTg, vv, I, J, cuda(ho),
                                cuda(so), free_mode=m, raw=True)
    med, raw = host(med), host(raw)
    refs = np.zeros((B, D, I[m]))
    for b in range(B):
        vb = [v[b].astype(np.float64) for v in vecs]
        refs[b] = orc.contract_free(fT_in, vb, m, J, ho, so)
        for d in range(D):
            e = rel_l2(raw[b, d], refs[b, d])
            assert e <= rtol, f"T(..I..) b={b} d={d}: {e:.3e}"
        mref = orc.median(refs[b])
        scale = np.linalg.norm(refs[b], axis=1).max()
        assert np.linalg.norm(med[b] - mref) <= rtol * scale


@pytest.mark.parametrize("D", [1, 3, 4])
def test_contract_small(fcs, ctx, orc, D):
    I, J = [20, 20, 20], [13, 11, 17]
    T, ho, so, fT, vecs = _contract_setup(orc, I, J, D, 3, 31)
    _check_all(fcs, ctx, orc, I, J, ho, so, fT, vecs)
    _check_free(fcs, ctx, orc, I, J, ho, so, fT, vecs, 0)


@pytest.mark.parametrize("m", [0, 1, 2])
def test_contract_als_modes(fcs, ctx, orc, m):
    """Distinct vectors per mode and every free mode (the ALS columns)."""
    I, J = [30, 25, 40], [37, 23, 51]
    T, ho, so, fT, vecs = _contract_setup(orc, I, J, 5, 4, 41, same=False)
    _check_all(fcs, ctx, orc, I, J, ho, so, fT, vecs)
    _check_free(fcs, ctx, orc, I, J, ho, so, fT, vecs, m)


def test_contract_order4_even_D(fcs, ctx, orc):
    I, J = [9, 8, 7, 6], [20, 30, 25, 15]
    T, ho, so, fT, vecs = _contract_setup(orc, I, J, 10, 2, 51, same=False)
    _check_all(fcs, ctx, orc, I, J, ho, so, fT, vecs)
    _check_free(fcs, ctx, orc, I, J, ho, so, fT, vecs, 3)


def test_contract_rtpm_step_reduced(fcs, ctx, orc):
    """The RTPM step at I = 100 with the full hash lengths (J_n = 2000,
    Jt = 5998, P = 8192), D = 5, 8 vectors; GPU dense -> GPU contract."""
    I, J, D, B = [100] * 3, [2000] * 3, 5, 8
    T, V, w = synth.rtpm_tensor(61, I=100, R=10, sigma=0.01)
    ho, so = orc.make_hashes(62, I, J, D)
    fT = orc.fcs_dense(T.astype(np.float64), J, ho, so)
    u = synth.unit_vectors(63, B, 100)
    fT_dev = fcs.fcs_sketch_dense(ctx, cuda(T), J, cuda(ho), cuda(so))
    assert_sketch_close(host(fT_dev), fT)
    # oracle-sketch input (isolates the contraction kernels)
    _check_all(fcs, ctx, orc, I, J, ho, so, fT, [u] * 3)
    _check_free(fcs, ctx, orc, I, J, ho, so, fT, [u] * 3, 0)
    # whole GPU chain against the whole oracle chain
    _check_all(fcs, ctx, orc, I, J, ho, so, fT, [u] * 3, fT_dev=fT_dev)
    _check_free(fcs, ctx, orc, I, J, ho, so, fT, [u] * 3, 0, fT_dev=fT_dev)


def test_rtpm_step_full_size(fcs, ctx, orc):
    """The robust-tensor-power-method step at full size: symmetric 500^3 FP32
    tensor (rank 10, weights 10..1, noise sigma 0.01), J_n = 2000 (Jt = 5998,
    P = 8192), D = 5; 64 unit vectors; T(u,u,u) and T(I,u,u) with the median.
    The oracle computes the sketch and every contraction itself."""
    I, J, D, B = [500] * 3, [2000] * 3, 5, 64
    T, V, w = synth.rtpm_tensor(3, I=500, R=10, sigma=0.01)
    hg, sg = fcs.fcs_make_hashes(ctx, 3, I, J, D)
    ho, so = orc.make_hashes(3, I, J, D)
    fT_dev = fcs.fcs_sketch_dense(ctx, cuda(T), J, hg, sg)
    fT = orc.fcs_dense(T, J, ho, so)
    assert_sketch_close(host(fT_dev), fT)
    del T
    u = synth.unit_vectors(4, B, 500)
    _check_all(fcs, ctx, orc, I, J, ho, so, fT, [u] * 3, fT_dev=fT_dev)
    _check_free(fcs, ctx, orc, I, J, ho, so, fT, [u] * 3, 0, fT_dev=fT_dev)


# ------------------------------------------------------------------ recovery
def _recover_case(fcs, ctx, orc, I, J, D, M, seed):
    Jt = sum(J) - len(J) + 1
    sk = synth.gaussian(seed, (D, Jt))
    ho, so = orc.make_hashes(seed + 1, I, J, D)
    idx = synth.sample_indices(seed + 2, M, I)
    out, raw = fcs.fcs_recover(ctx, cuda(sk), I, J, cuda(ho), cuda(so), cuda(idx),
                               raw=True)
    ref, rref = orc.recover(sk.astype(np.float64), I, J, ho, so, idx, return_raw=True)
    assert np.array_equal(host(raw).astype(np.float64), rref)   # exact gathers
    np.testing.assert_allclose(host(out), ref, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("I,J,D,M", [
    ([20, 20, 20], [8, 8, 8], 1, 8000),
    ([512, 512, 512, 512], [1024] * 4, 10, 1 << 20),
    ([7, 9], [3, 4], 16, 1001),
    ([100], [17], 2, 33),
    ([3, 4, 5, 6, 7], [2, 3, 2, 3, 2], 5, 0),
])
def test_recover(fcs, ctx, orc, I, J, D, M):
    if M == 0:
        sk = torch.zeros((D, sum(J) - len(J) + 1), device="cuda")
        ho, so = orc.make_hashes(1, I, J, D)
        out = fcs.fcs_recover(ctx, sk, I, J, cuda(ho), cuda(so),
                              torch.zeros((0, len(I)), dtype=torch.int32, device="cuda"))
        assert out.shape == (0,)
        return
    _recover_case(fcs, ctx, orc, I, J, D, M, 71)


def test_recover_tiny_all_entries_from_cp(fcs, ctx, orc):
    """Config-1 style: recover all 8000 entries of the 20^3 sketch."""
    U, lam = synth.cp_factors(0, [20] * 3, 5)
    ho, so = orc.make_hashes(1, [20] * 3, [8] * 3, 1)
    sk = orc.fcs_cp([u.astype(np.float64) for u in U], lam.astype(np.float64),
                    [8] * 3, ho, so).astype(np.float32)
    idx = np.stack(np.unravel_index(np.arange(8000), (20, 20, 20)), 1).astype(np.int32)
    got = host(fcs.fcs_recover(ctx, cuda(sk), [20] * 3, [8] * 3, cuda(ho), cuda(so),
                               cuda(idx)))
    ref = orc.recover(sk.astype(np.float64), [20] * 3, [8] * 3, ho, so, idx)
    np.testing.assert_array_equal(got.astype(np.float64), ref)


def test_recover_batched(fcs, ctx, orc):
    I, J, D, M, nb = [64, 64, 64, 64], [128] * 4, 10, 5000, 4
    Jt = sum(J) - 3
    sk = synth.gaussian(81, (nb, D, Jt))
    ho, so = orc.make_hashes(82, I, J, D)
    idx = np.stack([synth.sample_indices(83 + b, M, I) for b in range(nb)])
    got = host(fcs.fcs_recover(ctx, cuda(sk), I, J, cuda(ho), cuda(so), cuda(idx)))
    for b in range(nb):
        ref = orc.recover(sk[b].astype(np.float64), I, J, ho, so, idx[b])
        np.testing.assert_allclose(got[b], ref, rtol=1e-6, atol=1e-7)


# ------------------------------------------------------------------ outer
@pytest.mark.parametrize("nb,D,La,Lb", [(3, 10, 2047, 2047), (2, 3, 5, 1),
                                        (1, 2, 100, 37), (4, 1, 1, 1),
                                        (1, 4, 4000, 4000)])
def test_outer_combine(fcs, ctx, orc, nb, D, La, Lb):
    fa = synth.gaussian(91, (nb, D, La))
    fb = synth.gaussian(92, (nb, D, Lb))
    got = host(fcs.fcs_sketch_outer(ctx, cuda(fa), cuda(fb)))
    for b in range(nb):
        ref = orc.outer_combine(fa[b].astype(np.float64), fb[b].astype(np.float64))
        assert_sketch_close(got[b], ref)


@pytest.mark.parametrize("nb,D,La,Lb", [(8, 10, 2047, 2047), (2, 3, 5, 1), (1, 4, 4000, 4000),
                                        (2, 2, 30000, 20000)])
def test_outer_autotune_both_shapes(fcs, orc, nb, D, La, Lb):
    """fcs_outer_autotune times both block shapes: its output (the shape
    timed last, twice the threads where there are two) and a later
    fcs_sketch_outer of the same shape (the tuner's choice) both equal the
    oracle; the last case (P = 2^16) has only the two-pass route."""
    c = fcs.Context()
    fa = synth.gaussian(95, (nb, D, La))
    fb = synth.gaussian(96, (nb, D, Lb))
    nt, last = fcs.fcs_outer_autotune(c, cuda(fa), cuda(fb))
    P = 1 << max(4, (La + Lb - 2).bit_length())
    if P > 16384:
        assert nt == 0
    else:
        base = max(32, P // 32)
        assert nt in (base, 2 * base) if 2 * base <= 1024 else nt == base
    got = host(fcs.fcs_sketch_outer(c, cuda(fa), cuda(fb)))
    last = host(last)
    for b in range(nb):
        ref = orc.outer_combine(fa[b].astype(np.float64), fb[b].astype(np.float64))
        assert_sketch_close(last[b], ref, what=f"last timed shape, item {b}")
        assert_sketch_close(got[b], ref, what=f"tuned shape, item {b}")
    c.close()


def test_kronecker_chain_small(fcs, ctx, orc):
    """FCS(A o B) from GPU sketches of A (modes 1,2) and B (modes 3,4) equals
    the oracle's dense FCS of the materialised order-4 tensor."""
    A, B = synth.gaussian(93, (12, 10)), synth.gaussian(94, (8, 14))
    I, J, D = [12, 10, 8, 14], [9, 7, 11, 6], 4
    ho, so = orc.make_hashes(95, I, J, D)
    fa = fcs.fcs_sketch_dense(ctx, cuda(A), J[:2], cuda(ho[:, :22].copy()),
                              cuda(so[:, :22].copy()))
    fb = fcs.fcs_sketch_dense(ctx, cuda(B), J[2:], cuda(ho[:, 22:].copy()),
                              cuda(so[:, 22:].copy()))
    got = host(fcs.fcs_sketch_outer(ctx, fa, fb))
    ref = orc.fcs_dense(np.multiply.outer(A.astype(np.float64), B.astype(np.float64)),
                        J, ho, so)
    assert_sketch_close(got, ref)
    idx = synth.sample_indices(96, 500, I)
    rec = host(fcs.fcs_recover(ctx, cuda(got), I, J, cuda(ho), cuda(so), cuda(idx)))
    rref = orc.recover(got.astype(np.float64), I, J, ho, so, idx)
    np.testing.assert_allclose(rec, rref, rtol=1e-6, atol=1e-7)


# ------------------------------------------------------------------ errors
def test_argument_errors(fcs, ctx):
    h, s = fcs.fcs_make_hashes(ctx, 1, [10, 10], [5, 5], 2)
    with pytest.raises(fcs.FcsError) as e:
        fcs.fcs_make_hashes(ctx, 1, [10] * 9, [5] * 9, 1)
    assert e.value.code == fcs.FCS_EINVAL
    with pytest.raises(fcs.FcsError) as e:
        fcs.fcs_make_hashes(ctx, 1, [10, 10], [5, 5], 17)
    assert e.value.code == fcs.FCS_EINVAL
    with pytest.raises(fcs.FcsError) as e:
        fcs.fcs_make_hashes(ctx, 1, [10, 0], [5, 5], 1)
    assert e.value.code == fcs.FCS_EINVAL
    U = [torch.randn(10, 3, device="cuda") for _ in range(2)]
    with pytest.raises(fcs.FcsError) as e:        # Jt > 2^20
        fcs.fcs_sketch_cp(ctx, U, None, [600000, 600000], h, s)
    assert e.value.code == fcs.FCS_EUNSUPPORTED
    with pytest.raises(ValueError):          # the binding checks the table stride
        fcs.fcs_sketch_dense(ctx, torch.randn(10, 10, device="cuda"), [5, 5], h, s,
                             ldh=3)
    import ctypes as C                        # and so does the C entry point
    T = torch.randn(10, 10, device="cuda")
    out = torch.empty((2, 9), device="cuda")
    rc = fcs.lib().fcs_sketch_dense(ctx.handle, 2, fcs._arr(C.c_int64, [10, 10]), None,
                                    fcs._arr(C.c_int32, [5, 5]), 2, C.c_void_p(T.data_ptr()),
                                    C.c_void_p(h.data_ptr()), C.c_void_p(s.data_ptr()), 3,
                                    C.c_void_p(out.data_ptr()), 1, 0, 0)
    assert rc == fcs.FCS_EINVAL


def test_budget_zero_refuses_workspace(fcs):
    c = fcs.Context(budget=0)
    h, s = fcs.fcs_make_hashes(c, 1, [10, 10], [5, 5], 2)
    out = fcs.fcs_sketch_dense(c, torch.randn(10, 10, device="cuda"), [5, 5], h, s)
    assert out.shape == (2, 9)
    U = [torch.randn(10, 3, device="cuda") for _ in range(2)]
    with pytest.raises(fcs.FcsError) as e:
        fcs.fcs_sketch_cp(c, U, None, [5, 5], h, s)
    assert e.value.code == fcs.FCS_ENOMEM_BUDGET
    assert c.workspace_bytes() == 0
    c.close()
