"""Pins for the oracle's Tensor Sketch, tensor-contraction compression, TRL,
RTPM and ALS routines (CPU only), each against something other than itself:
the Def. 2 loop against FCS folded mod J, Prop. 1's variance ordering, the
sketch of a materialised contraction, exact special cases, unbiasedness, and
recovery of known decompositions."""
from __future__ import annotations

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def alg(orc):
    from oracle import algorithms
    return algorithms


def test_ts_is_fcs_folded(orc, alg):
    """Def. 2 (bins (sum h) mod J) equals the Def. 4 sketch with its bins
    summed mod J (the circular convolution of eq. TS is the linear one of
    eq. FCS_syn folded), for several orders."""
    for N, I, J in [(3, [5, 6, 7], 9), (2, [11, 4], 5), (4, [3, 4, 3, 5], 7)]:
        h, s = orc.make_hashes(3 + N, I, [J] * N, 3)
        T = synth.gaussian(N, I)
        ts = orc.ts_dense(T, J, h, s)
        np.testing.assert_allclose(ts, alg.fold(orc.fcs_dense(T, [J] * N, h, s), J),
                                   rtol=1e-12, atol=1e-12)


def test_ts_order1_is_count_sketch(orc):
    I, J = [40], 13
    h, s = orc.make_hashes(9, I, [J], 2)
    x = synth.gaussian(4, I)
    for d in range(2):
        np.testing.assert_allclose(orc.ts_dense(x, J, h, s)[d],
                                   orc.count_sketch(x, h[d], s[d], J), atol=1e-12)


def test_prop1_fcs_variance_below_ts(orc, alg):
    """Prop. 1: with the same hash functions, <FCS M, FCS N> and <TS M, TS N>
    are both unbiased for <M, N> and the FCS estimate has the smaller
    variance.  3000 hash draws; the observed ratio is about 1.7."""
    I, J = [6, 7, 8], 10
    g = np.random.default_rng(0)
    Mt = g.standard_normal(I)
    Nt = Mt + 0.5 * g.standard_normal(I)
    exact = float((Mt * Nt).sum())
    S = 3000
    ef, et = np.zeros(S), np.zeros(S)
    for k in range(S):
        h, s = orc.make_hashes(1000 + k, I, [J] * 3, 1)
        fm, fn = orc.fcs_dense(Mt, [J] * 3, h, s)[0], orc.fcs_dense(Nt, [J] * 3, h, s)[0]
        ef[k] = fm @ fn
        et[k] = alg.fold(fm, J) @ alg.fold(fn, J)
    for e in (ef, et):
        assert abs(e.mean() - exact) <= 4 * e.std() / np.sqrt(S)
    assert et.var() >= 1.3 * ef.var()


def test_outer_sum_is_sketch_of_contraction(orc, alg):
    """Tensor-contraction compression: the sum over l of the convolved slice
    sketches equals the dense FCS (modes 1-4) of A contracted with B."""
    I1, I2, L, I3, I4 = 5, 6, 4, 3, 7
    g = np.random.default_rng(5)
    A = g.uniform(0, 10, (I1, I2, L))
    B = g.uniform(0, 10, (L, I3, I4))
    Cten = np.einsum("abl,lcd->abcd", A, B)
    J = [9, 8, 7, 10]
    h, s = orc.make_hashes(17, [I1, I2, I3, I4], J, 3)
    off = I1 + I2
    fa = np.stack([orc.fcs_dense(A[:, :, l], J[:2], h[:, :off], s[:, :off]) for l in range(L)])
    fb = np.stack([orc.fcs_dense(B[l], J[2:], h[:, off:], s[:, off:]) for l in range(L)])
    np.testing.assert_allclose(alg.outer_sum(fa, fb), orc.fcs_dense(Cten, J, h, s),
                               rtol=1e-11, atol=1e-9)


def test_sketch_inner_identity_hashes_exact(orc, alg):
    """Order 1 with identity hashes (h(i) = i, s = +1, J = I): the sketches
    are the vectors themselves, so the TRL products are exact."""
    Bn, C, I = 4, 3, 12
    g = np.random.default_rng(6)
    X, W, b = g.standard_normal((Bn, I)), g.standard_normal((C, I)), g.standard_normal(C)
    D = 3
    y, raw = alg.sketch_inner(np.repeat(X[:, None, :], D, 1), np.repeat(W[:, None, :], D, 1), b)
    np.testing.assert_allclose(y, X @ W.T + b[None, :], rtol=1e-12)


def test_sketch_inner_unbiased(orc, alg):
    I, J = [4, 5, 3], [6, 6, 6]
    g = np.random.default_rng(7)
    X, W = g.standard_normal([2] + I), g.standard_normal([2] + I)
    exact = np.einsum("bijk,cijk->bc", X, W)
    S = 2000
    est = np.zeros((S, 2, 2))
    for k in range(S):
        h, s = orc.make_hashes(5000 + k, I, J, 1)
        sa = np.stack([orc.fcs_dense(X[b], J, h, s) for b in range(2)])
        sw = np.stack([orc.fcs_dense(W[c], J, h, s) for c in range(2)])
        est[k] = alg.sketch_inner(sa, sw)[0]
    se = est.std(axis=0) / np.sqrt(S)
    assert np.all(np.abs(est.mean(axis=0) - exact) <= 4 * se)


def _odeco(seed, I, lams):
    V = synth.orthonormal_columns(seed, I, len(lams))
    T = np.einsum("r,ir,jr,kr->ijk", np.asarray(lams, float), V, V, V)
    return T, V


def test_rtpm_recovers_orthogonal_decomposition(orc, alg):
    """A noiseless symmetric orthogonally decomposable tensor: the sketched
    RTPM (long sketches, D = 3) finds the weights 5, 4, 3 and their vectors."""
    I, lams = 12, [5.0, 4.0, 3.0]
    T, V = _odeco(3, I, lams)
    J = [3000] * 3
    h, s = orc.make_hashes(21, [I] * 3, J, 3)
    fT = orc.fcs_dense(T, J, h, s)
    K, L, it = 3, 6, 12
    init = np.random.default_rng(8).standard_normal((K, L, I))
    lam, U = alg.rtpm(fT, 3, I, J, h, s, K, L, it, init)
    np.testing.assert_allclose(np.sort(lam)[::-1], lams, rtol=0.03)
    for k in range(K):
        r = int(np.argmin(np.abs(np.asarray(lams) - lam[k])))
        assert abs(float(U[k] @ V[:, r])) >= 0.99


def test_als_recovers_cp_tensor(orc, alg):
    """A noiseless asymmetric rank-3 tensor: sketched ALS (long sketches)
    reaches a small relative residual and the right weights."""
    I, R = [10, 12, 9], 3
    U, lam = synth.cp_factors(31, I, R)
    T = synth.cp_dense(U, lam).astype(np.float64)
    J = [3000] * 3
    h, s = orc.make_hashes(32, I, J, 3)
    fT = orc.fcs_dense(T, J, h, s)
    g = np.random.default_rng(9)
    init = [u.T + 0.3 * g.standard_normal((R, i)) for u, i in zip(U, I)]
    F, w = alg.als(fT, I, J, h, s, R, 12, init)
    That = np.einsum("r,ri,rj,rk->ijk", w, F[0], F[1], F[2])
    assert np.linalg.norm(That - T) / np.linalg.norm(T) <= 0.05
