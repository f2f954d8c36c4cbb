"""Pins for the FP64 oracle: each routine is checked against something other
than itself -- closed forms, published values, library routines (numpy's
convolve / FFT / bincount / einsum / median), invariants of the method, or
brute force on tiny inputs.  Chosen so that a dropped term, a wrong sign or
index, or a transposed operand in the oracle fails at least one of them.

CPU only (no GPU marker)."""
from __future__ import annotations

import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
P61 = (1 << 61) - 1


def _mode_tables(h, s, I, d=0):
    """Split one sketch's [sum I] tables into per-mode arrays."""
    out_h, out_s, off = [], [], 0
    for i in I:
        out_h.append(h[d, off:off + i].astype(np.int64))
        out_s.append(s[d, off:off + i].astype(np.int64))
        off += i
    return out_h, out_s


def _outer(vs):
    t = np.asarray(vs[0], dtype=np.float64)
    for v in vs[1:]:
        t = np.multiply.outer(t, np.asarray(v, dtype=np.float64))
    return t


# --------------------------------------------------------------------- hashes
def test_splitmix64_published_values(orc):
    vals = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    assert [orc.splitmix64(0, k) for k in range(len(vals))] == vals


def test_carter_wegman_against_bigint(orc):
    """h, s must equal the multiply-mod-prime family evaluated with Python's
    exact integers from the oracle's own coefficients."""
    I, J, D, seed = [37, 1000, 5], [7, 5000, 2], 3, 12345
    h, s = orc.make_hashes(seed, I, J, D)
    coef = orc.hash_coeffs(seed, len(I), D)
    for d in range(D):
        off = 0
        for n, (In, Jn) in enumerate(zip(I, J)):
            ah, bh, as_, bs = (int(c) for c in coef[d, n])
            assert 1 <= ah < P61 and 0 <= bh < P61 and 1 <= as_ < P61
            for i in range(In):
                assert h[d, off + i] == ((ah * i + bh) % P61) % Jn
                assert s[d, off + i] == 1 - 2 * (((as_ * i + bs) % P61) & 1)
            off += In


def test_coefficients_follow_draw_order(orc):
    """Four SplitMix64 draws per (d, n) in the order d-major, n-minor."""
    seed, N, D = 99, 3, 2
    coef = orc.hash_coeffs(seed, N, D)
    k = 0
    for d in range(D):
        for n in range(N):
            x = [orc.splitmix64(seed, k + j) for j in range(4)]
            assert int(coef[d, n, 0]) == 1 + x[0] % (P61 - 1)
            assert int(coef[d, n, 1]) == x[1] % P61
            assert int(coef[d, n, 2]) == 1 + x[2] % (P61 - 1)
            assert int(coef[d, n, 3]) == x[3] % P61
            k += 4


def test_hash_range_and_determinism(orc):
    I, J = [300, 200, 100], [17, 1, 64]
    h1, s1 = orc.make_hashes(7, I, J, 4)
    h2, s2 = orc.make_hashes(7, I, J, 4)
    assert np.array_equal(h1, h2) and np.array_equal(s1, s2)
    hm, sm = _mode_tables(h1, s1, I, 2)
    for n in range(3):
        assert hm[n].min() >= 0 and hm[n].max() < J[n]
        assert set(np.unique(sm[n])) <= {-1, 1}
    h3, _ = orc.make_hashes(8, I, J, 4)
    assert not np.array_equal(h1, h3)


def test_hash_pairwise_statistics(orc):
    """2-wise independence (Def. 1): over seeds, P[h(i)=h(j)] ~ 1/J and
    E[s(i)s(j)] ~ 0 for a fixed pair i != j."""
    J, trials = 16, 4000
    coll = 0
    sprod = 0
    for seed in range(trials):
        h, s = orc.make_hashes(seed, [64], [J], 1)
        coll += int(h[0, 3] == h[0, 41])
        sprod += int(s[0, 3]) * int(s[0, 41])
    p = coll / trials
    assert abs(p - 1 / J) < 4 * np.sqrt((1 / J) * (1 - 1 / J) / trials)
    assert abs(sprod / trials) < 4 / np.sqrt(trials)


def test_hash_uniformity_chi2(orc):
    J, I = 64, 64000
    h, s = orc.make_hashes(2024, [I], [J], 1)
    counts = np.bincount(h[0], minlength=J)
    chi2 = float(((counts - I / J) ** 2 / (I / J)).sum())
    assert chi2 < 63 + 6 * np.sqrt(2 * 63)        # mean 63, sd ~11
    assert abs(int(s[0].astype(np.int64).sum())) < 5 * np.sqrt(I)


# ------------------------------------------------------------ count sketch
def test_count_sketch_vs_bincount(orc):
    g = np.random.default_rng(0)
    x = g.standard_normal(500)
    h = g.integers(0, 37, 500).astype(np.int32)
    s = (1 - 2 * g.integers(0, 2, 500)).astype(np.int8)
    ref = np.bincount(h, weights=s * x, minlength=37)
    np.testing.assert_allclose(orc.count_sketch(x, h, s, 37), ref, rtol=1e-13,
                               atol=1e-13)


def test_linear_convolve_vs_numpy(orc):
    g = np.random.default_rng(1)
    for la, lb in [(1, 1), (1, 9), (13, 5), (64, 200)]:
        a, b = g.standard_normal(la), g.standard_normal(lb)
        np.testing.assert_allclose(orc.linear_convolve(a, b), np.convolve(a, b),
                                   rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------ dense FCS
def test_identity_hashes_give_linear_convolution(orc):
    """Proof of eq. FCS_syn: with h_n(i)=i, s_n=+1, J_n=I_n the FCS of a o b o c
    is the full linear convolution a * b * c."""
    g = np.random.default_rng(2)
    I = [5, 7, 3]
    vs = [g.standard_normal(i) for i in I]
    h, s = synth.ones_hashes(I)
    got = orc.fcs_dense(_outer(vs), I, h, s)[0]
    ref = np.convolve(np.convolve(vs[0], vs[1]), vs[2])
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_identity_hashes_polynomial_power_closed_form(orc):
    for line in open(os.path.join(GOLDEN, "poly_power.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        lhs, rhs = line.split(":")
        m, N = (int(t) for t in lhs.split())
        coeffs = [float(t) for t in rhs.split()]
        I = [m] * N
        h, s = synth.ones_hashes(I)
        got = orc.fcs_dense(np.ones(I), I, h, s)[0]
        np.testing.assert_array_equal(got, coeffs)


def test_order_one_is_count_sketch(orc):
    """N = 1: FCS reduces to the plain Count Sketch of Def. 1."""
    x = np.random.default_rng(3).standard_normal(400)
    h, s = orc.make_hashes(5, [400], [33], 2)
    got = orc.fcs_dense(x, [33], h, s)
    for d in range(2):
        ref = np.bincount(h[d], weights=s[d] * x, minlength=33)
        np.testing.assert_allclose(got[d], ref, rtol=1e-12, atol=1e-12)


def test_unit_hash_lengths_give_signed_total(orc):
    """J_n = 1 for all n: Jt = 1 and FCS = sum_i S(i) T(i)."""
    T = np.random.default_rng(4).standard_normal((6, 5, 4))
    h, s = orc.make_hashes(6, T.shape, [1, 1, 1], 3)
    got = orc.fcs_dense(T, [1, 1, 1], h, s)
    for d in range(3):
        _, sm = _mode_tables(h, s, T.shape, d)
        ref = np.einsum("ijk,i,j,k->", T, *sm)
        assert got[d].shape == (1,)
        np.testing.assert_allclose(got[d, 0], ref, rtol=1e-12)


def test_long_hash_definition(orc):
    """Def. 4: the long pair over column-major vec(T) (i_1 fastest)."""
    I, J = [4, 3, 5], [6, 2, 7]
    h, s = orc.make_hashes(11, I, J, 1)
    hm, sm = _mode_tables(h, s, I)
    H, S = orc.long_hash(I, h[0], s[0])
    for l in range(int(np.prod(I))):
        idx = np.unravel_index(l, I, order="F")
        assert H[l] == sum(hm[n][idx[n]] for n in range(3))
        assert S[l] == np.prod([sm[n][idx[n]] for n in range(3)])


def test_fcs_equals_count_sketch_under_long_hash(orc):
    """Def. 4 / eq. FCS: FCS(T) = CS(vec(T); h_{N+1}, s_{N+1})."""
    T = np.random.default_rng(12).standard_normal((4, 6, 5))
    J = [3, 8, 4]
    h, s = orc.make_hashes(13, T.shape, J, 2)
    dense = orc.fcs_dense(T, J, h, s)
    vecT = T.flatten(order="F")
    for d in range(2):
        H, S = orc.long_hash(T.shape, h[d], s[d])
        ref = np.bincount(H, weights=S * vecT, minlength=orc.jtilde(J))
        np.testing.assert_allclose(dense[d], ref, rtol=1e-12, atol=1e-12)


def test_layout_and_mode_order_invariance(orc):
    """FCS depends on entries and hashes only: Fortran layout and a mode
    permutation (with the hash tables permuted alike) give the same sketch."""
    T = np.random.default_rng(14).standard_normal((5, 4, 6))
    I, J = list(T.shape), [9, 3, 5]
    h, s = orc.make_hashes(15, I, J, 2)
    ref = orc.fcs_dense(T, J, h, s)
    np.testing.assert_allclose(orc.fcs_dense(np.asfortranarray(T), J, h, s), ref,
                               rtol=1e-12, atol=1e-12)
    perm = [2, 0, 1]
    offs = np.cumsum([0] + I)
    hp = np.concatenate([h[:, offs[p]:offs[p + 1]] for p in perm], axis=1)
    sp = np.concatenate([s[:, offs[p]:offs[p + 1]] for p in perm], axis=1)
    got = orc.fcs_dense(T.transpose(perm), [J[p] for p in perm], hp, sp)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_linearity(orc):
    g = np.random.default_rng(16)
    A, B = g.standard_normal((2, 6, 5, 4))
    J = [5, 5, 5]
    h, s = orc.make_hashes(17, A.shape, J, 2)
    lhs = orc.fcs_dense(2.5 * A - 0.75 * B, J, h, s)
    rhs = 2.5 * orc.fcs_dense(A, J, h, s) - 0.75 * orc.fcs_dense(B, J, h, s)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def test_one_sparse_tensor(orc):
    """One nonzero v at i: the sketch is S(i) v at bin H(i), zero elsewhere;
    recovery of that entry is exact."""
    I, J = [7, 8, 9], [4, 6, 5]
    h, s = orc.make_hashes(18, I, J, 3)
    T = np.zeros(I)
    i = (3, 5, 2)
    T[i] = 1.75
    sk = orc.fcs_dense(T, J, h, s)
    for d in range(3):
        hm, sm = _mode_tables(h, s, I, d)
        b = sum(hm[n][i[n]] for n in range(3))
        sg = np.prod([sm[n][i[n]] for n in range(3)])
        expect = np.zeros(orc.jtilde(J))
        expect[b] = sg * 1.75
        np.testing.assert_array_equal(sk[d], expect)
    rec = orc.recover(sk, I, J, h, s, np.array([i], dtype=np.int32))
    assert rec[0] == 1.75


def test_inner_product_unbiased(orc):
    """Prop. 1: <FCS(M), FCS(N)> is an unbiased estimate of <M, N>."""
    g = np.random.default_rng(19)
    M, N = g.standard_normal((2, 4, 5, 3))
    J = [4, 4, 4]
    trials = 3000
    est = np.empty(trials)
    for t in range(trials):
        h, s = orc.make_hashes(1000 + t, M.shape, J, 1)
        est[t] = orc.fcs_dense(M, J, h, s)[0] @ orc.fcs_dense(N, J, h, s)[0]
    truth = float((M * N).sum())
    se = est.std() / np.sqrt(trials)
    assert abs(est.mean() - truth) < 4 * se


def test_error_shrinks_with_hash_length(orc):
    """Cor. 1: the estimation error scales like 1/J."""
    g = np.random.default_rng(20)
    M = g.standard_normal((6, 6, 6))
    var = []
    for Jn in (3, 24):
        J = [Jn] * 3
        e = []
        for t in range(600):
            h, s = orc.make_hashes(5000 + t, M.shape, J, 1)
            f = orc.fcs_dense(M, J, h, s)[0]
            e.append(f @ f)
        var.append(np.var(e))
    assert var[1] < 0.5 * var[0]


# ------------------------------------------------------------ CP route
def test_cp_to_dense_vs_einsum(orc):
    U, lam = synth.cp_factors(21, [4, 5, 3], 3)
    ref = np.einsum("ar,br,cr,r->abc", *[u.astype(np.float64) for u in U],
                    lam.astype(np.float64))
    np.testing.assert_allclose(orc.cp_to_dense(U, lam), ref, rtol=1e-12)


@pytest.mark.parametrize("I,J,R,D", [([20, 20, 20], [8, 8, 8], 5, 2),
                                     ([6, 9, 4, 5], [5, 3, 7, 2], 3, 2),
                                     ([11], [6], 4, 1),
                                     ([7, 5], [1, 9], 2, 3)])
def test_cp_route_equals_dense_route(orc, I, J, R, D):
    """Eq. FCS_syn vs eq. FCS_asyn on the materialised CP tensor."""
    U, lam = synth.cp_factors(22, I, R)
    h, s = orc.make_hashes(23, I, J, D)
    cp = orc.fcs_cp(U, lam, J, h, s)
    dense = orc.fcs_dense(orc.cp_to_dense(U, lam), J, h, s)
    np.testing.assert_allclose(cp, dense, rtol=1e-11, atol=1e-11)


def test_cp_route_fft_form(orc):
    """Eq. FCS_syn third line with numpy's FFT: the zero-padded transform of
    any length >= Jt (here Jt itself and the next power of two) reproduces the
    direct convolution; the rank sum may sit inside or outside the IFFT."""
    I, J, R = [30, 25, 40], [16, 9, 21], 6
    U, lam = synth.cp_factors(24, I, R)
    h, s = orc.make_hashes(25, I, J, 2)
    cp = orc.fcs_cp(U, lam, J, h, s)
    Jt = orc.jtilde(J)
    for d in range(2):
        hm, sm = _mode_tables(h, s, I, d)
        for P in (Jt, 1 << (Jt - 1).bit_length()):
            acc = np.zeros(P)
            for r in range(R):
                prod = np.ones(P // 2 + 1, dtype=complex)
                for n in range(3):
                    cs = np.bincount(hm[n], weights=sm[n] * U[n][:, r].astype(float),
                                     minlength=J[n])
                    prod = prod * np.fft.rfft(cs, P)
                acc += lam[r] * np.fft.irfft(prod, P)
            np.testing.assert_allclose(acc[:Jt], cp[d], rtol=1e-9, atol=1e-9)


# ------------------------------------------------------------ contractions
def test_contract_all_definition_and_parseval(orc):
    """Eq. T_uvw: <FCS(T), FCS(u o v o w)> by materialising the rank-1 tensor,
    and by the FFT (Parseval) form of its second line."""
    g = np.random.default_rng(26)
    I, J = [9, 7, 8], [6, 5, 7]
    T = g.standard_normal(I)
    vs = [g.standard_normal(i) for i in I]
    h, s = orc.make_hashes(27, I, J, 3)
    fT = orc.fcs_dense(T, J, h, s)
    got = orc.contract_all(fT, vs, J, h, s)
    ref = np.einsum("dj,dj->d", fT, orc.fcs_dense(_outer(vs), J, h, s))
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-12)
    Jt = orc.jtilde(J)
    P = 1 << (Jt - 1).bit_length()
    for d in range(3):
        hm, sm = _mode_tables(h, s, I, d)
        F = np.ones(P, dtype=complex)
        for n in range(3):
            F = F * np.fft.fft(np.bincount(hm[n], weights=sm[n] * vs[n],
                                           minlength=J[n]), P)
        par = np.real(np.vdot(np.fft.fft(fT[d], P), F)) / P
        np.testing.assert_allclose(got[d], par, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("m", [0, 1, 2])
def test_contract_free_definition(orc, m):
    """Eq. T_Ivw first line (m = 0) and the ALS columns (m = 1, 2):
    <FCS(T), FCS(.. e_i ..)> with the rank-1 tensor materialised."""
    g = np.random.default_rng(28 + m)
    I, J = [6, 8, 7], [5, 6, 4]
    T = g.standard_normal(I)
    vs = [g.standard_normal(i) for i in I]
    h, s = orc.make_hashes(31, I, J, 2)
    fT = orc.fcs_dense(T, J, h, s)
    got = orc.contract_free(fT, vs, m, J, h, s)
    for i in range(I[m]):
        e = np.zeros(I[m])
        e[i] = 1.0
        ws = list(vs)
        ws[m] = e
        ref = np.einsum("dj,dj->d", fT, orc.fcs_dense(_outer(ws), J, h, s))
        np.testing.assert_allclose(got[:, i], ref, rtol=1e-11, atol=1e-12)


def test_contract_free_correlation_form(orc):
    """Eq. T_Ivw second line with numpy's FFT: z = IFFT(F(FCS T) conj F(CS_2 u)
    conj F(CS_3 u)), est_i = s_1(i) z(h_1(i)), for a power-of-two length."""
    g = np.random.default_rng(32)
    I, J = [20, 20, 20], [13, 11, 17]
    T = g.standard_normal(I)
    u = g.standard_normal(20)
    h, s = orc.make_hashes(33, I, J, 2)
    fT = orc.fcs_dense(T, J, h, s)
    got = orc.contract_free(fT, [u, u, u], 0, J, h, s)
    P = 1 << (orc.jtilde(J) - 1).bit_length()
    for d in range(2):
        hm, sm = _mode_tables(h, s, I, d)
        F = np.fft.fft(fT[d], P)
        for n in (1, 2):
            F = F * np.conj(np.fft.fft(np.bincount(hm[n], weights=sm[n] * u,
                                                   minlength=J[n]), P))
        z = np.real(np.fft.ifft(F))
        np.testing.assert_allclose(got[d], sm[0] * z[hm[0]], rtol=1e-9,
                                   atol=1e-11)


def test_contraction_estimates_unbiased(orc):
    """Cor. 1 premise: over hash draws the sketched T(u,u,u) and T(I,u,u)
    average to the exact contractions."""
    g = np.random.default_rng(34)
    I, J = [5, 5, 5], [4, 4, 4]
    T = g.standard_normal(I)
    u = g.standard_normal(5)
    trials = 3000
    e_all = np.empty(trials)
    e_free = np.empty((trials, 5))
    for t in range(trials):
        h, s = orc.make_hashes(9000 + t, I, J, 1)
        fT = orc.fcs_dense(T, J, h, s)
        e_all[t] = orc.contract_all(fT, [u, u, u], J, h, s)[0]
        e_free[t] = orc.contract_free(fT, [u, u, u], 0, J, h, s)[0]
    exact_all = np.einsum("ijk,i,j,k->", T, u, u, u)
    exact_free = np.einsum("ijk,j,k->i", T, u, u)
    assert abs(e_all.mean() - exact_all) < 4 * e_all.std() / np.sqrt(trials)
    se = e_free.std(axis=0) / np.sqrt(trials)
    assert np.all(np.abs(e_free.mean(axis=0) - exact_free) < 4 * se)


# ------------------------------------------------------------ median
@pytest.mark.parametrize("D", [1, 2, 3, 4, 5, 10])
def test_median_vs_numpy(orc, D):
    vals = np.random.default_rng(40 + D).standard_normal((D, 33))
    np.testing.assert_array_equal(orc.median(vals), np.median(vals, axis=0))


# ------------------------------------------------------------ recovery
def test_recover_matches_gather(orc):
    I, J = [6, 7, 8, 5], [4, 5, 3, 6]
    g = np.random.default_rng(41)
    sk = g.standard_normal((3, orc.jtilde(J)))
    h, s = orc.make_hashes(42, I, J, 3)
    idx = synth.sample_indices(43, 50, I)
    out, raw = orc.recover(sk, I, J, h, s, idx, return_raw=True)
    for d in range(3):
        hm, sm = _mode_tables(h, s, I, d)
        b = sum(hm[n][idx[:, n]] for n in range(4))
        sg = np.prod([sm[n][idx[:, n]] for n in range(4)], axis=0)
        np.testing.assert_array_equal(raw[d], sg * sk[d, b])
    np.testing.assert_array_equal(out, np.median(raw, axis=0))


def test_recover_unbiased(orc):
    """Each recovered entry averages to the true entry over hash draws."""
    g = np.random.default_rng(44)
    I, J = [4, 5, 6], [5, 5, 5]
    T = g.standard_normal(I)
    idx = synth.sample_indices(45, 6, I)
    trials = 3000
    est = np.empty((trials, 6))
    for t in range(trials):
        h, s = orc.make_hashes(20000 + t, I, J, 1)
        _, raw = orc.recover(orc.fcs_dense(T, J, h, s), I, J, h, s, idx,
                             return_raw=True)
        est[t] = raw[0]
    truth = T[tuple(idx.T)]
    se = est.std(axis=0) / np.sqrt(trials)
    assert np.all(np.abs(est.mean(axis=0) - truth) < 4 * se)


# ------------------------------------------------------------ Kronecker
def test_outer_combine_is_sketch_of_outer_product(orc):
    """Kronecker compression: conv(FCS(A; h1,h2), FCS(B; h3,h4)) equals the
    FCS of the order-4 tensor A o B under (h1..h4)."""
    g = np.random.default_rng(46)
    A, B = g.standard_normal((5, 4)), g.standard_normal((3, 6))
    I, J = [5, 4, 3, 6], [7, 4, 6, 5]
    h, s = orc.make_hashes(47, I, J, 2)
    fa = orc.fcs_dense(A, J[:2], h[:, :9], s[:, :9])
    fb = orc.fcs_dense(B, J[2:], h[:, 9:], s[:, 9:])
    got = orc.outer_combine(fa, fb)
    ref = orc.fcs_dense(np.multiply.outer(A, B), J, h, s)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
    for d in range(2):
        np.testing.assert_allclose(got[d], np.convolve(fa[d], fb[d]), rtol=1e-12,
                                   atol=1e-12)
