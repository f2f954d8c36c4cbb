"""FP64 CPU oracle: the paper's algorithms built on the sketch primitives.

TEST INFRASTRUCTURE ONLY (same rules as the rest of ``oracle/``: only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it; it shares no code with the CUDA library).

Each function follows one passage of the paper step by step, in numpy, on top
of the oracle's C primitives (``fcs_dense``, ``fcs_cp``, ``contract_all``,
``contract_free``, ``outer_combine``, ``median``).  Random starting points
are inputs, never drawn here.
"""
from __future__ import annotations

import numpy as np

from . import contract_all, contract_free, fcs_cp, median, outer_combine


def outer_sum(fa, fb) -> np.ndarray:
    """Tensor contraction compression (subsection of that name): the sketch
    of A contracted with B over one mode is the sum over the L slices of the
    full linear convolutions of the slice sketches,
        FCS(A (x)_{3,1} B) = sum_l FCS(A(:,:,l)) (*) FCS(B(l,:,:)).
    fa [L][D][La], fb [L][D][Lb] -> [D][La+Lb-1]."""
    fa = np.asarray(fa, dtype=np.float64)
    fb = np.asarray(fb, dtype=np.float64)
    out = outer_combine(fa[0], fb[0])
    for l in range(1, fa.shape[0]):
        out = out + outer_combine(fa[l], fb[l])
    return out


def fold(fcs, J: int) -> np.ndarray:
    """Sum of the bins congruent modulo J (rows of a [.., Jt] array)."""
    fcs = np.asarray(fcs, dtype=np.float64)
    out = np.zeros(fcs.shape[:-1] + (J,))
    for k in range(fcs.shape[-1]):
        out[..., k % J] += fcs[..., k]
    return out


def sketch_inner(sa, sw, bias=None):
    """Tensor regression layer from sketches (eq. net_compress):
    raw[b][c][d] = <FCS_d(X_b), FCS_d(W_c)>, Y[b][c] = median_d raw + bias[c].
    sa [B][D][Jt], sw [C][D][Jt].  Returns (Y [B][C], raw [B][C][D])."""
    sa = np.asarray(sa, dtype=np.float64)
    sw = np.asarray(sw, dtype=np.float64)
    B, D, _ = sa.shape
    C = sw.shape[0]
    raw = np.einsum("bdj,cdj->bcd", sa, sw)
    y = median(np.moveaxis(raw, 2, 0).reshape(D, B * C)).reshape(B, C)
    if bias is not None:
        y = y + np.asarray(bias, dtype=np.float64)[None, :]
    return y, raw


def rtpm(fcsT, N: int, I: int, J, h, s, K: int, L: int, n_iter: int, init):
    """Sketched robust tensor power method for a symmetric order-N tensor
    (RTPM subsection): for each of K components, n_iter power iterations
        u <- T(I,u,..,u) / ||T(I,u,..,u)||
    from each of L starting vectors (rows of init[k], normalised first), the
    eigenvalue T(u,..,u), the start with the largest eigenvalue kept; then the
    sketch is deflated by the linearity of FCS,
        FCS(T) <- FCS(T) - lambda FCS(u o .. o u)   (eq. FCS_syn, R = 1).
    Contractions are eqs. T_Ivw (free mode 0) and T_uvw with the median over
    the D sketches.  Returns (lambda [K], U [K][I])."""
    S = np.array(fcsT, dtype=np.float64)
    lam_out = np.zeros(K)
    U_out = np.zeros((K, I))
    for k in range(K):
        V = np.array(init[k], dtype=np.float64)
        V /= np.linalg.norm(V, axis=1, keepdims=True)
        for _ in range(n_iter):
            W = np.stack([median(contract_free(S, [None] + [V[l]] * (N - 1), 0, J, h, s,
                                               I=[I] * N))
                          for l in range(L)])
            V = W / np.linalg.norm(W, axis=1, keepdims=True)
        lam = np.array([median(contract_all(S, [V[l]] * N, J, h, s)[:, None])[0]
                        for l in range(L)])
        best = int(np.argmax(lam))
        lam_out[k] = lam[best]
        U_out[k] = V[best]
        S = S - fcs_cp([U_out[k][:, None]] * N, np.array([lam_out[k]]), J, h, s)
    return lam_out, U_out


def als(fcsT, I, J, h, s, R: int, n_iter: int, init):
    """Sketched CP-ALS (ALS subsection) for an order-N tensor: in each sweep,
    for each mode m, the columns T_(m)(..) = [T(.., I (mode m), ..)]_r with the
    r-th columns of the other factors (eq. T_Ivw, median over D), then the
    least-squares update with the Hadamard product of the other factors'
    Gram matrices,  F_m^T <- G^{-1} M^T,  G = *_{n != m} F_n F_n^T,
    and column normalisation (weights lambda).  Factors are held transposed,
    F_n [R][I_n]; init gives their starting values.  The solve is a
    Cholesky factorisation of G.  Returns (F list, lambda [R])."""
    N = len(I)
    F = [np.array(x, dtype=np.float64) for x in init]
    lam = np.ones(R)
    for _ in range(n_iter):
        for m in range(N):
            Mt = np.stack([median(contract_free(fcsT, [None if n == m else F[n][r]
                                                       for n in range(N)], m, J, h, s,
                                                I=I))
                           for r in range(R)])
            G = np.ones((R, R))
            for n in range(N):
                if n != m:
                    G *= F[n] @ F[n].T
            Lc = np.linalg.cholesky(G)
            X = np.linalg.solve(Lc.T, np.linalg.solve(Lc, Mt))
            lam = np.linalg.norm(X, axis=1)
            F[m] = X / lam[:, None]
    return F, lam
