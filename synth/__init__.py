"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds input construction only -- none of the sketching arithmetic.
Both the FP64 oracle and the CUDA library consume what it returns.  Every draw
is made in FP64 from ``numpy.random.default_rng(seed)`` and rounded to FP32, so
both sides see identical FP32 values.

Workload shapes follow the paper's experiments (its CPD, Kronecker-compression
and tensor-regression sections); the paper's datasets are not available, so
these seeded tensors stand in for them.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def cp_factors(seed: int, I, R: int, lam_lo: float = 0.5, lam_hi: float = 1.5):
    """Factor matrices U_n (I_n x R, row-major, N(0,1)) and weights
    lambda ~ U(lam_lo, lam_hi), all rounded to FP32."""
    g = _rng(seed)
    U = [g.standard_normal((int(i), R)).astype(np.float32) for i in I]
    lam = g.uniform(lam_lo, lam_hi, size=R).astype(np.float32)
    return U, lam


def cp_dense(U, lam) -> np.ndarray:
    """Dense FP32 tensor of a CP model (input construction for the dense
    route): sum_r lam_r u_r^(1) o ... o u_r^(N), evaluated in FP64."""
    N = len(U)
    letters = "abcdefgh"[:N]
    spec = ",".join(f"{c}r" for c in letters) + ",r->" + letters
    T = np.einsum(spec, *[u.astype(np.float64) for u in U],
                  lam.astype(np.float64), optimize=True)
    return T.astype(np.float32)


def orthonormal_columns(seed: int, I: int, R: int) -> np.ndarray:
    """Random orthonormal I x R basis (QR of an N(0,1) matrix), FP64."""
    g = _rng(seed)
    q, r = np.linalg.qr(g.standard_normal((I, R)))
    return q * np.sign(np.diag(r))[None, :]


def rtpm_tensor(seed: int, I: int = 500, R: int = 10, sigma: float = 0.01):
    """Symmetric order-3 tensor sum_r w_r v_r o v_r o v_r + N(0, sigma^2)
    noise, weights R, R-1, ..., 1 (the robust tensor power method workload).
    Returns (T FP32 [I,I,I], V FP64 [I,R], w FP64 [R])."""
    V = orthonormal_columns(seed, I, R)
    w = np.arange(R, 0, -1, dtype=np.float64)
    g = _rng(seed + 1)
    T = np.empty((I, I, I), dtype=np.float32)
    for a in range(I):                       # slab by slab: bounded memory
        slab = np.einsum("r,jr,kr->jk", w * V[a], V, V, optimize=True)
        slab += sigma * g.standard_normal((I, I))
        T[a] = slab.astype(np.float32)
    return T, V, w


def unit_vectors(seed: int, B: int, I: int) -> np.ndarray:
    """B random unit vectors (normalised N(0,1)), FP32 [B, I]."""
    g = _rng(seed)
    u = g.standard_normal((B, I))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    return u.astype(np.float32)


def gaussian(seed: int, shape) -> np.ndarray:
    """N(0,1) FP32 array."""
    return _rng(seed).standard_normal(shape).astype(np.float32)


def uniform(seed: int, shape, lo: float, hi: float) -> np.ndarray:
    """U(lo, hi) FP32 array."""
    return _rng(seed).uniform(lo, hi, size=shape).astype(np.float32)


def sample_indices(seed: int, M: int, dims) -> np.ndarray:
    """M uniformly sampled multi-indices into a tensor of shape `dims`,
    int32 [M, N]."""
    g = _rng(seed)
    cols = [g.integers(0, int(d), size=M) for d in dims]
    return np.stack(cols, axis=1).astype(np.int32)


def ones_hashes(I, D: int = 1):
    """Identity hash tables (h_n(i) = i, s_n(i) = +1) laid out [D, sum I];
    with J_n = I_n they turn FCS into a plain polynomial product."""
    h = np.concatenate([np.arange(int(i), dtype=np.int32) for i in I])
    s = np.ones_like(h, dtype=np.int8)
    return np.tile(h, (D, 1)), np.tile(s, (D, 1))
