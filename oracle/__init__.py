"""FP64 CPU oracle for Fast Count Sketch (Cao & Liu, "Efficient Tensor
Contraction via Fast Count Sketch").

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_2106_13062_gb300``; neither imports the other.

The arithmetic lives in ``fcs_oracle.c`` (plain loops, FP64); this module only
builds that file with gcc and marshals numpy arrays through ctypes.  Every
function names the passage of the paper it follows.  Inputs are widened to
FP64 from whatever the caller passes (the harness passes FP32-rounded values).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fcs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_fcs.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile fcs_oracle.c into liboracle_fcs.so (gcc, OpenMP) if stale."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            i64p = C.POINTER(C.c_int64)
            i32p = C.POINTER(C.c_int32)
            i8p = C.POINTER(C.c_int8)
            f64p = C.POINTER(C.c_double)
            u64p = C.POINTER(C.c_uint64)
            f64pp = C.POINTER(f64p)
            sig = {
                "fcso_splitmix64": (C.c_uint64, [C.c_uint64, C.c_uint64]),
                "fcso_hash_coeffs": (None, [C.c_uint64, C.c_int, C.c_int, u64p]),
                "fcso_make_hashes": (None, [C.c_uint64, C.c_int, i64p, i32p,
                                            C.c_int, i32p, i8p]),
                "fcso_count_sketch": (None, [C.c_int64, f64p, i32p, i8p,
                                             C.c_int64, f64p]),
                "fcso_linear_convolve": (None, [C.c_int64, f64p, C.c_int64,
                                                f64p, f64p]),
                "fcso_fcs_dense": (None, [C.c_int, i64p, i64p, i32p, C.c_int,
                                          f64p, i32p, i8p, f64p]),
                "fcso_long_hash": (None, [C.c_int, i64p, i32p, i8p, i32p, i8p]),
                "fcso_ts_dense": (None, [C.c_int, i64p, i64p, C.c_int32, C.c_int,
                                         f64p, i32p, i8p, f64p]),
                "fcso_cp_to_dense": (None, [C.c_int, i64p, C.c_int64, f64pp,
                                            i64p, f64p, f64p]),
                "fcso_fcs_cp": (None, [C.c_int, i64p, i32p, C.c_int64, C.c_int,
                                       f64pp, i64p, f64p, i32p, i8p, f64p]),
                "fcso_contract_all": (None, [C.c_int, i64p, i32p, C.c_int, f64p,
                                             f64pp, i32p, i8p, f64p]),
                "fcso_contract_free": (None, [C.c_int, i64p, i32p, C.c_int,
                                              C.c_int, f64p, f64pp, i32p, i8p,
                                              f64p]),
                "fcso_median": (None, [C.c_int, C.c_int64, f64p, f64p]),
                "fcso_recover": (None, [C.c_int, i64p, i32p, C.c_int, f64p, i32p,
                                        i8p, C.c_int64, i32p, f64p, f64p]),
                "fcso_outer_combine": (None, [C.c_int, C.c_int64, f64p,
                                              C.c_int64, f64p, f64p]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


# ---------------------------------------------------------------- marshalling
def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _i8(a):
    return np.ascontiguousarray(a, dtype=np.int8)


def _ptr_array(arrs):
    arr = (C.POINTER(C.c_double) * len(arrs))()
    for k, a in enumerate(arrs):
        arr[k] = _p(a, C.c_double)
    return arr


def jtilde(J) -> int:
    """Sketch length of Def. 4: sum_n J_n - N + 1."""
    return int(sum(int(j) for j in J) - len(J) + 1)


# ---------------------------------------------------------------- hashes
def splitmix64(seed: int, k: int) -> int:
    """k-th output (0-based) of SplitMix64 seeded with `seed`."""
    return int(_load().fcso_splitmix64(C.c_uint64(seed), C.c_uint64(k)))


def hash_coeffs(seed: int, N: int, D: int) -> np.ndarray:
    """(a_h, b_h, a_s, b_s) for every (d, n), shape [D, N, 4], uint64."""
    out = np.zeros((D, N, 4), dtype=np.uint64)
    _load().fcso_hash_coeffs(C.c_uint64(seed), N, D, _p(out, C.c_uint64))
    return out


def make_hashes(seed: int, I, J, D: int):
    """Hash/sign tables of Def. 4 for D sketches: h int32 [D, sum I],
    s int8 [D, sum I] (mode n at offset sum_{m<n} I_m)."""
    I = _i64(I)
    J = _i32(J)
    tot = int(I.sum())
    h = np.zeros((D, tot), dtype=np.int32)
    s = np.zeros((D, tot), dtype=np.int8)
    _load().fcso_make_hashes(C.c_uint64(seed), len(I), _p(I, C.c_int64),
                             _p(J, C.c_int32), D, _p(h, C.c_int32),
                             _p(s, C.c_int8))
    return h, s


# ---------------------------------------------------------------- sketches
def count_sketch(x, h, s, J: int) -> np.ndarray:
    """Def. 1: CS(x)_j = sum_{h(i)=j} s(i) x(i)."""
    x = _f64(x)
    h = _i32(h)
    s = _i8(s)
    out = np.zeros(J, dtype=np.float64)
    _load().fcso_count_sketch(len(x), _p(x, C.c_double), _p(h, C.c_int32),
                              _p(s, C.c_int8), J, _p(out, C.c_double))
    return out


def linear_convolve(a, b) -> np.ndarray:
    """Full linear convolution by direct summation."""
    a = _f64(a)
    b = _f64(b)
    out = np.zeros(len(a) + len(b) - 1, dtype=np.float64)
    _load().fcso_linear_convolve(len(a), _p(a, C.c_double), len(b),
                                 _p(b, C.c_double), _p(out, C.c_double))
    return out


def fcs_dense(T, J, h, s, D: int | None = None) -> np.ndarray:
    """Eq. FCS_asyn: dense-route FCS of T (any strides).  Returns [D, Jt]."""
    T = np.asarray(T)
    I = _i64(T.shape)
    Tb = T.astype(np.float64, copy=False)
    if not Tb.flags.c_contiguous and not Tb.flags.f_contiguous:
        Tb = np.ascontiguousarray(Tb)
    stride = _i64([st // Tb.itemsize for st in Tb.strides])
    h = _i32(h)
    s = _i8(s)
    D = h.shape[0] if D is None else D
    J = _i32(J)
    out = np.zeros((D, jtilde(J)), dtype=np.float64)
    _load().fcso_fcs_dense(len(I), _p(I, C.c_int64), _p(stride, C.c_int64),
                           _p(J, C.c_int32), D, _p(Tb, C.c_double),
                           _p(h, C.c_int32), _p(s, C.c_int8),
                           _p(out, C.c_double))
    return out


def ts_dense(T, J: int, h, s, D: int | None = None) -> np.ndarray:
    """Def. 2: Tensor Sketch of T (every hash length J; bins (sum h) mod J).
    Returns [D, J]."""
    T = np.asarray(T)
    I = _i64(T.shape)
    Tb = T.astype(np.float64, copy=False)
    if not Tb.flags.c_contiguous and not Tb.flags.f_contiguous:
        Tb = np.ascontiguousarray(Tb)
    stride = _i64([st // Tb.itemsize for st in Tb.strides])
    h = _i32(h)
    s = _i8(s)
    D = h.shape[0] if D is None else D
    out = np.zeros((D, int(J)), dtype=np.float64)
    _load().fcso_ts_dense(len(I), _p(I, C.c_int64), _p(stride, C.c_int64), int(J), D,
                          _p(Tb, C.c_double), _p(h, C.c_int32), _p(s, C.c_int8),
                          _p(out, C.c_double))
    return out


def long_hash(I, hd, sd):
    """Def. 4 long hash pair over column-major vec(T) for one sketch."""
    I = _i64(I)
    hd = _i32(hd)
    sd = _i8(sd)
    numel = int(np.prod(I))
    H = np.zeros(numel, dtype=np.int32)
    S = np.zeros(numel, dtype=np.int8)
    _load().fcso_long_hash(len(I), _p(I, C.c_int64), _p(hd, C.c_int32),
                           _p(sd, C.c_int8), _p(H, C.c_int32), _p(S, C.c_int8))
    return H, S


def cp_to_dense(U, lam=None) -> np.ndarray:
    """Materialise sum_r lambda_r u_r^(1) o ... o u_r^(N) (C order)."""
    U = [_f64(u) for u in U]
    I = _i64([u.shape[0] for u in U])
    R = U[0].shape[1]
    ld = _i64([u.shape[1] for u in U])
    lamp = None if lam is None else _f64(lam)
    T = np.zeros(tuple(int(i) for i in I), dtype=np.float64)
    _load().fcso_cp_to_dense(len(U), _p(I, C.c_int64), R, _ptr_array(U),
                             _p(ld, C.c_int64),
                             None if lamp is None else _p(lamp, C.c_double),
                             _p(T, C.c_double))
    return T


def fcs_cp(U, lam, J, h, s, D: int | None = None) -> np.ndarray:
    """Eq. FCS_syn (second line): CP-route FCS by direct linear convolution
    of the per-mode count sketches, summed over rank.  Returns [D, Jt]."""
    U = [_f64(u) for u in U]
    I = _i64([u.shape[0] for u in U])
    R = U[0].shape[1]
    ld = _i64([u.shape[1] for u in U])
    lamp = None if lam is None else _f64(lam)
    h = _i32(h)
    s = _i8(s)
    D = h.shape[0] if D is None else D
    J = _i32(J)
    out = np.zeros((D, jtilde(J)), dtype=np.float64)
    _load().fcso_fcs_cp(len(U), _p(I, C.c_int64), _p(J, C.c_int32), R, D,
                        _ptr_array(U), _p(ld, C.c_int64),
                        None if lamp is None else _p(lamp, C.c_double),
                        _p(h, C.c_int32), _p(s, C.c_int8), _p(out, C.c_double))
    return out


def contract_all(fcsT, vecs, J, h, s) -> np.ndarray:
    """Eq. T_uvw (first line): e_d = <FCS_d(T), FCS_d(v_1 o ... o v_N)>.
    Returns [D]."""
    fcsT = _f64(fcsT)
    vecs = [_f64(v) for v in vecs]
    I = _i64([len(v) for v in vecs])
    J = _i32(J)
    h = _i32(h)
    s = _i8(s)
    D = fcsT.shape[0]
    out = np.zeros(D, dtype=np.float64)
    _load().fcso_contract_all(len(vecs), _p(I, C.c_int64), _p(J, C.c_int32),
                              D, _p(fcsT, C.c_double), _ptr_array(vecs),
                              _p(h, C.c_int32), _p(s, C.c_int8),
                              _p(out, C.c_double))
    return out


def contract_free(fcsT, vecs, free_mode: int, J, h, s, I=None) -> np.ndarray:
    """Eq. T_Ivw (first line) with free mode m: est_d[i] =
    <FCS_d(T), FCS_d(.. e_i (mode m) ..)>.  vecs[m] may be None if I given.
    Returns [D, I_m]."""
    fcsT = _f64(fcsT)
    if I is None:
        I = [len(v) for v in vecs]
    I = _i64(I)
    vv = [(_f64(v) if v is not None else np.zeros(int(I[k])))
          for k, v in enumerate(vecs)]
    J = _i32(J)
    h = _i32(h)
    s = _i8(s)
    D = fcsT.shape[0]
    out = np.zeros((D, int(I[free_mode])), dtype=np.float64)
    _load().fcso_contract_free(len(vv), _p(I, C.c_int64), _p(J, C.c_int32), D,
                               free_mode, _p(fcsT, C.c_double), _ptr_array(vv),
                               _p(h, C.c_int32), _p(s, C.c_int8),
                               _p(out, C.c_double))
    return out


def median(vals) -> np.ndarray:
    """Median over the first axis (Sec. 4 opening; even D -> mean of the
    two middle values)."""
    vals = _f64(vals)
    D = vals.shape[0]
    rest = vals.shape[1:]
    count = int(np.prod(rest)) if rest else 1
    out = np.zeros(count, dtype=np.float64)
    _load().fcso_median(D, count, _p(vals, C.c_double), _p(out, C.c_double))
    return out.reshape(rest)


def recover(sketch, I, J, h, s, idx, return_raw: bool = False):
    """Decompressing rule (Kronecker / contraction compression subsections):
    median_d of prod_n s_n(i_n) * sketch_d[sum_n h_n(i_n)].  idx: [M, N]."""
    sketch = _f64(sketch)
    I = _i64(I)
    J = _i32(J)
    h = _i32(h)
    s = _i8(s)
    idx = _i32(idx)
    D = sketch.shape[0]
    M = idx.shape[0]
    raw = np.zeros((D, M), dtype=np.float64)
    out = np.zeros(M, dtype=np.float64)
    _load().fcso_recover(len(I), _p(I, C.c_int64), _p(J, C.c_int32), D,
                         _p(sketch, C.c_double), _p(h, C.c_int32),
                         _p(s, C.c_int8), M, _p(idx, C.c_int32),
                         _p(raw, C.c_double), _p(out, C.c_double))
    return (out, raw) if return_raw else out


def outer_combine(fa, fb) -> np.ndarray:
    """FCS(A o B) = FCS(A) (*) FCS(B) per sketch (Kronecker product
    compression).  fa: [D, La], fb: [D, Lb] -> [D, La+Lb-1]."""
    fa = _f64(fa)
    fb = _f64(fb)
    D, La = fa.shape
    Lb = fb.shape[1]
    out = np.zeros((D, La + Lb - 1), dtype=np.float64)
    _load().fcso_outer_combine(D, La, _p(fa, C.c_double), Lb,
                               _p(fb, C.c_double), _p(out, C.c_double))
    return out
