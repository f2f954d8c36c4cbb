"""Fast Count Sketch (Cao & Liu, "Efficient Tensor Contraction via Fast Count
Sketch") on one GB300: a thin Python binding over the C ABI of ``libfcs.so``.

Every function here only marshals arguments (torch tensors -> device pointers
and sizes, the current torch stream) and calls the C entry point of the same
name; all arithmetic runs in the library's CUDA kernels.  There is no CPU path:
if ``libfcs.so`` is missing or no GPU is present, calls raise.

Names follow the C ABI (``include/fcs.h``):
    fcs_make_hashes, fcs_sketch_dense, fcs_sketch_cp, fcs_contract,
    fcs_recover, fcs_sketch_outer
plus ``Context`` (fcs_create / fcs_destroy) and ``build()``.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
import weakref

import torch

from .build import LIB as _LIB_PATH, build  # noqa: F401

FCS_OK = 0
FCS_EINVAL = 1
FCS_ENOMEM_BUDGET = 2
FCS_ECUDA = 3
FCS_ETIMEOUT = 4
FCS_EUNSUPPORTED = 5
FCS_CONTRACT_ALL = 0
FCS_CONTRACT_FREE = 1

_lock = threading.Lock()
_lib = None


class FcsError(RuntimeError):
    """A libfcs call returned a non-zero status."""

    def __init__(self, code: int, msg: str):
        super().__init__(f"libfcs status {code}: {msg}")
        self.code = code


def lib() -> C.CDLL:
    """Load libfcs.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(
                    f"{_LIB_PATH} is missing: build it with "
                    "paper_2106_13062_gb300.build() (nvcc, sm_103a)")
            L = C.CDLL(_LIB_PATH)
            vp, i64p, i32p, i8p, f32p = (C.c_void_p, C.POINTER(C.c_int64),
                                         C.POINTER(C.c_int32), C.c_void_p,
                                         C.c_void_p)
            sig = {
                "fcs_version": (C.c_int, []),
                "fcs_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, vp,
                                         C.c_size_t]),
                "fcs_destroy": (C.c_int, [vp]),
                "fcs_set_stream": (C.c_int, [vp, vp]),
                "fcs_last_error": (C.c_char_p, [vp]),
                "fcs_workspace_bytes": (C.c_size_t, [vp]),
                "fcs_make_hashes": (C.c_int, [vp, C.c_uint64, C.c_int, i64p, i32p,
                                              C.c_int, vp, vp]),
                "fcs_sketch_dense": (C.c_int, [vp, C.c_int, i64p, i64p, i32p,
                                               C.c_int, vp, vp, vp, C.c_int64,
                                               vp, C.c_int64, C.c_int64,
                                               C.c_int64]),
                "fcs_sketch_cp": (C.c_int, [vp, C.c_int, i64p, i32p, C.c_int64,
                                            C.c_int, C.POINTER(C.c_void_p), i64p,
                                            vp, vp, vp, C.c_int64, vp]),
                "fcs_sketch_cp_seeded": (C.c_int, [vp, C.c_uint64, C.c_int, i64p, i32p,
                                                   C.c_int64, C.c_int, C.POINTER(C.c_void_p),
                                                   i64p, vp, vp, vp, vp]),
                "fcs_sketch_cp_host": (C.c_int, [vp, C.c_int, i64p, i32p, C.c_int64,
                                                 C.c_int, C.POINTER(C.c_void_p), i64p,
                                                 vp, C.c_uint64, vp]),
                "fcs_sketch_cp_noalloc": (C.c_int, [vp, C.c_int, i64p, i32p,
                                                    C.c_int64, C.c_int,
                                                    C.POINTER(C.c_void_p), i64p,
                                                    vp, vp, vp, C.c_int64, vp,
                                                    C.c_char_p, C.c_size_t]),
                "fcs_cache_spectra": (C.c_int, [vp, C.c_int]),
                "fcs_fold": (C.c_int, [vp, C.c_int64, C.c_int64, vp, C.c_int64, vp]),
                "fcs_sketch_inner": (C.c_int, [vp, C.c_int, C.c_int64, C.c_int64, vp,
                                               C.c_int64, vp, vp, vp, vp]),
                "fcs_sketch_outer_sum": (C.c_int, [vp, C.c_int64, C.c_int64, C.c_int,
                                                   C.c_int64, C.c_int64, vp, vp, vp]),
                "fcs_outer_autotune": (C.c_int, [vp, C.c_int64, C.c_int64, C.c_int,
                                                 C.c_int64, C.c_int64, vp, vp, vp,
                                                 C.POINTER(C.c_int)]),
                "fcs_rtpm": (C.c_int, [vp, C.c_int, C.c_int64, i32p, C.c_int, vp, vp,
                                       vp, C.c_int64, C.c_int, C.c_int, C.c_int, vp,
                                       vp, vp]),
                "fcs_als": (C.c_int, [vp, C.c_int, i64p, i32p, C.c_int, vp, vp, vp,
                                      C.c_int64, C.c_int, C.c_int,
                                      C.POINTER(C.c_void_p), vp]),
                "fcs_forget": (C.c_int, [vp, vp]),
                "fcs_contract": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, i64p,
                                           i32p, C.c_int, vp, C.c_int64,
                                           C.POINTER(C.c_void_p), vp, vp,
                                           C.c_int64, vp, vp]),
                "fcs_contract_both": (C.c_int, [vp, C.c_int, C.c_int, i64p, i32p,
                                                C.c_int, vp, C.c_int64,
                                                C.POINTER(C.c_void_p), vp, vp,
                                                C.c_int64, vp, vp, vp, vp]),
                "fcs_recover": (C.c_int, [vp, C.c_int, i64p, i32p, C.c_int, vp,
                                          vp, vp, C.c_int64, C.c_int64, vp, vp,
                                          vp, C.c_int64, C.c_int64, C.c_int64,
                                          C.c_int64]),
                "fcs_sketch_outer": (C.c_int, [vp, C.c_int64, C.c_int, C.c_int64,
                                               C.c_int64, vp, vp, vp]),
                "fcs_batch_plan_create": (C.c_int, [vp, C.c_int, C.POINTER(CpProblem),
                                                    C.c_int, C.POINTER(C.c_void_p)]),
                "fcs_batch_plan_launch": (C.c_int, [vp, vp]),
                "fcs_batch_plan_destroy": (C.c_int, [vp]),
                "fcs_batch_sketch_cp": (C.c_int, [vp, C.c_int, C.POINTER(CpProblem),
                                                  C.c_int]),
                "fcs_batch_autotune": (C.c_int, [vp, C.c_int, C.POINTER(CpProblem),
                                                 C.POINTER(C.c_int)]),
                "fcs_batch_plan_create_cfg": (C.c_int, [vp, C.c_int, C.POINTER(CpProblem),
                                                        C.c_int, C.c_int,
                                                        C.POINTER(BatchClassCfg),
                                                        C.POINTER(C.c_void_p)]),
                "fcs_batch_plan_config": (C.c_int, [vp, C.POINTER(C.c_int), C.c_int,
                                                    C.POINTER(BatchClassCfg),
                                                    C.POINTER(C.c_int)]),
                "fcs_server_create": (C.c_int, [C.POINTER(ServerConfig),
                                                C.POINTER(C.c_void_p)]),
                "fcs_server_destroy": (C.c_int, [vp]),
                "fcs_server_submit": (C.c_int, [vp, C.POINTER(Request),
                                                C.POINTER(C.c_int64)]),
                "fcs_server_poll": (C.c_int, [vp, C.c_int64, C.POINTER(Result)]),
                "fcs_server_wait": (C.c_int, [vp, C.c_int64, C.c_double,
                                              C.POINTER(Result)]),
                "fcs_server_cancel": (C.c_int, [vp, C.c_int64]),
                "fcs_server_release": (C.c_int, [vp, C.c_int64]),
                "fcs_server_stats": (C.c_int, [vp, C.POINTER(Stats)]),
                "fcs_server_reset_stats": (C.c_int, [vp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            del i8p, f32p
            _lib = L
    return _lib


class CpProblem(C.Structure):
    """Mirror of `fcs_cp_problem` (include/fcs.h)."""
    _fields_ = [("N", C.c_int), ("D", C.c_int), ("R", C.c_int64),
                ("I", C.c_int64 * 8), ("J", C.c_int32 * 8),
                ("U", C.c_void_p * 8), ("ldU", C.c_int64 * 8),
                ("lam", C.c_void_p), ("h", C.c_void_p), ("s", C.c_void_p),
                ("ldh", C.c_int64), ("out", C.c_void_p)]


class BatchClassCfg(C.Structure):
    """Mirror of `fcs_batch_class_cfg`."""
    _fields_ = [("fft_len", C.c_int), ("engine", C.c_int), ("thread_mult", C.c_int),
                ("items_per_cta", C.c_int), ("threads", C.c_int)]


FCS_REQ_CP = 0
FCS_REQ_CONTRACT = 1


class ServerConfig(C.Structure):
    """Mirror of `fcs_server_config`."""
    _fields_ = [("device", C.c_int), ("streams", C.c_int), ("max_inflight", C.c_int),
                ("max_batch", C.c_int), ("arena_bytes", C.c_size_t),
                ("staging_bytes", C.c_size_t), ("workspace_bytes", C.c_size_t)]


class Request(C.Structure):
    """Mirror of `fcs_request`."""
    _fields_ = [("kind", C.c_int), ("N", C.c_int), ("I", C.c_int64 * 8),
                ("J", C.c_int32 * 8), ("D", C.c_int), ("R", C.c_int64),
                ("seed", C.c_uint64), ("host_U", C.c_void_p * 8),
                ("host_lambda", C.c_void_p), ("host_out", C.c_void_p),
                ("keep_resident", C.c_int), ("sketch_id", C.c_int64),
                ("contract_kind", C.c_int), ("free_mode", C.c_int), ("B", C.c_int64),
                ("host_vecs", C.c_void_p * 8), ("host_result", C.c_void_p)]


class Result(C.Structure):
    """Mirror of `fcs_result`."""
    _fields_ = [("ticket", C.c_int64), ("state", C.c_int), ("status", C.c_int),
                ("sketch_id", C.c_int64), ("latency_s", C.c_double)]


class Stats(C.Structure):
    """Mirror of `fcs_stats`."""
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64),
                ("failed", C.c_int64), ("cancelled", C.c_int64),
                ("rounds", C.c_int64), ("sketches", C.c_int64),
                ("max_inflight_seen", C.c_int64), ("arena_used", C.c_size_t),
                ("p50_latency_s", C.c_double), ("p99_latency_s", C.c_double),
                ("mean_latency_s", C.c_double), ("busy_s", C.c_double),
                ("batch_launches", C.c_int64)]


def exported_symbols():
    """Names of the C entry points this binding expects libfcs.so to export."""
    return ["fcs_version", "fcs_create", "fcs_destroy", "fcs_set_stream",
            "fcs_last_error", "fcs_workspace_bytes", "fcs_make_hashes",
            "fcs_sketch_dense", "fcs_sketch_cp", "fcs_sketch_cp_seeded", "fcs_sketch_cp_noalloc",
            "fcs_sketch_cp_host",
            "fcs_contract", "fcs_contract_both", "fcs_cache_spectra", "fcs_forget",
            "fcs_fold", "fcs_sketch_inner", "fcs_rtpm", "fcs_als",
            "fcs_recover", "fcs_sketch_outer", "fcs_sketch_outer_sum", "fcs_outer_autotune",
            "fcs_batch_plan_create", "fcs_batch_plan_launch",
            "fcs_batch_plan_destroy", "fcs_batch_sketch_cp", "fcs_batch_autotune",
            "fcs_batch_plan_create_cfg", "fcs_batch_plan_config",
            "fcs_server_create", "fcs_server_destroy", "fcs_server_submit",
            "fcs_server_poll", "fcs_server_wait", "fcs_server_cancel",
            "fcs_server_release", "fcs_server_stats", "fcs_server_reset_stats"]


# ------------------------------------------------------------------ helpers
def _arr(ctype, vals):
    vals = [int(v) for v in vals]
    return (ctype * max(1, len(vals)))(*vals)


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _need(t: torch.Tensor, dtype, name: str, contiguous: bool = True):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if contiguous and not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _tables(h, s, ldh: int):
    """Check the hash tables and return the sketch-row stride to pass: h and s
    may be row-strided views (e.g. a run of modes of a wider table) as long as
    both share the row stride and each row is contiguous."""
    _need(h, torch.int32, "h", contiguous=False)
    _need(s, torch.int8, "s", contiguous=False)
    if h.dim() != 2 or s.shape != h.shape:
        raise ValueError("h and s must both be [D, sum I]")
    if h.stride(1) != 1 or s.stride(1) != 1:
        raise ValueError("hash table rows must be contiguous")
    if h.shape[0] > 1 and h.stride(0) != s.stride(0):
        raise ValueError("h and s must share the row stride")
    row = h.stride(0) if h.shape[0] > 1 else h.shape[1]
    if ldh and h.shape[0] > 1 and ldh != row:
        raise ValueError(f"ldh={ldh} disagrees with the tables' row stride {row}")
    return ldh or (row if row != h.shape[1] else 0)


def jtilde(J) -> int:
    """Sketch length of Def. 4: sum_n J_n - N + 1."""
    return int(sum(int(j) for j in J) - len(J) + 1)


def _same_device(name_tensors):
    """Every tensor of a call must live on one device (the one the call runs on)."""
    dev = None
    for name, t in name_tensors:
        if t is None:
            continue
        if dev is None:
            dev = t.device
        elif t.device != dev:
            raise ValueError(f"{name} is on {t.device}, expected {dev}")
    return dev


def _covers(h, I, name="h"):
    """The hash tables must hold at least sum(I_n) entries per sketch row."""
    tot = int(sum(int(i) for i in I))
    if h.shape[1] < tot:
        raise ValueError(f"{name} has {h.shape[1]} columns per sketch, sum(I_n) = {tot}")


def _room(t, n: int, name: str):
    """A caller-given output must hold at least n elements."""
    if t.numel() < n:
        raise ValueError(f"{name} holds {t.numel()} elements, the call writes {n}")


def _check_sketch(sk, J, I, h, s, others=()):
    """A sketch argument must be [.., D, Jt] with D matching the tables, and
    the tables must cover every mode."""
    if len(J) != len(I):
        raise ValueError("need one hash length J_n per mode")
    if sk.shape[-1] != jtilde(J):
        raise ValueError(f"sketch rows hold {sk.shape[-1]} bins, Jt = {jtilde(J)}")
    if sk.dim() < 2 or sk.shape[-2] > h.shape[0]:
        raise ValueError("sketch must be [.., D, Jt] with at least D rows of hash tables")
    _covers(h, I)
    _same_device([("sketch", sk), ("h", h), ("s", s),
                  *[(f"argument {k}", t) for k, t in enumerate(others)]])


def _check_cp(U, lam, J, h, s, out):
    """Shape checks shared by the CP-route wrappers: factors I_n x R with unit
    column stride, one hash length per mode, lambda of at least R entries,
    tables covering every mode, and room for D x Jt outputs."""
    N = len(U)
    if N < 1 or len(J) != N:
        raise ValueError("need one hash length J_n per factor matrix")
    R = U[0].shape[1]
    for k, u in enumerate(U):
        _need(u, torch.float32, f"U[{k}]", contiguous=False)
        if u.dim() != 2 or u.shape[1] != R or u.stride(1) != 1:
            raise ValueError("each U_n must be I_n x R with unit column stride")
    if lam is not None:
        _need(lam, torch.float32, "lambda")
        _room(lam, R, "lambda")
    _covers(h, [u.shape[0] for u in U])
    if out is not None:
        _need(out, torch.float32, "out")
        _room(out, h.shape[0] * jtilde(J), "out")
    _same_device([("U[0]", U[0]), *[(f"U[{k}]", u) for k, u in enumerate(U)],
                  ("lambda", lam), ("h", h), ("s", s), ("out", out)])
    return N, R


class Context:
    """An fcs_ctx bound to one device and (by default) torch's current
    stream of that device at each call."""

    def __init__(self, device: int | None = None, budget: int | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("libfcs needs a CUDA GPU; none is available")
        self.device = torch.cuda.current_device() if device is None else device
        h = C.c_void_p()
        stream = torch.cuda.current_stream(self.device).cuda_stream
        b = C.c_size_t(-1).value if budget is None else int(budget)
        rc = lib().fcs_create(C.byref(h), self.device, C.c_void_p(stream), b)
        if rc != FCS_OK:
            raise FcsError(rc, "fcs_create failed")
        self._h = h
        self._plans = weakref.WeakSet()      # batch plans, closed before the context

    @property
    def handle(self):
        return self._h

    def _sync_stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        lib().fcs_set_stream(self._h, C.c_void_p(s))

    def check(self, rc: int):
        if rc != FCS_OK:
            msg = lib().fcs_last_error(self._h).decode(errors="replace")
            raise FcsError(rc, msg)

    def workspace_bytes(self) -> int:
        return int(lib().fcs_workspace_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            for p in list(getattr(self, "_plans", ())):
                p.close()
            lib().fcs_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ calls
def fcs_make_hashes(ctx: Context, seed: int, I, J, D: int):
    """Hash/sign tables of Def. 4 for D sketches: (h int32 [D, sum I],
    s int8 [D, sum I]) on ctx's device."""
    ctx._sync_stream()
    tot = int(sum(int(i) for i in I))
    dev = torch.device("cuda", ctx.device)
    h = torch.empty((D, tot), dtype=torch.int32, device=dev)
    s = torch.empty((D, tot), dtype=torch.int8, device=dev)
    ctx.check(lib().fcs_make_hashes(ctx.handle, C.c_uint64(int(seed)), len(I),
                                    _arr(C.c_int64, I), _arr(C.c_int32, J), D,
                                    _ptr(h), _ptr(s)))
    return h, s


def fcs_sketch_dense(ctx: Context, T: torch.Tensor, J, h, s, ldh: int = 0,
                     batched: bool = False, out: torch.Tensor | None = None):
    """Eq. (FCS_asyn) dense-route FCS of T (any element strides).  With
    batched=True the first dimension of T indexes independent tensors.
    Returns [D, Jt] (or [B, D, Jt])."""
    ctx._sync_stream()
    _need(T, torch.float32, "T", contiguous=False)
    ldh = _tables(h, s, ldh)
    D = h.shape[0]
    Jt = jtilde(J)
    shape = list(T.shape[1:] if batched else T.shape)
    strides = list(T.stride()[1:] if batched else T.stride())
    nb = T.shape[0] if batched else 1
    if len(shape) != len(J):
        raise ValueError("T's order does not match len(J)")
    _covers(h, shape)
    if out is None:
        out = torch.empty(((nb,) if batched else ()) + (D, Jt),
                          dtype=torch.float32, device=T.device)
    _need(out, torch.float32, "out")
    _room(out, nb * D * Jt, "out")
    _same_device([("T", T), ("h", h), ("s", s), ("out", out)])
    ctx.check(lib().fcs_sketch_dense(
        ctx.handle, len(J), _arr(C.c_int64, shape), _arr(C.c_int64, strides),
        _arr(C.c_int32, J), D, _ptr(T), _ptr(h), _ptr(s), ldh, _ptr(out), nb,
        T.stride(0) if batched else 0, D * Jt))
    return out


def fcs_sketch_cp(ctx: Context, U, lam, J, h, s, ldh: int = 0,
                  out: torch.Tensor | None = None):
    """Eq. (FCS_syn) CP-route FCS of [[lam; U_1..U_N]] (U_n: I_n x R FP32,
    row-major).  Returns [D, Jt]."""
    ctx._sync_stream()
    ldh = _tables(h, s, ldh)
    N, R = _check_cp(U, lam, J, h, s, out)
    D = h.shape[0]
    Jt = jtilde(J)
    if out is None:
        out = torch.empty((D, Jt), dtype=torch.float32, device=U[0].device)
    ptrs = (C.c_void_p * N)(*[u.data_ptr() for u in U])
    ctx.check(lib().fcs_sketch_cp(
        ctx.handle, N, _arr(C.c_int64, [u.shape[0] for u in U]),
        _arr(C.c_int32, J), R, D, ptrs, _arr(C.c_int64, [u.stride(0) for u in U]),
        _ptr(lam), _ptr(h), _ptr(s), ldh, _ptr(out)))
    return out


def fcs_sketch_cp_seeded(ctx: Context, U, lam, J, D: int, seed: int,
                         out: torch.Tensor | None = None, h: torch.Tensor | None = None,
                         s: torch.Tensor | None = None):
    """fcs_make_hashes + fcs_sketch_cp in one call (fcs_sketch_cp_seeded): the
    hash tables of `seed` go to h (int32) and s (int8), both [D, sum I] and
    densely packed (allocated here unless given), and the sketch of
    [[lam; U_1..U_N]] to out [D, Jt].  Returns (out, h, s)."""
    ctx._sync_stream()
    if not U:
        raise ValueError("need at least one factor matrix")
    I = [int(u.shape[0]) for u in U]
    tot = sum(I)
    dev = U[0].device
    if h is None:
        h = torch.empty((int(D), tot), dtype=torch.int32, device=dev)
    if s is None:
        s = torch.empty((int(D), tot), dtype=torch.int8, device=dev)
    _need(h, torch.int32, "h")
    _need(s, torch.int8, "s")
    if tuple(h.shape) != (int(D), tot) or tuple(s.shape) != (int(D), tot):
        raise ValueError("h and s must be [D, sum I] (densely packed tables)")
    N, R = _check_cp(U, lam, J, h, s, out)
    Jt = jtilde(J)
    if out is None:
        out = torch.empty((int(D), Jt), dtype=torch.float32, device=dev)
    ptrs = (C.c_void_p * N)(*[u.data_ptr() for u in U])
    ctx.check(lib().fcs_sketch_cp_seeded(
        ctx.handle, C.c_uint64(int(seed)), N, _arr(C.c_int64, I), _arr(C.c_int32, J), R,
        int(D), ptrs, _arr(C.c_int64, [u.stride(0) for u in U]), _ptr(lam), _ptr(h), _ptr(s),
        _ptr(out)))
    return out, h, s


def fcs_sketch_cp_host(ctx: Context, U, lam, J, D: int, seed: int,
                       out: torch.Tensor | None = None):
    """CP-route FCS from host factors to a host sketch (fcs_sketch_cp_host):
    U_n are CPU float32 tensors I_n x R with unit column stride (pinned ones
    make the copies asynchronous), lam a CPU [R] tensor or None; hash tables
    from `seed` as fcs_make_hashes.  Returns the CPU [D, Jt] output (given or
    allocated pinned); it is complete once torch's current stream of the
    context's device has been synchronised."""
    ctx._sync_stream()
    N = len(U)
    if N < 1 or len(J) != N:
        raise ValueError("need one hash length J_n per factor matrix")
    R = U[0].shape[1]
    for k, u in enumerate(U):
        if not isinstance(u, torch.Tensor) or u.is_cuda or u.dtype != torch.float32:
            raise TypeError(f"U[{k}] must be a CPU float32 tensor")
        if u.dim() != 2 or u.shape[1] != R or u.stride(1) != 1:
            raise ValueError("each U_n must be I_n x R with unit column stride")
    if lam is not None:
        if lam.is_cuda or lam.dtype != torch.float32 or lam.numel() < R or not lam.is_contiguous():
            raise ValueError("lambda must be a contiguous CPU float32 tensor of at least R entries")
    Jt = jtilde(J)
    if out is None:
        out = torch.empty((D, Jt), dtype=torch.float32).pin_memory()
    if out.is_cuda or out.dtype != torch.float32 or not out.is_contiguous() or out.numel() < D * Jt:
        raise ValueError("out must be a contiguous CPU float32 tensor of D x Jt entries")
    ptrs = (C.c_void_p * N)(*[u.data_ptr() for u in U])
    ctx.check(lib().fcs_sketch_cp_host(
        ctx.handle, N, _arr(C.c_int64, [u.shape[0] for u in U]), _arr(C.c_int32, J), R, int(D),
        ptrs, _arr(C.c_int64, [u.stride(0) for u in U]),
        None if lam is None else C.c_void_p(lam.data_ptr()), C.c_uint64(int(seed)),
        C.c_void_p(out.data_ptr())))
    return out


def fcs_sketch_cp_noalloc(U, lam, J, h, s, ldh: int = 0,
                          out: torch.Tensor | None = None):
    """fcs_sketch_cp without a context and without device allocation inside
    the library (scratch lives in a fixed 4 MiB device array; see
    include/fcs.h).  Runs on the device that holds the tensors (made current
    for the call) and on torch's current stream of that device.  The output
    tensor is allocated here by torch unless `out` is given.  This call does
    not drop spectrum-cache entries of `out` in any context: call fcs_forget
    on each caching context after re-sketching into a cached buffer."""
    ldh = _tables(h, s, ldh)
    N, R = _check_cp(U, lam, J, h, s, out)
    D = h.shape[0]
    dev = U[0].device
    if out is None:
        out = torch.empty((D, jtilde(J)), dtype=torch.float32, device=dev)
    ptrs = (C.c_void_p * N)(*[u.data_ptr() for u in U])
    err = C.create_string_buffer(256)
    with torch.cuda.device(dev):
        stream = torch.cuda.current_stream(dev).cuda_stream
        rc = lib().fcs_sketch_cp_noalloc(
            C.c_void_p(stream), N, _arr(C.c_int64, [u.shape[0] for u in U]),
            _arr(C.c_int32, J), R, D, ptrs, _arr(C.c_int64, [u.stride(0) for u in U]),
            _ptr(lam), _ptr(h), _ptr(s), ldh, _ptr(out), err, 256)
    if rc != FCS_OK:
        raise FcsError(rc, err.value.decode(errors="replace"))
    return out


def fcs_cache_spectra(ctx: Context, enable: bool = True):
    """Turn the context's cache of sketch spectra for fcs_contract on or off
    (off drops every entry).  Cached entries are keyed by the sketch's data
    pointer: call fcs_forget before changing or freeing a cached sketch."""
    ctx.check(lib().fcs_cache_spectra(ctx.handle, 1 if enable else 0))


def fcs_forget(ctx: Context, sketch):
    """Drop the cached spectra of `sketch` (a tensor or a device address)."""
    p = sketch.data_ptr() if isinstance(sketch, torch.Tensor) else int(sketch)
    ctx.check(lib().fcs_forget(ctx.handle, C.c_void_p(p)))


def fcs_contract(ctx: Context, kind: int, fcsT: torch.Tensor, vecs, I, J, h, s,
                 free_mode: int = 0, ldh: int = 0, raw: bool = False):
    """Sketched contractions (eqs. T_uvw / T_Ivw).  vecs[n]: [B, I_n] FP32
    (vecs[free_mode] may be None for FCS_CONTRACT_FREE).  Returns the median
    over sketches ([B] or [B, I_m]) and, with raw=True, also the per-sketch
    values ([B, D] or [B, D, I_m])."""
    ctx._sync_stream()
    _need(fcsT, torch.float32, "fcsT")
    ldh = _tables(h, s, ldh)
    N = len(J)
    D = fcsT.shape[0]
    B = None
    ptrs = (C.c_void_p * N)()
    for n in range(N):
        v = vecs[n]
        if kind == FCS_CONTRACT_FREE and n == free_mode:
            ptrs[n] = None
            continue
        _need(v, torch.float32, f"vecs[{n}]")
        B = v.shape[0] if B is None else B
        if v.shape != (B, int(I[n])):
            raise ValueError(f"vecs[{n}] must be [B, I_{n}]")
        ptrs[n] = v.data_ptr()
    if B is None:
        raise ValueError("no vectors given")
    _check_sketch(fcsT, J, I, h, s, [v for v in vecs if v is not None])
    dev = fcsT.device
    if kind == FCS_CONTRACT_ALL:
        med = torch.empty((B,), dtype=torch.float32, device=dev)
        rawt = torch.empty((B, D), dtype=torch.float32, device=dev) if raw else None
    else:
        Im = int(I[free_mode])
        med = torch.empty((B, Im), dtype=torch.float32, device=dev)
        rawt = (torch.empty((B, D, Im), dtype=torch.float32, device=dev)
                if raw else None)
    ctx.check(lib().fcs_contract(
        ctx.handle, kind, free_mode, N, _arr(C.c_int64, I), _arr(C.c_int32, J), D,
        _ptr(fcsT), B, ptrs, _ptr(h), _ptr(s), ldh, _ptr(med), _ptr(rawt)))
    return (med, rawt) if raw else med


def fcs_contract_both(ctx: Context, fcsT: torch.Tensor, vecs, I, J, h, s,
                      free_mode: int = 0, ldh: int = 0, raw: bool = False):
    """T(v_1..v_N) and T(v_1, .., I (mode free_mode), .., v_N) from one set
    of transforms.  vecs[n]: [B, I_n] FP32 for every n.  Returns
    (all [B], free [B, I_m]) medians over the sketches and, with raw=True,
    also the per-sketch values ([B, D], [B, D, I_m])."""
    ctx._sync_stream()
    _need(fcsT, torch.float32, "fcsT")
    ldh = _tables(h, s, ldh)
    N = len(J)
    D = fcsT.shape[0]
    ptrs = (C.c_void_p * N)()
    B = None
    for n in range(N):
        v = vecs[n]
        _need(v, torch.float32, f"vecs[{n}]")
        B = v.shape[0] if B is None else B
        if v.shape != (B, int(I[n])):
            raise ValueError(f"vecs[{n}] must be [B, I_{n}]")
        ptrs[n] = v.data_ptr()
    _check_sketch(fcsT, J, I, h, s, vecs)
    dev = fcsT.device
    Im = int(I[free_mode])
    med_all = torch.empty((B,), dtype=torch.float32, device=dev)
    med_free = torch.empty((B, Im), dtype=torch.float32, device=dev)
    raw_all = torch.empty((B, D), dtype=torch.float32, device=dev) if raw else None
    raw_free = torch.empty((B, D, Im), dtype=torch.float32, device=dev) if raw else None
    ctx.check(lib().fcs_contract_both(
        ctx.handle, free_mode, N, _arr(C.c_int64, I), _arr(C.c_int32, J), D, _ptr(fcsT), B,
        ptrs, _ptr(h), _ptr(s), ldh, _ptr(med_all), _ptr(med_free), _ptr(raw_all),
        _ptr(raw_free)))
    return (med_all, med_free, raw_all, raw_free) if raw else (med_all, med_free)


def fcs_recover(ctx: Context, sketch: torch.Tensor, I, J, h, s, idx: torch.Tensor,
                ldh: int = 0, raw: bool = False):
    """Entry recovery (decompressing rule): median over sketches of
    prod s * sketch[sum h].  sketch [D, Jt] with idx [M, N], or batched
    sketch [B, D, Jt] with idx [B, M, N].  Returns [M] (or [B, M]), plus the
    raw [D, M] values with raw=True (unbatched only)."""
    ctx._sync_stream()
    _need(sketch, torch.float32, "sketch")
    _need(idx, torch.int32, "idx")
    ldh = _tables(h, s, ldh)
    N = len(J)
    batched = sketch.dim() == 3
    nb = sketch.shape[0] if batched else 1
    D = sketch.shape[-2]
    M = idx.shape[-2]
    if idx.shape[-1] != N:
        raise ValueError("idx must be [.., M, N]")
    if batched != (idx.dim() == 3) or (batched and idx.shape[0] != nb):
        raise ValueError("batched sketch [B, D, Jt] needs idx [B, M, N]")
    _check_sketch(sketch, J, I, h, s, [idx])
    out = torch.empty(((nb,) if batched else ()) + (M,), dtype=torch.float32,
                      device=sketch.device)
    rawt = None
    if raw:
        if batched:
            raise ValueError("raw output is only available unbatched")
        rawt = torch.empty((D, M), dtype=torch.float32, device=sketch.device)
    ctx.check(lib().fcs_recover(
        ctx.handle, N, _arr(C.c_int64, I), _arr(C.c_int32, J), D, _ptr(sketch),
        _ptr(h), _ptr(s), ldh, M, _ptr(idx), _ptr(out), _ptr(rawt), nb,
        D * sketch.shape[-1] if batched else 0, M * N if batched else 0,
        M if batched else 0))
    return (out, rawt) if raw else out


def fcs_sketch_outer(ctx: Context, fa: torch.Tensor, fb: torch.Tensor):
    """Sketch of an outer product from its factors' sketches (Kronecker
    compression): full linear convolution per sketch.  fa [.., D, La],
    fb [.., D, Lb] -> [.., D, La+Lb-1]."""
    ctx._sync_stream()
    _need(fa, torch.float32, "fa")
    _need(fb, torch.float32, "fb")
    if fa.shape[:-1] != fb.shape[:-1]:
        raise ValueError("fa and fb must share leading dimensions")
    D = fa.shape[-2]
    La, Lb = fa.shape[-1], fb.shape[-1]
    nb = fa.numel() // (D * La)
    out = torch.empty(fa.shape[:-1] + (La + Lb - 1,), dtype=torch.float32,
                      device=fa.device)
    ctx.check(lib().fcs_sketch_outer(ctx.handle, nb, D, La, Lb, _ptr(fa),
                                     _ptr(fb), _ptr(out)))
    return out


def fcs_sketch_outer_sum(ctx: Context, fa: torch.Tensor, fb: torch.Tensor):
    """Tensor contraction compression: sum over slices l of the convolved
    slice sketches.  fa [.., L, D, La], fb [.., L, D, Lb] -> [.., D, La+Lb-1]."""
    ctx._sync_stream()
    _need(fa, torch.float32, "fa")
    _need(fb, torch.float32, "fb")
    if fa.dim() < 3 or fa.shape[:-1] != fb.shape[:-1]:
        raise ValueError("fa and fb must be [.., L, D, len] with equal leading dims")
    Ls, D = fa.shape[-3], fa.shape[-2]
    La, Lb = fa.shape[-1], fb.shape[-1]
    nb = fa.numel() // (Ls * D * La)
    out = torch.empty(fa.shape[:-3] + (D, La + Lb - 1), dtype=torch.float32,
                      device=fa.device)
    ctx.check(lib().fcs_sketch_outer_sum(ctx.handle, nb, Ls, D, La, Lb, _ptr(fa),
                                         _ptr(fb), _ptr(out)))
    return out


def fcs_outer_autotune(ctx: Context, fa: torch.Tensor, fb: torch.Tensor, slices: bool = False) -> int:
    """Choose the block size of fcs_sketch_outer (slices=False: fa [.., D, La])
    or fcs_sketch_outer_sum (slices=True: fa [.., L, D, La]) for this shape by
    timing both on these inputs; later calls of the shape use it.  Returns
    (block size chosen, 0 for the two-pass route; the output of the shape
    timed last)."""
    ctx._sync_stream()
    _need(fa, torch.float32, "fa")
    _need(fb, torch.float32, "fb")
    if fa.shape[:-1] != fb.shape[:-1] or (slices and fa.dim() < 3):
        raise ValueError("fa and fb must share leading dimensions")
    Ls = fa.shape[-3] if slices else 1
    D = fa.shape[-2]
    La, Lb = fa.shape[-1], fb.shape[-1]
    nb = fa.numel() // (Ls * D * La)
    lead = fa.shape[:-3] if slices else fa.shape[:-2]
    out = torch.empty(tuple(lead) + (D, La + Lb - 1), dtype=torch.float32, device=fa.device)
    nt = C.c_int(0)
    ctx.check(lib().fcs_outer_autotune(ctx.handle, nb, Ls, D, La, Lb, _ptr(fa), _ptr(fb),
                                       _ptr(out), C.byref(nt)))
    return nt.value, out


def fcs_fold(ctx: Context, x: torch.Tensor, J: int):
    """Tensor Sketch (Def. 2) from FCS sketches with every J_n = J: sum of the
    bins congruent mod J.  x [.., Jt] -> [.., J]."""
    ctx._sync_stream()
    _need(x, torch.float32, "x")
    Jt = x.shape[-1]
    rows = x.numel() // Jt
    out = torch.empty(x.shape[:-1] + (int(J),), dtype=torch.float32, device=x.device)
    ctx.check(lib().fcs_fold(ctx.handle, rows, Jt, _ptr(x), int(J), _ptr(out)))
    return out


def fcs_sketch_inner(ctx: Context, sa: torch.Tensor, sw: torch.Tensor,
                     bias: torch.Tensor | None = None, raw: bool = False):
    """Compressed TRL (eq. net_compress): Y[b][c] = median_d <sa[b][d], sw[c][d]>
    + bias[c].  sa [B, D, Jt], sw [C, D, Jt].  Returns Y [B, C] (and raw
    [B, C, D] with raw=True)."""
    ctx._sync_stream()
    _need(sa, torch.float32, "sa")
    _need(sw, torch.float32, "sw")
    if bias is not None:
        _need(bias, torch.float32, "bias")
    Bn, D, Jt = sa.shape
    Cn = sw.shape[0]
    if sw.shape[1:] != (D, Jt):
        raise ValueError("sw must be [C, D, Jt] like sa")
    out = torch.empty((Bn, Cn), dtype=torch.float32, device=sa.device)
    r = torch.empty((Bn, Cn, D), dtype=torch.float32, device=sa.device) if raw else None
    ctx.check(lib().fcs_sketch_inner(ctx.handle, D, Jt, Bn, _ptr(sa), Cn, _ptr(sw),
                                     _ptr(bias), _ptr(out), _ptr(r)))
    return (out, r) if raw else out


def fcs_rtpm(ctx: Context, fcsT: torch.Tensor, I: int, J, h, s, init: torch.Tensor,
             n_iter: int, ldh: int = 0):
    """Sketched robust tensor power method (symmetric order len(J)).  init
    [K, L, I] starting vectors.  Returns (lambda [K], U [K, I])."""
    ctx._sync_stream()
    _need(fcsT, torch.float32, "fcsT")
    _need(init, torch.float32, "init")
    ldh = _tables(h, s, ldh)
    K, L, Ii = init.shape
    if Ii != int(I):
        raise ValueError("init must be [K, L, I]")
    _check_sketch(fcsT, J, [int(I)] * len(J), h, s, [init])
    lam = torch.empty(K, dtype=torch.float32, device=fcsT.device)
    U = torch.empty((K, Ii), dtype=torch.float32, device=fcsT.device)
    ctx.check(lib().fcs_rtpm(ctx.handle, len(J), int(I), _arr(C.c_int32, J), fcsT.shape[0],
                             _ptr(fcsT), _ptr(h), _ptr(s), ldh, K, L, int(n_iter),
                             _ptr(init), _ptr(lam), _ptr(U)))
    return lam, U


def fcs_als(ctx: Context, fcsT: torch.Tensor, I, J, h, s, F, n_iter: int, ldh: int = 0):
    """Sketched CP-ALS.  F: list of N tensors [R, I_n] (transposed factors),
    starting values in, unit-norm factors out (in place).  Returns lambda [R]."""
    ctx._sync_stream()
    _need(fcsT, torch.float32, "fcsT")
    ldh = _tables(h, s, ldh)
    for n, f in enumerate(F):
        _need(f, torch.float32, f"F[{n}]")
    R = F[0].shape[0]
    if len(F) != len(I) or any(f.dim() != 2 or f.shape != (R, int(i)) for f, i in zip(F, I)):
        raise ValueError("F must hold one [R, I_n] tensor per mode")
    _check_sketch(fcsT, J, I, h, s, F)
    lam = torch.empty(R, dtype=torch.float32, device=fcsT.device)
    fp = (C.c_void_p * len(F))(*[f.data_ptr() for f in F])
    ctx.check(lib().fcs_als(ctx.handle, len(I), _arr(C.c_int64, I), _arr(C.c_int32, J),
                            fcsT.shape[0], _ptr(fcsT), _ptr(h), _ptr(s), ldh, R, int(n_iter),
                            fp, _ptr(lam)))
    return lam


# ------------------------------------------------------------------ batching
def cp_problem(U, lam, J, h, s, ldh: int = 0, out: torch.Tensor | None = None):
    """Describe one CP-route sketch for the batch calls.  Returns the
    `CpProblem` structure and its output tensor ([D, Jt], allocated here
    unless given).  The caller keeps U, lam, h, s and out alive while any
    plan built from the description may run."""
    ldh = _tables(h, s, ldh)
    if len(U) > 8:
        raise ValueError("order > 8")
    N, R = _check_cp(U, lam, J, h, s, out)
    D = h.shape[0]
    if out is None:
        out = torch.empty((D, jtilde(J)), dtype=torch.float32, device=U[0].device)
    pr = CpProblem()
    pr.N, pr.D, pr.R = N, D, R
    for k in range(N):
        pr.I[k] = U[k].shape[0]
        pr.J[k] = int(J[k])
        pr.U[k] = U[k].data_ptr()
        pr.ldU[k] = U[k].stride(0)
    pr.lam = None if lam is None else lam.data_ptr()
    pr.h, pr.s, pr.ldh = h.data_ptr(), s.data_ptr(), ldh
    pr.out = out.data_ptr()
    return pr, out


def _problem_array(problems):
    arr = (CpProblem * len(problems))()
    for k, pr in enumerate(problems):
        arr[k] = pr
    return arr


class BatchPlan:
    """A batch of CP-route sketches uploaded once (fcs_batch_plan_create);
    `launch()` issues only device work on torch's current stream and may be
    captured into a CUDA graph."""

    def __init__(self, ctx: Context, problems, grain: int = 0, classes=None):
        """classes: None (autotuned or default shapes) or a list of
        (fft_len, thread_mult, items_per_cta[, engine]) per FFT-length class;
        engine 0 = slot FFT, 1 = warp-DIT (default: 1 for P = 8192 and 16384, else 0)."""
        self.ctx = ctx
        self._arr = _problem_array(problems)
        h = C.c_void_p()
        ctx._sync_stream()
        if classes is None:
            ctx.check(lib().fcs_batch_plan_create(ctx.handle, len(problems), self._arr,
                                                  grain, C.byref(h)))
        else:
            def one(c):
                p, t, i = (int(x) for x in c[:3])
                e = int(c[3]) if len(c) > 3 else (1 if p in (8192, 16384) else 0)
                return BatchClassCfg(p, e, t, i, 0)
            cfg = (BatchClassCfg * max(1, len(classes)))(*[one(c) for c in classes])
            ctx.check(lib().fcs_batch_plan_create_cfg(ctx.handle, len(problems), self._arr,
                                                      grain, len(classes), cfg, C.byref(h)))
        self._h = h
        ctx._plans.add(self)

    def config(self):
        """(grain, [(fft_len, thread_mult, items_per_cta, threads, engine), ...])
        the plan was built with, largest FFT first."""
        g, n = C.c_int(0), C.c_int(0)
        buf = (BatchClassCfg * 16)()
        ctx_check = lib().fcs_batch_plan_config(self._h, C.byref(g), 16, buf, C.byref(n))
        if ctx_check != FCS_OK:
            raise FcsError(ctx_check, "fcs_batch_plan_config failed")
        return g.value, [(c.fft_len, c.thread_mult, c.items_per_cta, c.threads, c.engine)
                         for c in buf[:min(16, n.value)]]

    def launch(self):
        self.ctx._sync_stream()
        self.ctx.check(lib().fcs_batch_plan_launch(self.ctx.handle, self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().fcs_batch_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fcs_batch_sketch_cp(ctx: Context, problems, grain: int = 0):
    """One-shot batch of CP-route sketches (plan, launch, wait, release)."""
    ctx._sync_stream()
    arr = _problem_array(problems)
    ctx.check(lib().fcs_batch_sketch_cp(ctx.handle, len(problems), arr, grain))


def fcs_batch_autotune(ctx: Context, problems) -> int:
    """Time the batch for each candidate grain and remember the best for this
    batch shape; returns that grain."""
    ctx._sync_stream()
    arr = _problem_array(problems)
    best = C.c_int(0)
    ctx.check(lib().fcs_batch_autotune(ctx.handle, len(problems), arr, C.byref(best)))
    return best.value


def fcs_batch_plan_create(ctx: Context, problems, grain: int = 0) -> BatchPlan:
    """C-ABI-named alias of BatchPlan(ctx, problems, grain)."""
    return BatchPlan(ctx, problems, grain)


def fcs_batch_plan_create_cfg(ctx: Context, problems, grain: int, classes) -> BatchPlan:
    """C-ABI-named alias of BatchPlan(ctx, problems, grain, classes)."""
    return BatchPlan(ctx, problems, grain, classes)


def fcs_batch_plan_config(plan: BatchPlan):
    """C-ABI-named alias of plan.config()."""
    return plan.config()


def fcs_batch_plan_launch(ctx: Context, plan: BatchPlan):
    """C-ABI-named alias of plan.launch() (ctx must be the plan's context)."""
    if plan.ctx is not ctx:
        raise ValueError("plan belongs to another context")
    plan.launch()


def fcs_batch_plan_destroy(plan: BatchPlan):
    """C-ABI-named alias of plan.close()."""
    plan.close()


# ------------------------------------------------------------------ serving
class FcsServer:
    """The request server (fcs_server_*).  Requests carry host numpy buffers;
    this object keeps them alive until the request finishes."""

    def __init__(self, device: int = 0, streams: int = 4, max_inflight: int = 64,
                 max_batch: int = 32, arena_bytes: int = 2 << 30,
                 staging_bytes: int = 512 << 20, workspace_bytes: int | None = None):
        cfg = ServerConfig(device, streams, max_inflight, max_batch, arena_bytes,
                           staging_bytes,
                           C.c_size_t(-1).value if workspace_bytes is None else workspace_bytes)
        h = C.c_void_p()
        rc = lib().fcs_server_create(C.byref(cfg), C.byref(h))
        if rc != FCS_OK:
            raise FcsError(rc, "fcs_server_create failed")
        self._h = h
        self._keep = {}

    def _submit(self, req, keep):
        t = C.c_int64()
        rc = lib().fcs_server_submit(self._h, C.byref(req), C.byref(t))
        if rc != FCS_OK:
            raise FcsError(rc, "fcs_server_submit rejected the request")
        self._keep[t.value] = keep
        return t.value

    def submit_cp(self, U, lam, J, D: int, seed: int, out=None, keep_resident=False):
        """Sketch the CP tensor [[lam; U_1..U_N]] (host float32 arrays) into
        `out` ([D, Jt] float32, host) and/or keep it resident."""
        import numpy as np
        U = [np.ascontiguousarray(u, dtype=np.float32) for u in U]
        lam = None if lam is None else np.ascontiguousarray(lam, dtype=np.float32)
        r = Request()
        r.kind, r.N, r.D, r.R, r.seed = FCS_REQ_CP, len(U), D, U[0].shape[1], seed
        for k, u in enumerate(U):
            r.I[k], r.J[k] = u.shape[0], int(J[k])
            r.host_U[k] = u.ctypes.data
        r.host_lambda = None if lam is None else lam.ctypes.data
        r.host_out = None if out is None else out.ctypes.data
        r.keep_resident = 1 if keep_resident else 0
        return self._submit(r, (U, lam, out))

    def submit_contract(self, sketch_id: int, I, J, kind: int, vecs, result,
                        free_mode: int = 0):
        """Contract host vectors ([B, I_n] float32) with resident sketch
        `sketch_id`; the median over sketches lands in `result`."""
        import numpy as np
        vv = [None if v is None else np.ascontiguousarray(v, dtype=np.float32) for v in vecs]
        r = Request()
        r.kind, r.N, r.sketch_id = FCS_REQ_CONTRACT, len(I), sketch_id
        r.contract_kind, r.free_mode = kind, free_mode
        r.B = next(v for v in vv if v is not None).shape[0]
        for k in range(len(I)):
            r.I[k], r.J[k] = int(I[k]), int(J[k])
            r.host_vecs[k] = None if vv[k] is None else vv[k].ctypes.data
        r.host_result = result.ctypes.data
        return self._submit(r, (vv, result))

    def poll(self, ticket: int) -> Result:
        res = Result()
        lib().fcs_server_poll(self._h, ticket, C.byref(res))
        if res.state >= 2:
            self._keep.pop(ticket, None)
        return res

    def wait(self, ticket: int, timeout_s: float = 60.0) -> Result:
        res = Result()
        rc = lib().fcs_server_wait(self._h, ticket, timeout_s, C.byref(res))
        if rc not in (FCS_OK, FCS_ETIMEOUT):
            raise FcsError(rc, "fcs_server_wait failed")
        if res.state >= 2:
            self._keep.pop(ticket, None)
        return res

    def cancel(self, ticket: int) -> int:
        return lib().fcs_server_cancel(self._h, ticket)

    def release(self, sketch_id: int) -> int:
        return lib().fcs_server_release(self._h, sketch_id)

    def stats(self) -> Stats:
        st = Stats()
        lib().fcs_server_stats(self._h, C.byref(st))
        return st

    def reset_stats(self):
        lib().fcs_server_reset_stats(self._h)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().fcs_server_destroy(self._h)
            self._h = C.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fcs_server_create(**kw) -> FcsServer:
    """C-ABI-named alias of FcsServer(**kw)."""
    return FcsServer(**kw)


def fcs_server_destroy(server: FcsServer):
    server.close()


def fcs_server_submit(server: FcsServer, kind: int, **kw) -> int:
    """Submit through the C entry point: kind FCS_REQ_CP takes the keywords of
    FcsServer.submit_cp, FCS_REQ_CONTRACT those of submit_contract."""
    return server.submit_cp(**kw) if kind == FCS_REQ_CP else server.submit_contract(**kw)


def fcs_server_poll(server: FcsServer, ticket: int) -> Result:
    return server.poll(ticket)


def fcs_server_wait(server: FcsServer, ticket: int, timeout_s: float = 60.0) -> Result:
    return server.wait(ticket, timeout_s)


def fcs_server_cancel(server: FcsServer, ticket: int) -> int:
    return server.cancel(ticket)


def fcs_server_release(server: FcsServer, sketch_id: int) -> int:
    return server.release(sketch_id)


def fcs_server_stats(server: FcsServer) -> Stats:
    return server.stats()


def fcs_server_reset_stats(server: FcsServer):
    server.reset_stats()
