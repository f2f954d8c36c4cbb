"""fcs_sketch_cp_noalloc: the CP-route sketch for callers that may not
allocate device memory (a host framework owning all device memory, loops that
cannot afford cudaMalloc's implicit synchronisation, fixed memory budgets).
Its scratch is a fixed device array inside the library.

Called here through the C ABI with ctypes and compared with the ordinary
fcs_sketch_cp on the same inputs, on two calls in a row (the shared scratch
keeps the previous call's contents, so the second call checks that the entry
point clears it).  This file is collected last."""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest
import torch

import synth
from gpu_common import SKETCH_RTOL, rel_l2

pytestmark = pytest.mark.gpu


def _call_noalloc(fcs, U, lam, J, h, s, out):
    L = fcs.lib()
    N, R = len(U), U[0].shape[1]
    ptrs = (C.c_void_p * N)(*[u.data_ptr() for u in U])
    err = C.create_string_buffer(512)
    stream = torch.cuda.current_stream().cuda_stream
    rc = L.fcs_sketch_cp_noalloc(
        C.c_void_p(stream), N, fcs._arr(C.c_int64, [u.shape[0] for u in U]),
        fcs._arr(C.c_int32, J), R, h.shape[0], ptrs,
        fcs._arr(C.c_int64, [u.stride(0) for u in U]),
        None if lam is None else C.c_void_p(lam.data_ptr()),
        C.c_void_p(h.data_ptr()), C.c_void_p(s.data_ptr()), 0,
        C.c_void_p(out.data_ptr()), err, 512)
    return rc, err.value.decode()


def test_noalloc_matches_sketch_cp_twice():
    import paper_2106_13062_gb300 as fcs
    fcs.build()
    ctx = fcs.Context()
    cases = [([200, 150, 300], [700, 900, 500], 17, 4, 5),     # P = 4096
             ([1000, 1000, 1000], [5000] * 3, 100, 10, 6)]     # P = 16384
    for I, J, R, D, seed in cases:
        U, lam = synth.cp_factors(seed, I, R)
        Ug = [torch.from_numpy(u).cuda() for u in U]
        lamg = torch.from_numpy(lam).cuda()
        h, s = fcs.fcs_make_hashes(ctx, seed, I, J, D)
        ref = fcs.fcs_sketch_cp(ctx, Ug, lamg, J, h, s)
        out = torch.full_like(ref, float("nan"))
        rc, msg = _call_noalloc(fcs, Ug, lamg, J, h, s, out)
        assert rc == 0, msg
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(a).all()
        for d in range(D):
            assert rel_l2(a[d], b[d]) <= SKETCH_RTOL
    ctx.close()


def test_noalloc_rejects_oversized_problem():
    import paper_2106_13062_gb300 as fcs
    fcs.build()
    I, J, R = [4096, 4096, 4096], [4000, 4000, 4000], 200       # 9.4 MiB of factors
    U = [torch.zeros((i, R), device="cuda") for i in I]
    h = torch.zeros((1, sum(I)), dtype=torch.int32, device="cuda")
    s = torch.ones((1, sum(I)), dtype=torch.int8, device="cuda")
    out = torch.zeros((1, sum(J) - 2), device="cuda")
    rc, msg = _call_noalloc(fcs, U, None, J, h, s, out)
    assert rc == fcs.FCS_ENOMEM_BUDGET
    assert "scratch" in msg


def test_noalloc_wrapper_and_spectrum_cache(orc):
    """Through the Python wrapper: the result equals fcs_sketch_cp's; a buffer
    re-sketched by the no-alloc call while a context caches its spectra is
    read correctly by later contractions once fcs_forget has dropped the
    entry (the entry point has no context, so it cannot drop it itself)."""
    import paper_2106_13062_gb300 as fcs
    fcs.build()
    ctx = fcs.Context()
    fcs.fcs_cache_spectra(ctx, True)
    I, J, R, D = [120, 90, 70], [300, 250, 200], 6, 3
    h, s = fcs.fcs_make_hashes(ctx, 41, I, J, D)
    Ua, lama = synth.cp_factors(42, I, R)
    Ub, lamb = synth.cp_factors(43, I, R)
    cu = lambda a: torch.from_numpy(a).cuda()  # noqa: E731
    buf = fcs.fcs_sketch_cp(ctx, [cu(u) for u in Ua], cu(lama), J, h, s)
    v = [cu(synth.unit_vectors(44 + n, 2, I[n])) for n in range(3)]
    vecs = [None, v[1], v[2]]
    fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_FREE, buf, vecs, I, J, h, s)   # caches buf
    ref = fcs.fcs_sketch_cp(ctx, [cu(u) for u in Ub], cu(lamb), J, h, s)
    fcs.fcs_sketch_cp_noalloc([cu(u) for u in Ub], cu(lamb), J, h, s, out=buf)
    torch.cuda.synchronize()
    for d in range(D):
        assert rel_l2(buf[d].cpu().numpy(), ref[d].cpu().numpy()) <= SKETCH_RTOL
    fcs.fcs_forget(ctx, buf)
    got = fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_FREE, buf, vecs, I, J, h, s)
    want = fcs.fcs_contract(ctx, fcs.FCS_CONTRACT_FREE, buf.clone(), vecs, I, J, h, s)
    torch.cuda.synchronize()
    assert rel_l2(got.cpu().numpy(), want.cpu().numpy()) <= 1e-6
    with pytest.raises(ValueError):
        fcs.fcs_sketch_cp_noalloc([cu(u) for u in Ub], cu(lamb), J, h, s, out=buf[:, :-1])
    ctx.close()
