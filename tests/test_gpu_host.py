"""fcs_sketch_cp_seeded (hash tables of a seed written by the factor
transpose launch, then the sketch) and fcs_sketch_cp_host (the same from
host factors to a host sketch: copies, tables, sketch and read-back queued by
the library) must equal fcs_make_hashes + fcs_sketch_cp on device copies of
the same inputs -- the tables bit for bit -- and the oracle.  Needs a GPU."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import synth
from gpu_common import assert_sketch_close, cuda, host

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


def _device_ref(fcs, ctx, U, lam, J, D, seed):
    I = [u.shape[0] for u in U]
    h, s = fcs.fcs_make_hashes(ctx, seed, I, J, D)
    Ug = [torch.from_numpy(np.ascontiguousarray(u)).cuda() for u in U]
    lg = None if lam is None else torch.from_numpy(lam).cuda()
    return host(fcs.fcs_sketch_cp(ctx, Ug, lg, J, h, s))


@pytest.mark.parametrize("I,J,R,D", [
    ([1000, 1000, 1000], [5000] * 3, 100, 10),        # the benchmark problem, P = 16384
    ([40, 50, 30], [20, 30, 25], 3, 2),               # P = 128
    ([120, 100, 90], [9000, 8000, 7000], 6, 2),       # P = 32768
])
def test_host_block_equals_device_call(fcs, ctx, orc, I, J, R, D):
    """Factors and lambda as views of one pinned host block (one merged copy)."""
    U, lam = synth.cp_factors(61, I, R)
    parts = [u.reshape(-1) for u in U] + [lam]
    block = torch.from_numpy(np.concatenate(parts)).pin_memory()
    offs = np.cumsum([0] + [p.size for p in parts])
    Uh = [block[offs[n]:offs[n + 1]].view(I[n], R) for n in range(len(I))]
    lh = block[offs[-2]:offs[-1]]
    out = fcs.fcs_sketch_cp_host(ctx, Uh, lh, J, D, seed=62)
    torch.cuda.synchronize()
    ref = _device_ref(fcs, ctx, U, lam, J, D, 62)
    assert_sketch_close(out.numpy(), ref.astype(np.float64))
    if np.prod(I) * R <= 1e6:
        ho, so = orc.make_hashes(62, I, J, D)
        want = orc.fcs_cp([u.astype(np.float64) for u in U], lam.astype(np.float64), J, ho, so)
        assert_sketch_close(out.numpy(), want)


def test_host_pageable_strided_and_no_lambda(fcs, ctx):
    """Pageable host memory, a factor that is a column slice of a wider
    matrix (leading dimension > R), no lambda; two calls in a row reuse the
    staging buffer."""
    I, J, R, D = [300, 200, 250], [700, 900, 500], 12, 4
    U, _ = synth.cp_factors(71, I, R)
    wide = synth.gaussian(72, (I[1], R + 9))
    U[1] = wide[:, 3:3 + R]                          # leading dimension R + 9
    Uh = [torch.from_numpy(u) for u in U]
    assert Uh[1].stride(0) == R + 9
    for seed in (73, 74):
        out = fcs.fcs_sketch_cp_host(ctx, Uh, None, J, D, seed=seed)
        torch.cuda.synchronize()
        ref = _device_ref(fcs, ctx, U, None, J, D, seed)
        assert_sketch_close(out.numpy(), ref.astype(np.float64))


@pytest.mark.parametrize("I,J,R,D", [
    ([1000, 1000, 1000], [5000] * 3, 100, 10),        # the benchmark problem, P = 16384
    ([100, 120, 90], [3000, 2000, 1000], 7, 3),       # P = 8192
    ([300, 200, 250], [700, 900, 500], 12, 4),        # P = 4096
    ([40, 50], [20, 30], 3, 2),                       # P = 64
    ([7, 5, 6, 4, 3], [9, 8, 7, 6, 5], 2, 16),        # order 5, D = 16, P = 32
    ([120, 100, 90], [9000, 8000, 7000], 6, 2),       # P = 32768: tables by their own launch
    ([3000], [6000], 4, 1),                           # one mode, one sketch, P = 8192
    ([6, 5, 4, 3, 4, 5, 6, 3], [7, 6, 5, 4, 5, 6, 7, 4], 2, 3),   # order 8, P = 64
    ([300, 200, 250], [100000, 90000, 80000], 2, 2),  # P = 2^18: two-pass route (no oracle sketch)
])
def test_seeded_equals_tables_then_sketch(fcs, ctx, orc, I, J, R, D):
    U, lam = synth.cp_factors(81, I, R)
    Ug, lg = [cuda(u) for u in U], cuda(lam)
    out, h, s = fcs.fcs_sketch_cp_seeded(ctx, Ug, lg, J, D, seed=82)
    h2, s2 = fcs.fcs_make_hashes(ctx, 82, I, J, D)
    torch.cuda.synchronize()
    assert torch.equal(h, h2) and torch.equal(s, s2)
    ref = host(fcs.fcs_sketch_cp(ctx, Ug, lg, J, h2, s2))
    assert_sketch_close(host(out), ref.astype(np.float64))
    if sum(I) * D <= 20000:
        ho, so = orc.make_hashes(82, I, J, D)
        assert np.array_equal(host(h), ho) and np.array_equal(host(s), so)
    if np.prod(I) * R <= 1e6:
        ho, so = orc.make_hashes(82, I, J, D)
        want = orc.fcs_cp([u.astype(np.float64) for u in U], lam.astype(np.float64), J, ho, so)
        assert_sketch_close(host(out), want)


def test_seeded_given_buffers_strided_no_lambda(fcs, ctx):
    """Caller-given table and output buffers (reused by a second seed), a
    factor that is a column slice of a wider matrix, no lambda; tables of the
    wrong shape are refused before any launch."""
    I, J, R, D = [300, 200, 250], [5000, 4000, 3000], 12, 5          # P = 16384
    U, _ = synth.cp_factors(83, I, R)
    Ug = [cuda(u) for u in U]
    Ug[1] = cuda(synth.gaussian(84, (I[1], R + 5)))[:, 2:2 + R]   # a column slice on the device
    assert Ug[1].stride(0) == R + 5
    tot = sum(I)
    h = torch.empty((D, tot), dtype=torch.int32, device="cuda")
    s = torch.empty((D, tot), dtype=torch.int8, device="cuda")
    out = torch.empty((D, sum(J) - 2), dtype=torch.float32, device="cuda")
    for seed in (85, 86):
        o, hh, ss = fcs.fcs_sketch_cp_seeded(ctx, Ug, None, J, D, seed, out=out, h=h, s=s)
        assert o.data_ptr() == out.data_ptr() and hh.data_ptr() == h.data_ptr()
        h2, s2 = fcs.fcs_make_hashes(ctx, seed, I, J, D)
        ref = host(fcs.fcs_sketch_cp(ctx, Ug, None, J, h2, s2))
        torch.cuda.synchronize()
        assert torch.equal(h, h2) and torch.equal(s, s2)
        assert_sketch_close(host(out), ref.astype(np.float64))
    with pytest.raises(ValueError):
        fcs.fcs_sketch_cp_seeded(ctx, Ug, None, J, D, 87, h=h[:, :tot - 1].contiguous(), s=s)
