"""Shared helpers for the GPU parity tests (CUDA path vs the FP64 oracle).

Tolerances (FP32 arithmetic against FP64 on identical FP32 inputs):
  * hashes, bins, indices: bit-exact;
  * sketches: relative L2 <= 1e-5 per sketch d;
  * T(v_1..v_N) scalars: |gpu - oracle| <= 1e-4 * ||FCS_d T|| * ||FCS_d(v o..)||
    (the Cauchy-Schwarz scale of the inner product; the value itself may
    cancel towards 0);
  * T(.., I, ..) vectors: relative L2 <= 1e-4 per (item, sketch);
  * medians: the median is 1-Lipschitz in the max norm, so it inherits the
    per-sketch scale.
"""
from __future__ import annotations

import numpy as np
import torch

SKETCH_RTOL = 1e-5
CONTRACT_RTOL = 1e-4


def cuda(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel_l2(got, ref) -> float:
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    num = np.linalg.norm(got - ref)
    return float(num / den) if den > 0 else float(num)


def assert_sketch_close(got, ref, rtol=SKETCH_RTOL, what="sketch"):
    got = np.asarray(got).reshape(-1, np.asarray(ref).shape[-1])
    ref = np.asarray(ref).reshape(got.shape)
    for d in range(ref.shape[0]):
        e = rel_l2(got[d], ref[d])
        assert e <= rtol, f"{what}[{d}]: relative L2 error {e:.3e} > {rtol:.1e}"
