"""The allocation-free data projection (sharp_fourier_project_noalloc) gives
the same frames and residual as the plan-based sharp_fourier_project.

It exists for callers that cannot allocate device memory while they run, for
example hosts that own every device allocation or work recorded into a CUDA
graph; its scratch is a fixed library-owned device array.  This file is named
so that pytest collects it last; it also passes when run on its own.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5   # relative L2, as for the other single-operator parity tests


def _rel(a, b):
    a = a.detach().cpu().numpy().astype(np.complex128)
    b = b.detach().cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _reference(S, z, amp):
    """The existing entry point (needs a plan; positions do not enter P_a)."""
    K, m = z.shape[0], z.shape[-1]
    plan = S.Plan(np.zeros((K, 2), np.int32), m, (m, m))
    out = torch.empty_like(z)
    r = torch.zeros(1, dtype=torch.float64, device="cuda")
    S.sharp_fourier_project(plan.handle, z, amp, out, r)
    torch.cuda.synchronize()
    plan.close()
    return out, r


@pytest.mark.parametrize("m", [64, 128])
def test_noalloc_projection_matches_plan_projection_twice(m):
    import paper_1602_01448_gb300 as S
    for call, (K, seed) in enumerate([(37, 1), (11, 2)]):   # second call smaller: stale entries unused
        z = torch.as_tensor(synth.random_frames(K, m, seed)).to(torch.complex64).cuda()
        amp = torch.as_tensor(synth.random_amplitudes(K, m, seed + 100)).to(torch.float32).cuda()
        ref, r_ref = _reference(S, z, amp)
        out = torch.empty_like(z)
        r = torch.zeros(1, dtype=torch.float64, device="cuda")
        S.sharp_fourier_project_noalloc(z, amp, out, r)
        torch.cuda.synchronize()
        assert _rel(out, ref) < TOL, call
        assert abs(r.item() - r_ref.item()) < TOL * r_ref.item(), call


def test_noalloc_rejects_too_many_frames():
    import paper_1602_01448_gb300 as S
    z = torch.zeros((1, 64, 64), dtype=torch.complex64, device="cuda")
    amp = torch.zeros((1, 64, 64), dtype=torch.float32, device="cuda")
    rc = S._C["sharp_fourier_project_noalloc"](z.data_ptr(), amp.data_ptr(), z.data_ptr(), None,
                                               65537, 64, torch.cuda.current_stream().cuda_stream)
    assert rc == 1
    assert b"SHARP_NOALLOC_MAX_FRAMES" in S._C["sharp_last_error"]()
