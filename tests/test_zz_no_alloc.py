"""The allocation-free data projection (sharp_fourier_project_noalloc) gives
the same frames and residual as the plan-based sharp_fourier_project and as
the FP64 oracle's P_a (Eq. 7), and allocates no device memory.

It exists for callers that cannot allocate device memory while they run, for
example hosts that own every device allocation or real-time loops that must
not wait on the allocator; its scratch is a fixed library-owned device array.
This file is named so that pytest collects it last; it also passes when run
on its own.
"""
import numpy as np
import pytest
import torch

import oracle as O
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
        # and directly against the oracle's P_a and ||P_a z - z||^2
        z_h = z.cpu().numpy().astype(np.complex128)
        a_h = amp.cpu().numpy().astype(np.float64)
        p_o = O.data_project(z_h, a_h)
        got = out.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got - p_o) < TOL * np.linalg.norm(p_o), call
        r_o = O.norm(p_o - z_h) ** 2
        assert abs(r.item() - r_o) < TOL * r_o, call


@pytest.mark.parametrize("m", [64, 128])
def test_noalloc_call_leaves_device_memory_unchanged(m):
    import paper_1602_01448_gb300 as S
    K = 19
    z = torch.as_tensor(synth.random_frames(K, m, 7)).to(torch.complex64).cuda()
    amp = torch.as_tensor(synth.random_amplitudes(K, m, 8)).to(torch.float32).cuda()
    out = torch.empty_like(z)
    r = torch.zeros(1, dtype=torch.float64, device="cuda")
    S.sharp_fourier_project_noalloc(z, amp, out, r)      # first call: module load, symbol lookup
    torch.cuda.synchronize()
    first = out.clone()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        S.sharp_fourier_project_noalloc(z, amp, out, r)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert _rel(out, first) < TOL


def test_noalloc_rejects_too_many_frames():
    import paper_1602_01448_gb300 as S
    z = torch.zeros((1, 64, 64), dtype=torch.complex64, device="cuda")
    amp = torch.zeros((1, 64, 64), dtype=torch.float32, device="cuda")
    rc = S._C["sharp_fourier_project_noalloc"](z.data_ptr(), amp.data_ptr(), z.data_ptr(), None,
                                               65537, 64, torch.cuda.current_stream().cuda_stream)
    assert rc == 1
    assert b"SHARP_NOALLOC_MAX_FRAMES" in S._C["sharp_last_error"]()
