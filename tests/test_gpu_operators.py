"""GPU parity of the single operators against the FP64 oracle (Eqs. 1, 5, 7-10,
14): relative L2 <= 1e-5 in FP32, at sizes that span several tiles and a
ragged tail, with and without periodic wrap."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from tests.gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _lib():
    import paper_1602_01448_gb300 as S
    return S


def _case(m, wrap, seed=0):
    """A few frames over a ragged object (not a multiple of the 32-px tile),
    including frames at both edges (and across them with wrap)."""
    rng = np.random.default_rng(seed)
    ny, nx = m + 75, m + 101
    if wrap:
        pos = np.array([[0, 0], [ny - m // 2, nx - 7], [5, nx - m + 40], [ny - 3, 11], [30, 40]], np.int32)
    else:
        pos = np.array([[0, 0], [ny - m, nx - m], [0, nx - m], [ny - m, 0], [37, 51], [12, 80]], np.int32)
    obj = synth.random_object((ny, nx), rng)
    w = synth.gaussian_probe(m, m / 6.0, rng)
    return pos, obj, w, (ny, nx)


@pytest.mark.parametrize("m", [64, 128, 256])
@pytest.mark.parametrize("wrap", [False, True])
def test_split_forward_model_and_overlap(m, wrap):
    S = _lib()
    pos, obj, w, shape = _case(m, wrap)
    plan = S.Plan(pos, m, shape, wrap=wrap)
    z = host(plan.q_gather(dev(obj), dev(w)))
    assert rel_l2(z, O.split(obj, w, pos, wrap)) < 1e-6
    amp = host(plan.forward_amplitudes(dev(obj), dev(w)))
    assert rel_l2(amp, O.forward_amplitudes(obj, w, pos, wrap)) < TOL
    zz = synth.random_frames(len(pos), m, 3)
    psi, zo = plan.overlap_project(dev(w), dev(zz))
    ref_psi = O.object_update(zz, w, pos, shape, wrap)
    assert rel_l2(host(psi), ref_psi) < TOL
    assert rel_l2(host(zo), O.split(ref_psi, w, pos, wrap)) < TOL


@pytest.mark.parametrize("m", [64, 128, 256])
def test_fourier_projection(m):
    S = _lib()
    pos, obj, w, shape = _case(m, False)
    plan = S.Plan(pos, m, shape)
    z = synth.random_frames(len(pos), m, 4)
    a = synth.random_amplitudes(len(pos), m, 5)
    a[1] = 0.0                                   # an all-zero frame of data
    z[2] = 0.0                                   # |Fz| = 0 everywhere: phase-1 reading
    out, r = plan.fourier_project(dev(z), dev(a, torch.float32))
    ref = O.data_project(z, a.astype(np.float32).astype(np.float64))
    assert rel_l2(host(out), ref) < TOL
    assert abs(r.item() - O.norm(ref - z) ** 2) < 1e-5 * O.norm(ref - z) ** 2
    # in place
    zt = dev(z)
    S.sharp_fourier_project(plan.handle, zt, dev(a, torch.float32), zt)
    assert rel_l2(host(zt), ref) < TOL


@pytest.mark.parametrize("m", [64, 128, 256])
@pytest.mark.parametrize("wrap", [False, True])
def test_probe_update(m, wrap):
    S = _lib()
    pos, obj, w, shape = _case(m, wrap, seed=2)
    plan = S.Plan(pos, m, shape, wrap=wrap)
    z = synth.random_frames(len(pos), m, 6)
    got = host(plan.probe_update(dev(obj), dev(z), dev(w)))
    ref = O.probe_update(z, obj, pos, w, wrap)
    assert rel_l2(got, ref) < TOL


def test_probe_update_fixed_point_at_truth():
    S = _lib()
    pos, obj, w, shape = _case(64, False, seed=3)
    plan = S.Plan(pos, 64, shape)
    z = plan.q_gather(dev(obj), dev(w))
    got = host(plan.probe_update(dev(obj), z, dev(w) * 0))
    assert rel_l2(got, w) < 1e-6


@pytest.mark.parametrize("m", [64, 128, 256])
def test_amp_loss_and_adjoint(m):
    S = _lib()
    pos, obj, w, shape = _case(m, False, seed=4)
    rng = np.random.default_rng(9)
    a = O.forward_amplitudes(obj, w, pos) * (1 + 0.1 * rng.standard_normal((len(pos), m, m)))
    a = np.abs(a).astype(np.float32).astype(np.float64)
    psi = obj * (1 + 0.05 * rng.standard_normal(shape))
    plan = S.Plan(pos, m, shape)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    S.sharp_amp_loss(plan.handle, dev(psi), dev(w), dev(a, torch.float32), loss)
    ref = O.amp_loss(psi, w, a, pos)
    assert abs(loss.item() - ref) < 1e-5 * ref
    g_obj = torch.empty(shape, dtype=torch.complex64, device="cuda")
    g_w = torch.empty((m, m), dtype=torch.complex64, device="cuda")
    S.sharp_amp_loss_backward(plan.handle, dev(psi), dev(w), dev(a, torch.float32), 1.0, g_obj, g_w)
    rg_obj, rg_w = O.amp_loss_grad(psi, w, a, pos)
    assert rel_l2(host(g_obj), rg_obj) < TOL
    assert rel_l2(host(g_w), rg_w) < TOL


def test_autograd_function_matches_oracle_gradient():
    S = _lib()
    pos, obj, w, shape = _case(64, False, seed=5)
    rng = np.random.default_rng(10)
    a = np.abs(O.forward_amplitudes(obj, w, pos) + 0.05).astype(np.float32).astype(np.float64)
    psi = obj * (1 + 0.05 * rng.standard_normal(shape))
    plan = S.Plan(pos, 64, shape)
    tpsi = dev(psi).requires_grad_(True)
    tw = dev(w).requires_grad_(True)
    loss = S.amp_loss(plan, tpsi, tw, dev(a, torch.float32))
    (3.0 * loss).backward()
    rg_obj, rg_w = O.amp_loss_grad(psi, w, a, pos)
    assert rel_l2(host(tpsi.grad), 6.0 * rg_obj) < TOL
    assert rel_l2(host(tw.grad), 6.0 * rg_w) < TOL


def test_solution_error_matches_oracle():
    S = _lib()
    pos, obj, w, shape = _case(64, False, seed=6)
    rng = np.random.default_rng(11)
    psi = obj * np.exp(0.4j) + 1e-3 * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    plan = S.Plan(pos, 64, shape)
    out = host(plan.solution_error(dev(psi), dev(obj), dev(w))).real
    psi32 = psi.astype(np.complex64).astype(np.complex128)
    obj32 = obj.astype(np.complex64).astype(np.complex128)
    assert abs(out[0] - O.eps_0_object(psi32, obj32, w, pos, shape)) < 1e-4 * out[0]
    assert abs(out[1] - O.object_nrmse(psi32, obj32, w, pos, shape)) < 1e-4 * out[1]


def test_bad_arguments_are_rejected():
    S = _lib()
    pos = dev(np.array([[0, 0], [300, 0]], np.int32))
    with pytest.raises(S.SharpError) as e:
        S.sharp_plan_create(2, 64, 256, 256, pos)
    assert e.value.code == 1
    with pytest.raises(S.SharpError) as e:
        S.sharp_plan_create(2, 96, 512, 512, dev(np.zeros((2, 2), np.int32)))
    assert e.value.code == 2
    plan = S.Plan(np.zeros((1, 2), np.int32), 64, (64, 64))
    with pytest.raises(S.SharpError) as e:
        S.sharp_raar_step(plan.handle, dev(np.zeros((1, 64, 64), np.complex64)),
                          dev(np.zeros((64, 64), np.complex64)), dev(np.zeros((64, 64), np.complex64)),
                          None, dev(np.zeros((1, 64, 64), np.float32)), None, 1)
    assert e.value.code == 5
