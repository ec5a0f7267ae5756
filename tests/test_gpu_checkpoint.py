"""Deterministic overlap sums and checkpoint / resume of a RAAR reconstruction
(Sec. 2.2 iteration; the state of a step is the frame state c, the images
psi_y and psi, the probe and the probe that formed the iterate).

With sharp_plan_set_deterministic the overlap sums are gathered per image tile
in a fixed order instead of scattered with atomics, so two runs give
bit-identical iterates, objects and probes; they agree with the default
(atomic) path and the FP64 oracle within the FP32 bounds.  A run checkpointed
after three steps and resumed in a new plan ends bit-identical to an
uninterrupted run; the metrics, added up per block over whichever frames the
block took, agree to FP32 rounding.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from tests.gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu


def _lib():
    import paper_1602_01448_gb300 as S
    return S


def _scan(m, seed):
    rng = np.random.default_rng(seed)
    side, step = 3, m // 4
    n = (side - 1) * step + m + 23
    shape = (n, n)
    obj = synth.random_object(shape, rng)
    w = synth.gaussian_probe(m, m / 6.0, rng)
    pos = synth.raster_positions(side, side, step, m, shape, rng, jitter=1)
    inten = O.forward_amplitudes(obj, w, pos) ** 2
    a = np.sqrt(synth.poisson_intensities(inten, 1e6, rng)).astype(np.float32).astype(np.float64)
    psi0 = synth.random_object(shape, rng, phase_sigma=1.0)
    w0 = synth.perturb_probe(w, rng, 0.1)
    return pos, shape, a, psi0, w0


def _plan(S, pos, m, shape, psi0, w0, deterministic, precision="fp32"):
    p = S.Plan(pos, m, shape, beta=0.75, probe_every=2, residual_every=3, precision=precision)
    p.set_deterministic(deterministic)
    p.raar_init(dev(psi0), dev(w0))
    return p


def _state(p):
    return [t.clone() for t in (p.c, p.psi_y, p.psi, p.probe)]


@pytest.mark.parametrize("m,prec", [(64, "fp32"), (128, "fp32"), (256, "fp32"), (128, "bf16x3"), (256, "fp16s")])
def test_deterministic_steps_are_bit_identical_and_match(m, prec):
    S = _lib()
    pos, shape, a, psi0, w0 = _scan(m, 100 + m)
    ta = dev(a, torch.float32)
    n_steps = 5
    runs = []
    for det in (True, True, False):
        p = _plan(S, pos, m, shape, psi0, w0, det, prec)
        for _ in range(n_steps):
            p.raar_step(ta)
        p.status()
        runs.append(_state(p))
    for x, y in zip(runs[0], runs[1]):
        assert torch.equal(x, y)
    tol = {"fp32": 1e-5, "bf16x3": 5e-5, "fp16s": 3e-3}[prec]
    for x, y in zip(runs[0], runs[2]):       # atomic path: same arithmetic, another summation order
        assert rel_l2(host(x), host(y)) < 2 * n_steps * tol
    ref = O.raar_reconstruct(a, pos, shape, w0, psi0, n_steps, beta=0.75, probe_every=2)
    D = O.illumination(ref["w"], pos, shape)
    vis = D > 1e-3 * D.max()
    assert rel_l2(host(runs[0][2]), ref["psi"], vis) < 2 * n_steps * tol
    assert rel_l2(host(runs[0][3]), ref["w"]) < 2 * n_steps * tol


@pytest.mark.parametrize("m", [128, 256])
def test_checkpoint_resume_is_bit_identical(m):
    S = _lib()
    pos, shape, a, psi0, w0 = _scan(m, 200 + m)
    ta = dev(a, torch.float32)
    straight = _plan(S, pos, m, shape, psi0, w0, True)
    mets = []
    for _ in range(6):
        mets.append(host(straight.raar_step(ta)).real.copy())
    first = _plan(S, pos, m, shape, psi0, w0, True)
    for _ in range(3):                        # step 2 updated the probe; step 3 formed B' from it
        first.raar_step(ta)
    ckpt = first.checkpoint()
    first.close()
    resumed = S.Plan(pos, m, shape, beta=0.75, probe_every=2, residual_every=3)
    resumed.set_deterministic(True)
    resumed.restore(ckpt)
    for k in range(3):
        met = host(resumed.raar_step(ta)).real
        ref = mets[3 + k]
        # eps_a: per-block FP32 partial sums over the frames each block took
        assert abs(met[0] - ref[0]) <= 1e-6 * ref[0]
    resumed.status()
    for x, y in zip(_state(straight), _state(resumed)):
        assert torch.equal(x, y)


def test_checkpoint_arguments_and_batch_rejects_deterministic_plans():
    S = _lib()
    pos, shape, a, psi0, w0 = _scan(64, 300)
    p = S.Plan(pos, 64, shape)
    pc = torch.empty((64, 64), dtype=torch.complex64, device="cuda")
    import ctypes
    info = (ctypes.c_int * 4)(-1, 1, 0, 0)
    with pytest.raises(S.SharpError):
        S._check(S._C["sharp_raar_restore"](p.handle, pc.data_ptr(), pc.data_ptr(), info,
                                            torch.cuda.current_stream().cuda_stream))
    with pytest.raises(S.SharpError):         # checkpoint before sharp_raar_init
        S._check(S._C["sharp_raar_checkpoint"](p.handle, pc.data_ptr(), pc.data_ptr(), info,
                                               torch.cuda.current_stream().cuda_stream))
    p.set_deterministic(True)
    p.raar_init(dev(psi0), dev(w0))
    with pytest.raises(S.SharpError):
        S.Batch([p], [dev(a, torch.float32)])
