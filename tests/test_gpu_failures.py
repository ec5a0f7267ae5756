"""Failure detection of the frame passes, exercised without faulting the GPU.

* A bounded wait that runs out: the plan's wait limit set to zero polls makes
  every first wait of a frame pass (bulk copy of the frame state, tensor-core
  MMA completion, at 128^2 and in the 256^2 tensor-core passes) give up at
  once.  The kernel then drains its own copies and
  MMAs in flight with the full limit, releases its tensor memory and returns;
  sharp_plan_status reports SHARP_ERR_TIMEOUT once, and the plan, restarted
  with the default limit, matches the FP64 oracle again (Sec. 2.2 steps).
* Invalid data: a measured amplitude that is NaN (Eq. 1 gives a = |F z| >= 0)
  and a probe with no illumination at all (Q*Q = 0 everywhere, Eq. 9) raise
  SHARP_ERR_INVALID_ARG through sharp_plan_status.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from tests.gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu

TIMEOUT, INVALID = 4, 1
# object error after two steps: FP32 operators (1e-5 per step), the
# tensor-core modes at their projection bounds (two per step)
PSI_TOL = {"fp32": 2e-5, "bf16x3": 4 * 5e-5, "fp16s": 4 * 3e-3}
MET_TOL = {"fp32": 1e-4, "bf16x3": 2e-3, "fp16s": 3e-2}


def _lib():
    import paper_1602_01448_gb300 as S
    return S


def _scan(m, seed):
    rng = np.random.default_rng(seed)
    side, step = 3, m // 4
    n = (side - 1) * step + m + 19
    shape = (n, n)
    obj = synth.random_object(shape, rng)
    w = synth.gaussian_probe(m, m / 6.0, rng)
    pos = synth.raster_positions(side, side, step, m, shape, rng, jitter=1)
    inten = O.forward_amplitudes(obj, w, pos) ** 2
    a = np.sqrt(synth.poisson_intensities(inten, 1e6, rng)).astype(np.float32).astype(np.float64)
    psi0 = synth.random_object(shape, rng, phase_sigma=1.0)
    return w, pos, shape, a, psi0


def _expect(S, plan, code):
    with pytest.raises(S.SharpError) as ei:
        plan.status()
    assert ei.value.code == code, str(ei.value)
    plan.status()   # reported once, then cleared


@pytest.mark.parametrize("m,prec", [(64, "fp32"), (128, "fp32"), (128, "fp16s"), (128, "bf16x3"), (256, "fp16s"),
                                    (256, "bf16x3")])
def test_wait_that_runs_out_reports_timeout_and_the_plan_recovers(m, prec):
    S = _lib()
    w, pos, shape, a, psi0 = _scan(m, 31 + m)
    ta = dev(a, torch.float32)
    plan = S.Plan(pos, m, shape, residual_every=1, precision=prec)
    plan.raar_init(dev(psi0), dev(w))
    plan.set_wait_limit(0)
    plan.raar_step(ta)
    _expect(S, plan, TIMEOUT)
    plan.raar_step(ta)                     # and again on the next step
    _expect(S, plan, TIMEOUT)
    # default limit, fresh start: the oracle's first two steps
    plan.set_wait_limit(-1)
    plan.raar_init(dev(psi0), dev(w))
    ref = O.raar_reconstruct(a, pos, shape, w, psi0, 2, beta=0.75)
    for step_i in range(2):
        met = host(plan.raar_step(ta)).real
        rec = ref["history"][step_i]
        for j, key in enumerate(("eps_a", "eps_q", "eps_delta")):
            assert abs(met[j] - rec[key]) <= MET_TOL[prec] * rec[key] + 2e-6, (step_i, key)
    plan.status()
    D = O.illumination(w, pos, shape)
    vis = D > 1e-3 * D.max()
    assert rel_l2(host(plan.psi), ref["psi"], vis) < PSI_TOL[prec]


def test_batch_wait_that_runs_out_reports_timeout():
    S = _lib()
    plans, amps = [], []
    for k, m in enumerate((64, 128)):
        w, pos, shape, a, psi0 = _scan(m, 50 + k)
        p = S.Plan(pos, m, shape, residual_every=1)
        p.raar_init(dev(psi0), dev(w))
        plans.append(p)
        amps.append(dev(a, torch.float32))
    plans[1].set_wait_limit(0)
    batch = S.Batch(plans, amps, use_graphs=False)
    batch.step()
    with pytest.raises(S.SharpError) as ei:
        batch.status()
    assert ei.value.code == TIMEOUT
    _expect(S, plans[1], TIMEOUT)
    batch.close()


@pytest.mark.parametrize("m,prec", [(64, "fp32"), (128, "fp32"), (256, "fp32"), (128, "fp16s")])
def test_nan_amplitude_is_reported(m, prec):
    S = _lib()
    w, pos, shape, a, psi0 = _scan(m, 70 + m)
    plan = S.Plan(pos, m, shape, residual_every=1, precision=prec)
    plan.raar_init(dev(psi0), dev(w))
    ta = dev(a, torch.float32)
    plan.raar_step(ta)
    plan.status()                          # clean data: no error
    ta[1, 3, 5] = float("nan")
    plan.raar_step(ta)
    _expect(S, plan, INVALID)
    ta[1, 3, 5] = -1.0                     # a negative amplitude is not |F z| either
    plan.raar_step(ta)
    _expect(S, plan, INVALID)


def test_zero_probe_is_reported():
    S = _lib()
    w, pos, shape, a, psi0 = _scan(64, 90)
    plan = S.Plan(pos, 64, shape)
    plan.raar_init(dev(psi0), dev(np.zeros_like(w)))
    _expect(S, plan, INVALID)
    plan.raar_init(dev(psi0), dev(w))
    plan.status()


def test_wait_limit_arguments():
    S = _lib()
    w, pos, shape, a, psi0 = _scan(64, 91)
    plan = S.Plan(pos, 64, shape)
    with pytest.raises(S.SharpError):
        plan.set_wait_limit(1 << 40)
    plan.set_wait_limit(1000)
    plan.set_wait_limit(-1)
