"""Gradient-based reconstruction through the library's amplitude loss
(sum_i || |F z_i| - a_i ||^2 with z = Q psi: the residual of the data
projection, Eq. 7, used as a loss) and its hand-written adjoint, driven by
torch.optim.Adam, against RAAR (Sec. 2.2) on the same data: a 40 x 40 raster
(step 10 px) of 128^2 frames over a periodic 512^2 object, Poisson noise at
1e6 photons per frame, known probe, flat start, 200 steps each.

Adam's learning rate 0.1 was chosen from {0.003, 0.01, 0.03, 0.1} on this
workload (eps_0 after 200 steps: 0.38, 0.27, 0.081, 0.066); RAAR reaches
0.064 by step 50 and stays there (the noise floor of this data).
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from tests.gpu_util import dev, note

pytestmark = pytest.mark.gpu

ADAM_LR = 0.1
STEPS = 200


def test_adam_on_amplitude_loss_and_raar_reach_the_noise_floor():
    import paper_1602_01448_gb300 as S
    s = synth.scan_wrapped_raster()
    rng = np.random.default_rng(44)
    inten = O.forward_amplitudes(s.obj, s.probe, s.pos, True) ** 2
    a = np.sqrt(synth.poisson_intensities(inten, s.photons, rng)).astype(np.float32)
    plan = S.Plan(s.pos, s.m, s.shape, wrap=True, residual_every=0)
    ta = torch.as_tensor(a).cuda()
    tw, tobj = dev(s.probe), dev(s.obj)
    psi0 = np.ones(s.shape, complex)

    plan.raar_init(dev(psi0), tw)
    for _ in range(STEPS):
        plan.raar_step(ta, metrics=False)
    e_raar = plan.solution_error(plan.psi, tobj, tw)[0].item()

    psi = dev(psi0).requires_grad_(True)
    opt = torch.optim.Adam([psi], lr=ADAM_LR)
    losses = []
    for _ in range(STEPS):
        opt.zero_grad()
        loss = S.amp_loss(plan, psi, tw, ta)
        loss.backward()
        opt.step()
        losses.append(loss.item())
    e_adam = plan.solution_error(psi.detach(), tobj, tw)[0].item()
    note(f"eps_0 after {STEPS} steps: RAAR {e_raar:.4f}, Adam(lr={ADAM_LR}) {e_adam:.4f}; "
          f"loss {losses[0]:.4g} -> {losses[-1]:.4g}")
    assert losses[-1] < losses[0] / 30
    assert e_raar < 0.075 and e_adam < 0.08
    assert e_adam < 1.25 * e_raar
