"""GPU parity of the fused RAAR step against the FP64 oracle (Sec. 2.2
reconstruction sequence, Eqs. 7-14)."""
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


def _gpu_frames(plan, w_form):
    """z = w_f . psi_y(r + x_i) + c_i, rebuilt on the host from the GPU state."""
    return O.split(host(plan.psi_y), w_form, host(plan.pos).real.astype(int), bool(plan.params.wrap)) + host(plan.c)


def _noisy_scan(m, K_side, step, n_extra, seed, photons=1e5, wrap=False):
    rng = np.random.default_rng(seed)
    ext = (K_side - 1) * step + m
    n = ext + n_extra
    shape = (n, n)
    obj = synth.random_object(shape, rng)
    w = synth.gaussian_probe(m, m / 6.0, rng)
    pos = synth.raster_positions(K_side, K_side, step, m, shape, rng, jitter=1)
    inten = O.forward_amplitudes(obj, w, pos) ** 2
    a = np.sqrt(synth.poisson_intensities(inten, photons, rng)) if photons else np.sqrt(inten)
    a = a.astype(np.float32).astype(np.float64)
    return obj, w, pos, shape, a


def _check_metrics(gpu, rec, first):
    assert abs(gpu[0] - rec["eps_a"]) <= 1e-4 * rec["eps_a"] + 2e-6
    assert abs(gpu[1] - rec["eps_q"]) <= 1e-4 * rec["eps_q"] + 2e-6
    assert abs(gpu[2] - rec["eps_delta"]) <= 1e-4 * rec["eps_delta"] + 2e-6


@pytest.mark.parametrize("m,side,step", [(64, 5, 12), (128, 4, 24), (256, 3, 48)])
def test_raar_steps_match_oracle(m, side, step):
    S = _lib()
    obj, w, pos, shape, a = _noisy_scan(m, side, step, 37, seed=m)
    # a broadband start (random object): with a flat start the frame spectra
    # are the probe's, whose far tails sit below FP32 resolution, and P_a's
    # phase there is rounding noise on any FP32 path
    psi0 = synth.random_object(shape, np.random.default_rng(m + 1), phase_sigma=1.0)
    n_steps = 4
    ref = O.raar_reconstruct(a, pos, shape, w, psi0, n_steps, beta=0.75)
    plan = S.Plan(pos, m, shape, beta=0.75, residual_every=1)
    plan.raar_init(dev(psi0), dev(w))
    ta = dev(a, torch.float32)
    zs = [O.split(psi0, w, pos)]
    for step_i in range(n_steps):
        met = host(plan.raar_step(ta)).real
        _check_metrics(met, ref["history"][step_i], step_i == 0)
        assert abs(met[3] - O.norm(a)) < 1e-5 * O.norm(a)
    z_gpu = _gpu_frames(plan, w)
    assert rel_l2(z_gpu, ref["z"]) < 1e-5 * n_steps
    D = O.illumination(w, pos, shape)
    vis = D > 1e-12 * D.max()
    assert rel_l2(host(plan.psi), ref["psi"], vis) < 1e-5 * n_steps


def test_raar_with_probe_refinement_matches_oracle():
    S = _lib()
    m = 64
    obj, w, pos, shape, a = _noisy_scan(m, 6, 10, 30, seed=7, photons=1e6)
    rng = np.random.default_rng(3)
    w0 = synth.perturb_probe(w, rng, 0.1)
    psi0 = rng.uniform(0, 1, shape).astype(complex)
    n_steps = 6
    ref = O.raar_reconstruct(a, pos, shape, w0, psi0, n_steps, beta=0.75, probe_every=2)
    plan = S.Plan(pos, m, shape, beta=0.75, probe_every=2, residual_every=1)
    plan.raar_init(dev(psi0), dev(w0))
    ta = dev(a, torch.float32)
    for step_i in range(n_steps):
        met = host(plan.raar_step(ta)).real
        _check_metrics(met, ref["history"][step_i], step_i == 0)
    assert rel_l2(host(plan.probe), ref["w"]) < 1e-4
    D = O.illumination(ref["w"], pos, shape)
    vis = D > 1e-3 * D.max()
    assert rel_l2(host(plan.psi), ref["psi"], vis) < 1e-4


def test_residual_cadence_and_nan_off_cadence():
    S = _lib()
    obj, w, pos, shape, a = _noisy_scan(64, 4, 12, 20, seed=11)
    psi0 = np.ones(shape, complex)
    ref = O.raar_reconstruct(a, pos, shape, w, psi0, 6, beta=0.8)
    plan = S.Plan(pos, 64, shape, beta=0.8, residual_every=3)
    plan.raar_init(dev(psi0), dev(w))
    ta = dev(a, torch.float32)
    for step_i in range(6):
        met = host(plan.raar_step(ta)).real
        rec = ref["history"][step_i]
        assert abs(met[0] - rec["eps_a"]) <= 1e-4 * rec["eps_a"] + 2e-6
        if (step_i + 1) % 3 == 0:
            _check_metrics(met, rec, False)
        else:
            assert np.isnan(met[1]) and np.isnan(met[2])


def test_exact_data_is_a_fixed_point_on_gpu():
    S = _lib()
    obj, w, pos, shape, a = _noisy_scan(64, 5, 12, 16, seed=5, photons=None)
    plan = S.Plan(pos, 64, shape)
    plan.raar_init(dev(obj), dev(w))
    ta = dev(a, torch.float32)
    for _ in range(5):
        met = host(plan.raar_step(ta)).real
    assert met[0] < 2e-6 and met[1] < 2e-6
    D = O.illumination(w, pos, shape)
    vis = D > 1e-3 * D.max()
    assert rel_l2(host(plan.psi), obj, vis) < 2e-6


def test_small_raster_nrmse_within_2_percent_of_oracle():
    # 100 frames of 64^2, 256^2 object, noiseless, known probe, 100 iterations.
    # eps_0 of the GPU object tracks the oracle's within 1.02x at every
    # checkpoint where the oracle's eps_0 is above 1e-6; at iteration 100 the
    # oracle sits at ~5e-7, within 4x of the FP32 pipeline's rounding floor
    # (~1.2e-7, reproduced by a float32 CPU emulation), where the ratio is
    # rounding noise (observed 1.00-1.05): bounded at 1.10 there.
    S = _lib()
    s = synth.scan_small_raster()
    a = O.forward_amplitudes(s.obj, s.probe, s.pos).astype(np.float32).astype(np.float64)
    ref = O.raar_reconstruct(a, s.pos, s.shape, s.probe, s.psi_init, 100, psi_true=s.obj,
                             record_metrics=False)
    e_ref = [h["eps_0"] for h in ref["history"]]
    plan = S.Plan(s.pos, s.m, s.shape, residual_every=0)
    plan.raar_init(dev(s.psi_init), dev(s.probe))
    ta = dev(a, torch.float32)
    tobj, tw = dev(s.obj), dev(s.probe)
    ratios = {}
    for it in range(1, 101):
        plan.raar_step(ta, metrics=False)
        if it % 10 == 0:
            e_gpu = plan.solution_error(plan.psi, tobj, tw)[0].item()
            ratios[it] = e_gpu / e_ref[it - 1]
    e_host = O.eps_0_object(host(plan.psi), s.obj, s.probe, s.pos, s.shape)
    assert abs(e_gpu - e_host) < 1e-3 * e_host + 1e-9
    for it, r in ratios.items():
        if e_ref[it - 1] > 1e-6:
            assert r <= 1.02, (it, r, ratios)
    assert ratios[100] <= 1.10, ratios
    print("eps_0 ratio GPU/oracle by iteration:", {k: round(v, 4) for k, v in ratios.items()})


def test_full_size_fermat_step_on_sampled_outputs():
    # The 2500-frame 128^2 Fermat scan over a 1024^2 object, one fused step in
    # the launch configuration the benchmark times; checked on sampled frames
    # (c update) and a sampled image patch (object update) that the oracle
    # computes frame by frame.
    S = _lib()
    s = synth.scan_fermat()
    m, K = s.m, s.K
    rng = np.random.default_rng(0)
    plan = S.Plan(s.pos, m, s.shape, beta=0.75, residual_every=1)
    amp = plan.forward_amplitudes(dev(s.obj), dev(s.probe))
    amp.mul_(1.0 + 0.05 * torch.randn(amp.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(1)))
    amp.abs_()
    plan.raar_init(dev(s.psi_init), dev(s.probe_init))
    # run one step so that c != 0, then snapshot the inputs of the checked step
    plan.raar_step(amp)
    c_in = plan.c.clone()
    psiy_in = host(plan.psi_y)
    plan.raar_step(amp)
    w = s.probe_init
    frames = rng.choice(K, 6, replace=False)
    a_h = host(amp).real
    c_in_h = {int(i): host(c_in[int(i)]) for i in frames}
    for i in frames:
        i = int(i)
        z = O.split(psiy_in, w, s.pos[i:i + 1])[0] + c_in_h[i]
        p = O.data_project(z[None], a_h[i][None])[0]
        c_ref = (1 - 1.5) * p + 0.75 * z
        assert rel_l2(host(plan.c[i]), c_ref) < 1e-5
    # object on a 6x6 patch near the scan centre: A = sum conj(w) P_a z over
    # every frame touching the patch
    y0, x0, P = 500, 520, 6
    cover = [i for i in range(K) if s.pos[i, 0] < y0 + P and y0 < s.pos[i, 0] + m
             and s.pos[i, 1] < x0 + P and x0 < s.pos[i, 1] + m]
    assert len(cover) > 50
    c_all = host(c_in[torch.tensor(cover, device="cuda")])
    A = np.zeros((P, P), complex)
    Dp = np.zeros((P, P))
    for j, i in enumerate(cover):
        z = O.split(psiy_in, w, s.pos[i:i + 1])[0] + c_all[j]
        p = O.data_project(z[None], a_h[i][None])[0]
        ya, yb = max(y0, s.pos[i, 0]), min(y0 + P, s.pos[i, 0] + m)
        xa, xb = max(x0, s.pos[i, 1]), min(x0 + P, s.pos[i, 1] + m)
        ly, lx = ya - s.pos[i, 0], xa - s.pos[i, 1]
        sl = (slice(ly, ly + yb - ya), slice(lx, lx + xb - xa))
        A[ya - y0:yb - y0, xa - x0:xb - x0] += np.conj(w[sl]) * p[sl]
        Dp[ya - y0:yb - y0, xa - x0:xb - x0] += np.abs(w[sl]) ** 2
    D_full = O.illumination(w, s.pos, s.shape)[y0:y0 + P, x0:x0 + P]
    np.testing.assert_allclose(Dp, D_full, rtol=1e-12)
    assert rel_l2(host(plan.psi)[y0:y0 + P, x0:x0 + P], A / Dp) < 1e-5
