"""GPU parity of the fused RAAR step against the FP64 oracle (Sec. 2.2
reconstruction sequence, Eqs. 7-14)."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from tests.gpu_util import dev, host, rel_l2, note

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


# (256, 3, 48, 38, 2): 256^2 frames over an even-width object with metrics
# every 2nd step, so half the steps run the frame pass without metrics (the
# path of the timed 10^4-frame raster) and write the eps_Delta buffer that
# the next step reads
@pytest.mark.parametrize("m,side,step,extra,every", [(64, 5, 12, 37, 1), (128, 4, 24, 37, 1), (256, 3, 48, 37, 1),
                                                     (256, 3, 48, 38, 2)])
def test_raar_steps_match_oracle(m, side, step, extra, every):
    S = _lib()
    obj, w, pos, shape, a = _noisy_scan(m, side, step, extra, seed=m)
    # a broadband start (random object): with a flat start the frame spectra
    # are the probe's, whose far tails sit below FP32 resolution, and P_a's
    # phase there is rounding noise on any FP32 path
    psi0 = synth.random_object(shape, np.random.default_rng(m + 1), phase_sigma=1.0)
    n_steps = 4
    ref = O.raar_reconstruct(a, pos, shape, w, psi0, n_steps, beta=0.75)
    plan = S.Plan(pos, m, shape, beta=0.75, residual_every=every)
    plan.raar_init(dev(psi0), dev(w))
    ta = dev(a, torch.float32)
    for step_i in range(n_steps):
        met = host(plan.raar_step(ta)).real
        if (step_i + 1) % every == 0:
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


def _beta_tolerance(beta, steps, e_op=1e-5):
    """Parity bound of a RAAR run with relaxation beta after `steps` steps.

    The image pass forms A/D = psi + (C' - b B')/((1-2b) D) from the FP32
    frame pass (Sec. 2.2 RAAR update, Luke form): an error of e_op (the FP32
    single-operator bound) in the frame-pass sums reaches the object once
    directly and once through the factor 1/|1-2b|, and the errors of
    successive steps add: steps * (1 + 1/|1-2b|) * e_op."""
    return steps * (1.0 + 1.0 / abs(1.0 - 2.0 * beta)) * e_op


@pytest.mark.parametrize("beta", [1.0, 0.75, 0.55, 0.51])
def test_raar_beta_range_matches_oracle(beta):
    # beta = 1 is Douglas-Rachford (2 P_Q P_a - P_Q - P_a + I); beta near 1/2
    # makes 1/(1-2b) in the image pass large (51 at beta = 0.51)
    S = _lib()
    obj, w, pos, shape, a = _noisy_scan(64, 4, 12, 21, seed=13)
    psi0 = synth.random_object(shape, np.random.default_rng(14), phase_sigma=1.0)
    n_steps = 3
    ref = O.raar_reconstruct(a, pos, shape, w, psi0, n_steps, beta=beta)
    plan = S.Plan(pos, 64, shape, beta=beta, residual_every=1)
    plan.raar_init(dev(psi0), dev(w))
    ta = dev(a, torch.float32)
    for step_i in range(n_steps):
        met = host(plan.raar_step(ta)).real
        rec = ref["history"][step_i]
        tol = max(1e-4, _beta_tolerance(beta, step_i + 1))
        for j, key in enumerate(("eps_a", "eps_q", "eps_delta")):
            assert abs(met[j] - rec[key]) <= tol * rec[key] + 2e-6, (step_i, key, met[j], rec[key])
    D = O.illumination(w, pos, shape)
    vis = D > 1e-3 * D.max()
    err = rel_l2(host(plan.psi), ref["psi"], vis)
    note(f"beta {beta}: object rel err {err:.2e} after {n_steps} steps (bound {_beta_tolerance(beta, n_steps):.1e})")
    assert err < _beta_tolerance(beta, n_steps)


def test_beta_at_one_half_is_rejected():
    S = _lib()
    pos = np.array([[0, 0], [8, 8]], np.int32)
    for beta in (0.5, 0.25):
        with pytest.raises(S.SharpError) as ei:
            S.Plan(pos, 64, (80, 80), beta=beta)
        assert ei.value.code == 1 and "beta" in str(ei.value)


def test_single_frame_scan_matches_oracle():
    S = _lib()
    m = 128
    rng = np.random.default_rng(15)
    shape = (m + 9, m + 3)
    obj = synth.random_object(shape, rng)
    w = synth.gaussian_probe(m, m / 6.0, rng)
    pos = np.array([[5, 2]], np.int32)
    a = O.forward_amplitudes(obj, w, pos) * (1 + 0.1 * rng.standard_normal((1, m, m)))
    a = np.abs(a).astype(np.float32).astype(np.float64)
    psi0 = synth.random_object(shape, rng, phase_sigma=1.0)
    ref = O.raar_reconstruct(a, pos, shape, w, psi0, 3)
    plan = S.Plan(pos, m, shape, residual_every=1)
    plan.raar_init(dev(psi0), dev(w))
    for step_i in range(3):
        met = host(plan.raar_step(dev(a, torch.float32))).real
        _check_metrics(met, ref["history"][step_i], step_i == 0)
    D = O.illumination(w, pos, shape)
    vis = D > 1e-3 * D.max()
    assert rel_l2(host(plan.psi), ref["psi"], vis) < 3e-5
    assert np.all(host(plan.psi)[~(D > 1e-12 * D.max())] == 0)


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
    # 100 frames of 64^2, 256^2 object, noiseless, known probe, 100
    # iterations: eps_0 (Eq. 14) of the GPU object stays within 1.02x of the
    # FP64 oracle's at every 10th iteration, iteration 100 included (the
    # oracle reaches ~4.9e-7 there).
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
    note("eps_0 ratio GPU/oracle by iteration:", {k: round(v, 4) for k, v in ratios.items()})
    for it, r in ratios.items():
        assert r <= 1.02, (it, r, ratios)


_AMP_CACHE = {}


def _host_amplitudes(s, seed, chunk=500):
    """Amplitudes of the scan from the oracle's forward model (Eq. 1), with
    5 % multiplicative noise, computed on the host in chunks of frames (kept
    for the other tests of the same scan)."""
    key = (s.name, s.seed, seed)
    if key in _AMP_CACHE:
        return _AMP_CACHE[key]
    _AMP_CACHE.clear()
    rng = np.random.default_rng(seed)
    out = np.empty((s.K, s.m, s.m), np.float32)
    for k0 in range(0, s.K, chunk):
        a = O.forward_amplitudes(s.obj, s.probe, s.pos[k0:k0 + chunk], s.wrap)
        out[k0:k0 + chunk] = np.abs(a * (1.0 + 0.05 * rng.standard_normal(a.shape)))
    _AMP_CACHE[key] = out
    return out


def _sampled_step_parity(s, patch, beta=0.75, n_frames=6, precision="fp32", tol=1e-5):
    """One fused RAAR step of a full-size scan, in the launch configuration the
    benchmark times, checked on sampled frames (state update) and on a small
    image patch (object update) that the oracle computes frame by frame."""
    S = _lib()
    m, K = s.m, s.K
    rng = np.random.default_rng(0)
    a_h = _host_amplitudes(s, 1)
    plan = S.Plan(s.pos, m, s.shape, beta=beta, wrap=s.wrap, residual_every=1, precision=precision)
    amp = dev(a_h, torch.float32)
    plan.raar_init(dev(s.psi_init), dev(s.probe_init))
    # run one step so that c != 0, then snapshot the inputs of the checked step
    plan.raar_step(amp)
    c_in = plan.c.clone()
    psiy_in = host(plan.psi_y)
    plan.raar_step(amp)
    w = s.probe_init
    a_h = a_h.astype(np.float64)
    for i in rng.choice(K, n_frames, replace=False):
        i = int(i)
        z = O.split(psiy_in, w, s.pos[i:i + 1], s.wrap)[0] + host(c_in[i])
        p = O.data_project(z[None], a_h[i][None])[0]
        c_ref = (1 - 2 * beta) * p + beta * z
        assert rel_l2(host(plan.c[i]), c_ref) < tol, i
    # object on a small patch away from the object edges: A = sum conj(w) P_a z
    # over every frame touching the patch
    y0, x0, P = patch
    cover = [i for i in range(K) if s.pos[i, 0] < y0 + P and y0 < s.pos[i, 0] + m
             and s.pos[i, 1] < x0 + P and x0 < s.pos[i, 1] + m]
    assert len(cover) > 20
    c_all = host(c_in[torch.tensor(cover, device="cuda")])
    A = np.zeros((P, P), complex)
    Dp = np.zeros((P, P))
    for j, i in enumerate(cover):
        z = O.split(psiy_in, w, s.pos[i:i + 1], s.wrap)[0] + c_all[j]
        p = O.data_project(z[None], a_h[i][None])[0]
        ya, yb = max(y0, s.pos[i, 0]), min(y0 + P, s.pos[i, 0] + m)
        xa, xb = max(x0, s.pos[i, 1]), min(x0 + P, s.pos[i, 1] + m)
        ly, lx = ya - s.pos[i, 0], xa - s.pos[i, 1]
        sl = (slice(ly, ly + yb - ya), slice(lx, lx + xb - xa))
        A[ya - y0:yb - y0, xa - x0:xb - x0] += np.conj(w[sl]) * p[sl]
        Dp[ya - y0:yb - y0, xa - x0:xb - x0] += np.abs(w[sl]) ** 2
    D_full = O.illumination(w, s.pos, s.shape, s.wrap)[y0:y0 + P, x0:x0 + P]
    np.testing.assert_allclose(Dp, D_full, rtol=1e-12)
    assert rel_l2(host(plan.psi)[y0:y0 + P, x0:x0 + P], A / Dp) < tol


def test_full_size_fermat_step_on_sampled_outputs():
    # 2500 frames of 128^2 on a Fermat spiral over a 1024^2 object
    _sampled_step_parity(synth.scan_fermat(), (500, 520, 6))


def test_full_size_large_raster_step_on_sampled_outputs():
    # 10^4 frames of 256^2 on a 100 x 100 raster over a 3072^2 object
    _sampled_step_parity(synth.scan_large_raster(), (1500, 1490, 6))


def test_full_size_wrapped_raster_step_on_sampled_outputs():
    # 1600 frames of 128^2 on a 40 x 40 raster over a periodic 512^2 object
    _sampled_step_parity(synth.scan_wrapped_raster(), (250, 260, 6))


def test_large_frames_nrmse_trajectory_against_oracle():
    # 256^2 frames (the 10^4-frame raster's frame size, step 24 +-1 px and
    # probe) on a 10 x 10 raster, noiseless, known probe, flat start, 16
    # steps: eps_0 (Eq. 14) of the GPU object stays within 1.02x of the FP64
    # oracle's at every 4th step
    S = _lib()
    rng = np.random.default_rng(23)
    m = 256
    shape = (9 * 24 + m + 64,) * 2
    obj = synth.random_object(shape, rng)
    w = synth.gaussian_probe(m, 40.0, rng)
    pos = synth.raster_positions(10, 10, 24, m, shape, rng, jitter=1)
    a = O.forward_amplitudes(obj, w, pos).astype(np.float32).astype(np.float64)
    psi0 = np.ones(shape, complex)
    n_it = 16
    ref = O.raar_reconstruct(a, pos, shape, w, psi0, n_it, psi_true=obj, record_metrics=False)
    e_ref = [h["eps_0"] for h in ref["history"]]
    plan = S.Plan(pos, m, shape, residual_every=0)
    plan.raar_init(dev(psi0), dev(w))
    ta = dev(a, torch.float32)
    tobj, tw = dev(obj), dev(w)
    out = {}
    for it in range(1, n_it + 1):
        plan.raar_step(ta, metrics=False)
        if it % 4 == 0:
            out[it] = (plan.solution_error(plan.psi, tobj, tw)[0].item(), e_ref[it - 1])
    note("256^2 eps_0 (GPU, oracle):", {k: (f"{g:.4e}", f"{r:.4e}") for k, (g, r) in out.items()})
    for it, (g, r) in out.items():
        assert abs(g / r - 1) <= 0.02, (it, g, r)
