"""GPU parity of the illumination refinement and initialisation (Sec. 2.2:
drift and Fourier-space pathologies, reconstruction sequence steps 2 and 7;
Sec. 3.2 threshold variant) against the FP64 oracle."""
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


def _plan(S, m, K=3):
    rng = np.random.default_rng(m)
    n = m + 40
    pos = rng.integers(0, n - m + 1, size=(K, 2)).astype(np.int32)
    return S.Plan(pos, m, (n, n)), pos, (n, n)


def _drifted_probe(m, seed, d):
    rng = np.random.default_rng(seed)
    w = synth.gaussian_probe(m, m / 8.0, rng) * (1 + 0.2 * rng.standard_normal((m, m)))
    return np.roll(w, d, axis=(0, 1))


def _clear_of_rounding(w, margin=1e-2):
    """The centring shift is an integer taken from the centroid (FP32 |w|^2 on
    the GPU, FP64 in the oracle).  Both sides take the same decision when the
    centroid offset is away from a rounding boundary; the test inputs are
    chosen so, and this checks it."""
    m = w.shape[0]
    for c in O.probe_centroid(w):
        t = c - m / 2 + 0.5
        assert abs(t - round(t)) > margin, (c, m)


def _band_mask(m, keep):
    """Low-pass Fourier mask in the unshifted layout: |q| <= keep per axis."""
    q = np.minimum(np.arange(m), m - np.arange(m))
    return ((q[:, None] <= keep) & (q[None, :] <= keep)).astype(np.float64)


@pytest.mark.parametrize("m", [64, 128, 256])
def test_centring_matches_oracle(m):
    S = _lib()
    plan, _, _ = _plan(S, m)
    w = _drifted_probe(m, 1, (7, -4))
    _clear_of_rounding(w)
    plan.set_probe_refinement(center=True)
    got = host(plan.probe_refine(dev(w)))
    ref, d = O.probe_center(w)
    assert d == (7, -4)
    assert rel_l2(got, ref) < 1e-6


@pytest.mark.parametrize("m", [64, 128, 256])
def test_fourier_constraints_match_oracle(m):
    S = _lib()
    plan, _, _ = _plan(S, m)
    w = _drifted_probe(m, 2, (0, 0))
    mask = _band_mask(m, m // 5)
    plan.set_probe_refinement(mask=dev(mask, torch.float32))
    got = host(plan.probe_refine(dev(w)))
    assert rel_l2(got, O.probe_fourier_mask(w, mask)) < TOL
    a_w = np.abs(O.fft2u(synth.gaussian_probe(m, m / 6.0, 3))).astype(np.float32).astype(np.float64)
    plan.set_probe_refinement(amplitude=dev(a_w, torch.float32))
    wt = dev(w)
    plan.probe_refine(wt, out=wt)                       # in place
    assert rel_l2(host(wt), O.probe_fourier_amplitude(w, a_w)) < TOL
    # mask, then centring, in one call
    wd = _drifted_probe(m, 4, (-5, 9))
    _clear_of_rounding(O.probe_fourier_mask(wd, mask))
    plan.set_probe_refinement(mask=dev(mask, torch.float32), center=True)
    got = host(plan.probe_refine(dev(wd)))
    assert rel_l2(got, O.refine_probe(wd, probe_mask=mask, probe_com=True)) < TOL
    plan.set_probe_refinement()
    np.testing.assert_array_equal(host(plan.probe_refine(dev(wd))), host(dev(wd)))


@pytest.mark.parametrize("m", [64, 128, 256])
@pytest.mark.parametrize("threshold", [0.0, 0.05])
def test_mean_frame_initialisation_matches_oracle(m, threshold):
    S = _lib()
    rng = np.random.default_rng(5)
    K = 7
    n = m + 50
    pos = rng.integers(0, n - m + 1, size=(K, 2)).astype(np.int32)
    obj = synth.random_object((n, n), rng)
    w = synth.gaussian_probe(m, m / 6.0, rng)
    a = O.forward_amplitudes(obj, w, pos).astype(np.float32).astype(np.float64)
    plan = S.Plan(pos, m, (n, n))
    got = host(plan.probe_init_mean(dev(a, torch.float32), threshold))
    ref = O.probe_from_mean_frame(a, threshold)
    assert rel_l2(got, ref) < TOL


def test_raar_with_mask_and_centring_matches_oracle(monkeypatch):
    S = _lib()
    import oracle.sharp_oracle as OS
    centre = OS.probe_center

    def checked_centre(w):       # every centring in the oracle run is clear of rounding
        _clear_of_rounding(w)
        return centre(w)

    monkeypatch.setattr(OS, "probe_center", checked_centre)
    m = 64
    rng = np.random.default_rng(7)
    side, step = 6, 10
    n = (side - 1) * step + m + 30
    shape = (n, n)
    obj = synth.random_object(shape, rng)
    w = synth.gaussian_probe(m, m / 6.0, rng)
    pos = synth.raster_positions(side, side, step, m, shape, rng, jitter=1)
    inten = O.forward_amplitudes(obj, w, pos) ** 2
    a = np.sqrt(synth.poisson_intensities(inten, 1e6, rng)).astype(np.float32).astype(np.float64)
    w0 = np.roll(synth.perturb_probe(w, rng, 0.1), (3, -2), axis=(0, 1))
    psi0 = rng.uniform(0, 1, shape).astype(complex)
    mask = _band_mask(m, 20)
    n_steps = 6
    ref = O.raar_reconstruct(a, pos, shape, w0, psi0, n_steps, beta=0.75, probe_every=2, probe_mask=mask,
                             probe_com=True, record_metrics=False)
    plan = S.Plan(pos, m, shape, beta=0.75, probe_every=2, residual_every=0)
    plan.set_probe_refinement(mask=dev(mask, torch.float32), center=True)
    plan.raar_init(dev(psi0), dev(w0))
    ta = dev(a, torch.float32)
    for _ in range(n_steps):
        plan.raar_step(ta, metrics=False)
    assert rel_l2(host(plan.probe), ref["w"]) < 1e-4
    D = O.illumination(ref["w"], pos, shape)
    vis = D > 1e-3 * D.max()
    assert rel_l2(host(plan.psi), ref["psi"], vis) < 1e-4


def test_refinement_arguments_are_checked():
    S = _lib()
    plan, _, _ = _plan(S, 64)
    with pytest.raises(S.SharpError) as e:
        S._check(S._C["sharp_plan_set_probe_refinement"](plan.handle, 3, None, 0, None))
    assert e.value.code == 1
    with pytest.raises(S.SharpError) as e:
        S._check(S._C["sharp_plan_set_probe_refinement"](plan.handle, 1, None, 0, None))
    assert e.value.code == 1
    amp = torch.zeros((3, 64, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(S.SharpError) as e:
        plan.probe_init_mean(amp, threshold=1.5)
    assert e.value.code == 1
