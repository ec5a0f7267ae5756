"""Pins of the oracle's RAAR update, metrics and gradient (Sec. 2.2,
Eqs. 11-14 of arXiv:1602.01448) against special cases and independent
compositions."""
import numpy as np
import pytest

import oracle as O
import synth


def _exact(seed=5, wrap=False):
    s = synth.scan_tiny(seed=seed, wrap=wrap)
    a = O.forward_amplitudes(s.obj, s.probe, s.pos, wrap)
    return s, a


def reflect_a(z, a):
    return 2 * O.data_project(z, a) - z


def reflect_q(z, s):
    return 2 * O.overlap_project(z, s.probe, s.pos, s.shape, s.wrap) - z


@pytest.mark.parametrize("beta", [0.5, 0.75, 0.9, 1.0])
def test_raar_luke_form_equals_reflector_composition(beta):
    # Luke's RAAR: beta/2 (R_Q R_a + I) z + (1 - beta) P_a z
    s, a = _exact()
    z = synth.random_frames(s.K, s.m, 11)
    expect = beta / 2 * (reflect_q(reflect_a(z, a), s) + z) + (1 - beta) * O.data_project(z, a)
    got = O.raar_update(z, a, s.probe, s.pos, s.shape, beta)
    np.testing.assert_allclose(got, expect, atol=1e-11)


def test_raar_beta_one_is_douglas_rachford():
    s, a = _exact()
    z = synth.random_frames(s.K, s.m, 12)
    pa = O.data_project(z, a)
    pq = lambda u: O.overlap_project(u, s.probe, s.pos, s.shape)
    dr = 2 * pq(pa) - pq(z) - pa + z
    np.testing.assert_allclose(O.raar_update(z, a, s.probe, s.pos, s.shape, 1.0), dr, atol=1e-11)


@pytest.mark.parametrize("form", ["luke", "printed"])
@pytest.mark.parametrize("wrap", [False, True])
def test_exact_frames_are_a_fixed_point(form, wrap):
    s, a = _exact(wrap=wrap)
    z0 = O.split(s.obj, s.probe, s.pos, wrap)
    z1 = O.raar_update(z0, a, s.probe, s.pos, s.shape, 0.75, wrap, form)
    np.testing.assert_allclose(z1, z0, atol=1e-11)


def test_overlap_of_update_equals_overlap_of_data_projection():
    # Q* z+ = Q* P_a z: the identity the fused GPU step relies on.
    s, a = _exact()
    z = synth.random_frames(s.K, s.m, 13)
    for beta in (0.6, 0.75, 1.0):
        zp = O.raar_update(z, a, s.probe, s.pos, s.shape, beta)
        np.testing.assert_allclose(O.overlap(zp, s.probe, s.pos, s.shape),
                                   O.overlap(O.data_project(z, a), s.probe, s.pos, s.shape), atol=1e-11)


def test_printed_sign_does_not_converge_but_luke_does():
    rng = np.random.default_rng(0)
    shape, m = (48, 48), 16
    obj = synth.random_object(shape, rng, phase_sigma=2.0)
    w = synth.aperture_probe(m, 6.0)
    pos = synth.raster_positions(8, 8, 4, m, shape, rng, jitter=0)
    a = O.forward_amplitudes(obj, w, pos)
    psi0 = np.ones(shape, complex)
    luke = O.raar_reconstruct(a, pos, shape, w, psi0, 120, form="luke")
    printed = O.raar_reconstruct(a, pos, shape, w, psi0, 120, form="printed")
    assert luke["history"][-1]["eps_a"] < 1e-3
    assert printed["history"][-1]["eps_a"] > 0.1
    assert O.norm(printed["z"]) > 1.5 * O.norm(O.split(psi0, w, pos))


def test_metrics_vanish_at_truth_and_eps0_is_phase_invariant():
    s, a = _exact()
    z0 = O.split(s.obj, s.probe, s.pos)
    assert O.eps_a(z0, a) < 1e-13
    assert O.eps_q(z0, a, s.probe, s.pos, s.shape) < 1e-13
    assert O.eps_0(z0, z0, s.probe, s.pos, s.shape) < 1e-15
    ph = np.exp(0.7j)
    assert O.eps_0(ph * z0, z0, s.probe, s.pos, s.shape) < 1e-14
    assert O.eps_0_object(ph * s.obj, s.obj, s.probe, s.pos, s.shape) < 1e-14
    assert O.object_nrmse(ph * s.obj, s.obj, s.probe, s.pos, s.shape) < 1e-14


def test_eps0_closed_form_phase_matches_grid_search():
    s, a = _exact()
    z0 = O.split(s.obj, s.probe, s.pos)
    z = z0 * np.exp(0.3j) + 0.05 * synth.random_frames(s.K, s.m, 2)
    u = O.overlap(z, s.probe, s.pos, s.shape)
    v = O.overlap(z0, s.probe, s.pos, s.shape)
    phis = np.linspace(-np.pi, np.pi, 200001)
    inner = np.vdot(v.ravel(), u.ravel())  # sum conj(v) u
    vals = np.sqrt(np.maximum(O.norm(u) ** 2 + O.norm(v) ** 2 - 2 * np.real(np.exp(1j * phis) * inner), 0))
    best = vals.min() / O.norm(v)
    assert abs(O.eps_0(z, z0, s.probe, s.pos, s.shape) - best) < 1e-7
    # eps_0 at z = Q psi equals the object form with D weights
    psi = s.obj * np.exp(0.2j) + 0.01
    assert abs(O.eps_0(O.split(psi, s.probe, s.pos), z0, s.probe, s.pos, s.shape)
               - O.eps_0_object(psi, s.obj, s.probe, s.pos, s.shape)) < 1e-12


def test_metric_definitions_by_hand():
    s, a = _exact()
    z = synth.random_frames(s.K, s.m, 21)
    na = np.sqrt(np.sum(a ** 2))
    Z = np.fft.fft2(z, norm="ortho")
    pa_z = np.fft.ifft2(a * np.exp(1j * np.angle(Z)), norm="ortho")
    assert abs(O.eps_a(z, a) - np.sqrt(np.sum(np.abs(pa_z - z) ** 2)) / na) < 1e-12
    zz = synth.random_frames(s.K, s.m, 22)
    assert abs(O.eps_delta(z, zz, a) - np.sqrt(np.sum(np.abs(z - zz) ** 2)) / na) < 1e-12


# ---------------------------------------------------------------- gradient
def _fd_instance():
    s = synth.scan_tiny(seed=7)
    rng = np.random.default_rng(7)
    a = O.forward_amplitudes(s.obj, s.probe, s.pos) * (1 + 0.05 * rng.standard_normal((s.K, s.m, s.m)))
    a = np.abs(a)
    psi = s.obj * (1 + 0.1 * (rng.standard_normal(s.shape) + 1j * rng.standard_normal(s.shape)))
    w = s.probe * (1 + 0.1 * (rng.standard_normal((s.m, s.m)) + 1j * rng.standard_normal((s.m, s.m))))
    return s, a, psi, w


def test_gradient_matches_central_differences():
    s, a, psi, w = _fd_instance()
    g_psi, g_w = O.amp_loss_grad(psi, w, a, s.pos)
    rng = np.random.default_rng(1)
    h = 1e-6
    errs = []
    for _ in range(12):
        y, x = rng.integers(4, 28, size=2)
        for unit in (1.0, 1j):
            dp = np.zeros_like(psi)
            dp[y, x] = h * unit
            fd = (O.amp_loss(psi + dp, w, a, s.pos) - O.amp_loss(psi - dp, w, a, s.pos)) / (2 * h)
            an = 2 * (g_psi[y, x].real if unit == 1.0 else g_psi[y, x].imag)
            errs.append(abs(fd - an) / max(abs(an), 1e-3))
        y, x = rng.integers(0, s.m, size=2)
        for unit in (1.0, 1j):
            dw = np.zeros_like(w)
            dw[y, x] = h * unit
            fd = (O.amp_loss(psi, w + dw, a, s.pos) - O.amp_loss(psi, w - dw, a, s.pos)) / (2 * h)
            an = 2 * (g_w[y, x].real if unit == 1.0 else g_w[y, x].imag)
            errs.append(abs(fd - an) / max(abs(an), 1e-3))
    assert max(errs) < 1e-6, max(errs)


def test_gradient_vanishes_at_truth():
    s = synth.scan_tiny(seed=7)
    a = O.forward_amplitudes(s.obj, s.probe, s.pos)
    g_psi, g_w = O.amp_loss_grad(s.obj, s.probe, a, s.pos)
    assert O.norm(g_psi) < 1e-12 and O.norm(g_w) < 1e-12
    assert O.amp_loss(s.obj, s.probe, a, s.pos) < 1e-25


def test_gradient_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    s, a, psi, w = _fd_instance()
    tpsi = torch.tensor(psi, dtype=torch.complex128, requires_grad=True)
    tw = torch.tensor(w, dtype=torch.complex128, requires_grad=True)
    ta = torch.tensor(a)
    loss = 0
    for (r0, c0), ai in zip(s.pos, ta):
        zi = tw * tpsi[r0:r0 + s.m, c0:c0 + s.m]
        loss = loss + ((torch.fft.fft2(zi, norm="ortho").abs() - ai) ** 2).sum()
    loss.backward()
    g_psi, g_w = O.amp_loss_grad(psi, w, a, s.pos)
    # torch returns 2 dL/d conj(x) for a real loss
    np.testing.assert_allclose(tpsi.grad.numpy(), 2 * g_psi, atol=1e-10)
    np.testing.assert_allclose(tw.grad.numpy(), 2 * g_w, atol=1e-10)
    assert abs(loss.item() - O.amp_loss(psi, w, a, s.pos)) < 1e-10 * loss.item()


def test_eps_q_by_hand():
    s, a = _exact()
    z = synth.random_frames(s.K, s.m, 23)
    D = O.illumination(s.probe, s.pos, s.shape)
    img = np.zeros(s.shape, complex)
    for i, (r0, c0) in enumerate(s.pos):
        img[r0:r0 + s.m, c0:c0 + s.m] += np.conj(s.probe) * z[i]
    psi = np.where(D > 0, img / np.where(D > 0, D, 1), 0)
    pz = np.stack([s.probe * psi[r0:r0 + s.m, c0:c0 + s.m] for r0, c0 in s.pos])
    expect = np.sqrt(np.sum(np.abs(pz - z) ** 2)) / np.sqrt(np.sum(a ** 2))
    assert abs(O.eps_q(z, a, s.probe, s.pos, s.shape) - expect) < 1e-12


def test_object_nrmse_by_hand():
    # The secondary object report (reading R8): over the pixels whose
    # illumination D = Q*Q reaches 10 % of its maximum, the relative error of
    # psi against psi_true after the closed-form global phase.  Written out
    # with explicit loops over the frame windows and the selected pixels.
    s = synth.scan_tiny(seed=12)
    rng = np.random.default_rng(31)
    psi = s.obj * np.exp(0.7j) + 0.05 * (rng.standard_normal(s.shape) + 1j * rng.standard_normal(s.shape))
    D = np.zeros(s.shape)
    for r0, c0 in s.pos:
        for y in range(s.m):
            for x in range(s.m):
                D[r0 + y, c0 + x] += abs(s.probe[y, x]) ** 2
    dmax = max(D.ravel())
    num = 0j
    pairs = []
    for y in range(s.shape[0]):
        for x in range(s.shape[1]):
            if D[y, x] >= 0.1 * dmax:
                num += np.conj(psi[y, x]) * s.obj[y, x]
                pairs.append((psi[y, x], s.obj[y, x]))
    ph = num / abs(num)
    err = np.sqrt(sum(abs(ph * u - v) ** 2 for u, v in pairs))
    ref = np.sqrt(sum(abs(v) ** 2 for _, v in pairs))
    got = O.object_nrmse(psi, s.obj, s.probe, s.pos, s.shape)
    assert abs(got - err / ref) < 1e-12
    # pixels below the threshold do not count: changing them leaves it unchanged
    low = D < 0.1 * dmax
    assert low.any()
    psi2 = np.where(low, 123.0 + 4j, psi)
    assert abs(O.object_nrmse(psi2, s.obj, s.probe, s.pos, s.shape) - got) < 1e-14
    # and one pixel just above the threshold does
    hi = np.argwhere(~low)[0]
    psi3 = psi.copy()
    psi3[tuple(hi)] += 1.0
    assert abs(O.object_nrmse(psi3, s.obj, s.probe, s.pos, s.shape) - got) > 1e-6


def test_reconstruct_loop_order_and_metric_convention():
    # Step l: z-update with the current probe, object from z^(l), probe from
    # (psi^(l), z^(l)) on probe steps; metrics describe the entering iterate.
    s = synth.scan_tiny(seed=9)
    rng = np.random.default_rng(2)
    a = np.abs(O.forward_amplitudes(s.obj, s.probe, s.pos) * (1 + 0.02 * rng.standard_normal((s.K, s.m, s.m))))
    w0 = s.probe * 1.1
    psi0 = np.ones(s.shape, complex)
    out = O.raar_reconstruct(a, s.pos, s.shape, w0, psi0, 4, beta=0.8, probe_every=2)
    w = w0.copy()
    z = O.split(psi0, w, s.pos)
    zs, formed = [z], [w]          # formed[l]: probe that formed zs[l]
    for step in range(1, 5):
        z = O.raar_update(z, a, w, s.pos, s.shape, 0.8)
        formed.append(w)
        psi = O.object_update(z, w, s.pos, s.shape)
        if step % 2 == 0:
            w = O.probe_update(z, psi, s.pos, w)
        zs.append(z)
    np.testing.assert_allclose(out["z"], zs[-1], atol=1e-12)
    np.testing.assert_allclose(out["w"], w, atol=1e-12)
    np.testing.assert_allclose(out["psi"], psi, atol=1e-12)
    for step, rec in enumerate(out["history"], start=1):
        zin = zs[step - 1]
        assert abs(rec["eps_a"] - O.eps_a(zin, a)) < 1e-13
        assert abs(rec["eps_q"] - O.eps_q(zin, a, formed[step - 1], s.pos, s.shape)) < 1e-13
        zprev = zs[step - 2] if step >= 2 else np.zeros_like(zin)
        assert abs(rec["eps_delta"] - O.eps_delta(zin, zprev, a)) < 1e-13


def test_small_raster_reaches_paper_threshold():
    # Fig. 3 caption: reconstruction counts as achieved at eps_0 < 5e-4 on a
    # noiseless, exact-probe simulation.  The 100-frame 64^2 raster must get
    # there within its 100 iterations, with eps_0 falling overall.
    s = synth.scan_small_raster()
    a = O.forward_amplitudes(s.obj, s.probe, s.pos)
    out = O.raar_reconstruct(a, s.pos, s.shape, s.probe, s.psi_init, 100,
                             psi_true=s.obj, record_metrics=False)
    e0 = [h["eps_0"] for h in out["history"]]
    assert e0[-1] < 5e-4
    assert e0[-1] < 1e-2 * e0[0]
    assert all(e0[k + 10] < e0[k] for k in range(0, 90, 10))
