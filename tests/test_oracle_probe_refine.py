"""Pins of the oracle's illumination refinement and initialisation (Sec. 2.2:
the drift and Fourier-space pathologies and reconstruction sequence steps 2
and 7; Sec. 3.2 threshold variant) against closed forms, brute-force sums and
invariants that do not go through the functions under test."""
import math

import numpy as np
import pytest

import oracle as O
import synth
from tests.test_oracle_operators import brute_dft2


def brute_idft2(F):
    """Unitary inverse 2D DFT written out as the double sum, sign e^{+2 pi i}."""
    m = F.shape[0]
    out = np.zeros((m, m), dtype=np.complex128)
    for y in range(m):
        for x in range(m):
            acc = 0.0 + 0.0j
            for ky in range(m):
                for kx in range(m):
                    ph = 2 * math.pi * (ky * y + kx * x) / m
                    acc += F[ky, kx] * complex(math.cos(ph), math.sin(ph))
            out[y, x] = acc / m
    return out


# ------------------------------------------------------------------ centring
def test_centroid_of_point_and_two_points():
    w = np.zeros((16, 16), complex)
    w[3, 11] = 2.0 + 1.0j
    assert O.probe_centroid(w) == (3.0, 11.0)
    w[5, 11] = 1.0j                   # weights |w|^2 = 5 at row 3, 1 at row 5
    cy, cx = O.probe_centroid(w)
    assert abs(cy - (5 * 3 + 1 * 5) / 6) < 1e-15 and cx == 11.0


@pytest.mark.parametrize("d", [(5, -3), (0, 7), (-8, 0), (1, 1)])
def test_center_undoes_an_integer_roll(d):
    m = 64
    w = synth.gaussian_probe(m, 6.0, 3)                  # centred at m/2
    drifted = np.roll(w, d, axis=(0, 1))
    out, got = O.probe_center(drifted)
    assert got == d
    np.testing.assert_array_equal(out, w)


def test_center_leaves_a_centred_probe_alone():
    w = synth.gaussian_probe(128, 20.0, 5)
    out, d = O.probe_center(w)
    assert d == (0, 0)
    np.testing.assert_array_equal(out, w)


def test_centred_probe_has_centroid_within_half_a_pixel():
    rng = np.random.default_rng(4)
    m = 32
    for _ in range(5):
        w = synth.gaussian_probe(m, 4.0, rng) * (1 + 0.3 * rng.standard_normal((m, m)))
        w = np.roll(w, tuple(rng.integers(-6, 7, 2)), axis=(0, 1))
        out, _ = O.probe_center(w)
        cy, cx = O.probe_centroid(out)
        assert abs(cy - m / 2) <= 0.5 + 1e-12 and abs(cx - m / 2) <= 0.5 + 1e-12


# ------------------------------------------------------------------ Fourier constraints
def test_fourier_mask_against_bruteforce_transforms():
    m = 8
    rng = np.random.default_rng(1)
    w = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    mask = (rng.uniform(size=(m, m)) > 0.4).astype(float)
    ref = brute_idft2(brute_dft2(w) * mask)
    np.testing.assert_allclose(O.probe_fourier_mask(w, mask), ref, rtol=0, atol=1e-12)


def test_fourier_mask_identities():
    m = 16
    rng = np.random.default_rng(2)
    w = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    np.testing.assert_allclose(O.probe_fourier_mask(w, np.ones((m, m))), w, atol=1e-12)
    mask = (rng.uniform(size=(m, m)) > 0.5).astype(float)
    once = O.probe_fourier_mask(w, mask)
    np.testing.assert_allclose(O.probe_fourier_mask(once, mask), once, atol=1e-12)
    spec = brute_dft2(once)
    assert np.abs(spec[mask == 0]).max() < 1e-12


def test_fourier_amplitude_against_bruteforce_transforms():
    m = 8
    rng = np.random.default_rng(3)
    w = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    a_w = rng.uniform(0.1, 2.0, size=(m, m))
    W = brute_dft2(w)
    ref = brute_idft2(a_w * W / np.abs(W))
    np.testing.assert_allclose(O.probe_fourier_amplitude(w, a_w), ref, rtol=0, atol=1e-12)


def test_fourier_amplitude_identities():
    m = 16
    rng = np.random.default_rng(4)
    w = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    a_w = rng.uniform(0.0, 2.0, size=(m, m))
    out = O.probe_fourier_amplitude(w, a_w)
    np.testing.assert_allclose(np.abs(brute_dft2(out)), a_w, atol=1e-12)
    np.testing.assert_allclose(O.probe_fourier_amplitude(out, a_w), out, atol=1e-12)
    np.testing.assert_allclose(O.probe_fourier_amplitude(w, np.abs(brute_dft2(w))), w, atol=1e-12)
    # zero spectrum: phase 1, so the result is the inverse transform of a_w
    np.testing.assert_allclose(O.probe_fourier_amplitude(np.zeros((m, m)), a_w), brute_idft2(a_w), atol=1e-12)


# ------------------------------------------------------------------ initial illumination
def _probe_with_positive_spectrum(m, seed):
    """A probe whose centred spectrum is real and positive: the inverse DFT of
    a positive spectrum even in q (so the probe is real), rolled to the centre."""
    rng = np.random.default_rng(seed)
    S = rng.uniform(0.5, 2.0, size=(m, m))
    S = 0.5 * (S + np.roll(S[::-1, ::-1], 1, axis=(0, 1)))     # S(q) = S(-q)
    return np.roll(brute_idft2(S), (m // 2, m // 2), axis=(0, 1)), S


def test_mean_frame_init_recovers_a_probe_with_positive_centred_spectrum():
    m = 8
    w, S = _probe_with_positive_spectrum(m, 7)
    # identical frames of the probe over a unit object: a = |F w| = S
    a = np.stack([np.abs(brute_dft2(w))] * 3)
    np.testing.assert_allclose(a[0], S, atol=1e-12)
    np.testing.assert_allclose(O.probe_from_mean_frame(a), w, atol=1e-12)


def test_mean_frame_init_is_a_mean_not_a_sum():
    rng = np.random.default_rng(8)
    a = rng.uniform(0.0, 1.0, size=(3, 16, 16))
    w1 = O.probe_from_mean_frame(a)
    w2 = O.probe_from_mean_frame(np.concatenate([a, a]))
    np.testing.assert_allclose(w1, w2, atol=1e-13)
    # |F w0| is the root of the mean intensity, frame by frame of a 2-frame set
    a2 = np.stack([np.full((8, 8), 3.0), np.full((8, 8), 4.0)])
    np.testing.assert_allclose(np.abs(brute_dft2(O.probe_from_mean_frame(a2))), math.sqrt(12.5), atol=1e-12)


def test_threshold_init_closed_form():
    # m = 4, mean intensity with values 4 at q = 0 and 1 at the four nearest
    # neighbours (q = (0, +-1), (+-1, 0)); threshold 0.2 keeps those five, whose
    # mean is 1.6.  The centred inverse transform of sqrt(1.6) on that support
    # is (sqrt(1.6)/4) [1 + 2 cos(pi (x-2)/2) + 2 cos(pi (y-2)/2)].
    inten = np.zeros((4, 4))
    inten[0, 0] = 4.0
    for q in [(0, 1), (0, 3), (1, 0), (3, 0)]:
        inten[q] = 1.0
    inten[2, 2] = 0.5                  # below 0.2 * 4: dropped
    a = np.sqrt(inten)[None]
    out = O.probe_from_mean_frame(a, threshold=0.2)
    y, x = np.mgrid[0:4, 0:4]
    ref = math.sqrt(1.6) / 4 * (1 + 2 * np.cos(np.pi * (x - 2) / 2) + 2 * np.cos(np.pi * (y - 2) / 2))
    np.testing.assert_allclose(out, ref, atol=1e-14)


# ------------------------------------------------------------------ in the loop
def test_refinement_order_mask_then_centre():
    m = 16
    rng = np.random.default_rng(9)
    w = np.roll(synth.gaussian_probe(m, 2.0, 1), (3, -2), axis=(0, 1))
    mask = np.ones((m, m))
    mask[m // 2 - 2:m // 2 + 3, :] = 0.0        # drop a band of high frequencies
    got = O.refine_probe(w, probe_mask=mask, probe_com=True)
    ref, _ = O.probe_center(O.probe_fourier_mask(w, mask))
    np.testing.assert_allclose(got, ref, atol=1e-14)
    # a mask takes precedence over amplitudes
    got2 = O.refine_probe(w, probe_mask=mask, probe_amp=np.ones((m, m)))
    np.testing.assert_allclose(got2, O.probe_fourier_mask(w, mask), atol=1e-14)


def test_reconstruction_with_centring_keeps_the_probe_centred():
    s = synth.scan_tiny(m=16, n=32, rows=3, cols=3, step=4)
    a = O.forward_amplitudes(s.obj, s.probe, s.pos)
    w0 = np.roll(s.probe, (2, -1), axis=(0, 1))
    out = O.raar_reconstruct(a, s.pos, s.shape, w0, s.psi_init, 4, probe_every=2, probe_com=True,
                             record_metrics=False)
    cy, cx = O.probe_centroid(out["w"])
    assert abs(cy - 8) <= 0.5 and abs(cx - 8) <= 0.5


def test_exact_data_fixed_point_survives_refinement():
    s = synth.scan_tiny(m=16, n=32, rows=3, cols=3, step=4)
    a = O.forward_amplitudes(s.obj, s.probe, s.pos)
    a_w = np.abs(O.fft2u(s.probe))
    out = O.raar_reconstruct(a, s.pos, s.shape, s.probe, s.obj, 4, probe_every=1, probe_amp=a_w,
                             probe_com=True, record_metrics=False)
    np.testing.assert_allclose(out["w"], s.probe, atol=1e-10)
