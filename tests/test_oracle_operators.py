"""Pins of the oracle's operators against definitions that do not go through
the oracle: brute-force sums, closed forms, adjointness and projector
identities (Eqs. 2, 5, 7, 8, 9, 10 of arXiv:1602.01448)."""
import math

import numpy as np
import pytest

import oracle as O
import synth


def brute_dft2(f):
    """Unitary 2D DFT written out as the double sum, sign e^{-2 pi i}."""
    m = f.shape[0]
    out = np.zeros((m, m), dtype=np.complex128)
    for ky in range(m):
        for kx in range(m):
            acc = 0.0 + 0.0j
            for y in range(m):
                for x in range(m):
                    acc += f[y, x] * complex(math.cos(-2 * math.pi * (ky * y + kx * x) / m),
                                             math.sin(-2 * math.pi * (ky * y + kx * x) / m))
            out[ky, kx] = acc / m
    return out


@pytest.mark.parametrize("m", [4, 8, 16])
def test_fft_matches_bruteforce(m):
    z = synth.random_frames(1, m, 10 + m)[0]
    np.testing.assert_allclose(O.fft2u(z), brute_dft2(z), rtol=0, atol=1e-12)


def test_fft_sign_plane_wave():
    # e^{+2 pi i k0.r/m} must land on +k0 with value m (unitary scale) under
    # the e^{-2 pi i} forward transform: pins the sign reading of Eq. 2.
    m = 16
    ky0, kx0 = 3, 5
    y, x = np.mgrid[0:m, 0:m]
    f = np.exp(2j * np.pi * (ky0 * y + kx0 * x) / m)
    F = O.fft2u(f)
    expect = np.zeros((m, m), complex)
    expect[ky0, kx0] = m
    np.testing.assert_allclose(F, expect, atol=1e-12)


def test_fft_delta_and_parseval_and_inverse():
    m = 32
    d = np.zeros((m, m), complex)
    d[0, 0] = 1.0
    np.testing.assert_allclose(O.fft2u(d), np.full((m, m), 1.0 / m), atol=1e-15)
    z = synth.random_frames(3, m, 7)
    Z = O.fft2u(z)
    assert abs(O.norm(Z) - O.norm(z)) < 1e-12 * O.norm(z)
    np.testing.assert_allclose(O.ifft2u(Z), z, atol=1e-13)


def _tiny_geometry(wrap):
    rng = np.random.default_rng(3)
    m, shape = 5, (11, 13)
    if wrap:
        pos = np.array([[0, 0], [8, 10], [3, 11], [9, 2]], np.int32)
    else:
        pos = np.array([[0, 0], [6, 8], [3, 4], [2, 7]], np.int32)
    w = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    psi = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return m, shape, pos, w, psi


@pytest.mark.parametrize("wrap", [False, True])
def test_split_and_overlap_bruteforce(wrap):
    m, shape, pos, w, psi = _tiny_geometry(wrap)
    ny, nx = shape
    z = O.split(psi, w, pos, wrap)
    for i, (r0, c0) in enumerate(pos):
        for y in range(m):
            for x in range(m):
                assert abs(z[i, y, x] - w[y, x] * psi[(r0 + y) % ny, (c0 + x) % nx]) < 1e-14
    zz = synth.random_frames(len(pos), m, 5)
    img = np.zeros(shape, complex)
    D = np.zeros(shape)
    for i, (r0, c0) in enumerate(pos):
        for y in range(m):
            for x in range(m):
                img[(r0 + y) % ny, (c0 + x) % nx] += np.conj(w[y, x]) * zz[i, y, x]
                D[(r0 + y) % ny, (c0 + x) % nx] += abs(w[y, x]) ** 2
    np.testing.assert_allclose(O.overlap(zz, w, pos, shape, wrap), img, atol=1e-12)
    np.testing.assert_allclose(O.illumination(w, pos, shape, wrap), D, atol=1e-12)


def test_split_rejects_out_of_range_without_wrap():
    m, shape, pos, w, psi = _tiny_geometry(True)
    with pytest.raises(ValueError):
        O.split(psi, w, pos, wrap=False)


@pytest.mark.parametrize("wrap", [False, True])
def test_overlap_is_adjoint_of_split(wrap):
    m, shape, pos, w, psi = _tiny_geometry(wrap)
    z = synth.random_frames(len(pos), m, 9)
    lhs = np.vdot(O.split(psi, w, pos, wrap).ravel(), z.ravel())
    rhs = np.vdot(psi.ravel(), O.overlap(z, w, pos, shape, wrap).ravel())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # D = Q*Q 1 through the operators themselves
    ones = np.ones(shape, complex)
    np.testing.assert_allclose(O.overlap(O.split(ones, w, pos, wrap), w, pos, shape, wrap).real,
                               O.illumination(w, pos, shape, wrap), atol=1e-12)


def test_data_projection_properties():
    m = 16
    z = synth.random_frames(4, m, 1)
    a = synth.random_amplitudes(4, m, 2)
    p = O.data_project(z, a)
    np.testing.assert_allclose(np.abs(O.fft2u(p)), a, atol=1e-12)           # |F P_a z| = a
    np.testing.assert_allclose(O.data_project(p, a), p, atol=1e-12)         # idempotent
    np.testing.assert_allclose(O.data_project(z, np.abs(O.fft2u(z))), z, atol=1e-12)  # consistent z fixed
    # distance property: P_a z is the closest point of the constraint set
    q = O.ifft2u(a * np.exp(1j * np.random.default_rng(0).uniform(0, 2 * np.pi, a.shape)))
    assert O.norm(p - z) <= O.norm(q - z) + 1e-12


def test_data_projection_zero_modulus_reading():
    m = 8
    z = np.zeros((1, m, m), complex)
    a = synth.random_amplitudes(1, m, 4)
    # Fz = 0 everywhere: reading R3 gives Z' = a (phase 1)
    np.testing.assert_allclose(O.fft2u(O.data_project(z, a)), a.astype(complex), atol=1e-12)


def _scan(wrap=False):
    s = synth.scan_tiny(wrap=wrap)
    return s


def test_overlap_projection_properties():
    s = _scan()
    z = synth.random_frames(s.K, s.m, 3)
    pz = O.overlap_project(z, s.probe, s.pos, s.shape)
    np.testing.assert_allclose(O.overlap_project(pz, s.probe, s.pos, s.shape), pz, atol=1e-11)
    u = synth.random_frames(s.K, s.m, 4)
    pu = O.overlap_project(u, s.probe, s.pos, s.shape)
    assert abs(np.vdot(pu.ravel(), z.ravel()) - np.vdot(u.ravel(), pz.ravel())) < 1e-10 * O.norm(u) * O.norm(z)
    # (I - P_Q) z is orthogonal to range(Q)
    resid = z - pz
    psi = synth.random_frames(1, s.shape[0], 5)[0]
    assert abs(np.vdot(O.split(psi, s.probe, s.pos).ravel(), resid.ravel())) < 1e-10 * O.norm(z) * O.norm(psi)
    # range(Q) is fixed
    qpsi = O.split(s.obj, s.probe, s.pos)
    np.testing.assert_allclose(O.overlap_project(qpsi, s.probe, s.pos, s.shape), qpsi, atol=1e-11)


def test_object_update_recovers_visited_pixels_and_zeroes_the_rest():
    s = _scan()
    z = O.split(s.obj, s.probe, s.pos)
    psi = O.object_update(z, s.probe, s.pos, s.shape)
    D = O.illumination(s.probe, s.pos, s.shape)
    vis = D > 1e-12 * D.max()
    np.testing.assert_allclose(psi[vis], s.obj[vis], rtol=1e-10)
    assert np.all(psi[~vis] == 0)
    assert (~vis).any()


def test_probe_update_bruteforce_and_fixed_point():
    s = _scan()
    z = O.split(s.obj, s.probe, s.pos)
    w = O.probe_update(z, s.obj, s.pos, np.zeros_like(s.probe))
    np.testing.assert_allclose(w, s.probe, rtol=1e-10, atol=1e-14)
    # brute force on random data
    rng = np.random.default_rng(8)
    zz = synth.random_frames(s.K, s.m, 8)
    psi = rng.standard_normal(s.shape) + 1j * rng.standard_normal(s.shape)
    num = np.zeros((s.m, s.m), complex)
    den = np.zeros((s.m, s.m))
    for i, (r0, c0) in enumerate(s.pos):
        for y in range(s.m):
            for x in range(s.m):
                num[y, x] += np.conj(psi[r0 + y, c0 + x]) * zz[i, y, x]
                den[y, x] += abs(psi[r0 + y, c0 + x]) ** 2
    np.testing.assert_allclose(O.probe_update(zz, psi, s.pos, s.probe), num / den, rtol=1e-11)


def test_probe_update_keeps_old_value_where_object_is_zero():
    s = _scan()
    psi = np.zeros(s.shape, complex)
    w_old = s.probe * 3.0
    z = synth.random_frames(s.K, s.m, 1)
    np.testing.assert_array_equal(O.probe_update(z, psi, s.pos, w_old), w_old)
