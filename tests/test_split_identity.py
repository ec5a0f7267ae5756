"""The radix-2 split of the unitary 256^2 transform (Eq. 2) that the 256^2
frame passes use, checked on the CPU against numpy's FFT.

With n = nu + 128 p, k = 2 kappa + a per axis and omega = exp(-2 pi i / 256):
  forward:  Z[2 kappa1 + a][2 kappa2 + b] = X_ab[kappa1][kappa2] / 256,
            X_ab the raw 128^2 DFT of
            y_ab[nu1][nu2] = omega^(a nu1 + b nu2) sum_pq (-1)^(a p + b q) z[nu1 + 128 p][nu2 + 128 q];
  inverse:  c[nu1 + 128 p][nu2 + 128 q]
            = 1/256 sum_ab (-1)^(a p + b q) omega^-(a nu1 + b nu2) R_ab[nu1][nu2],
            R_ab the raw (unnormalised) inverse 128^2 DFT of U_ab[kappa1][kappa2] = U[2 kappa1 + a][2 kappa2 + b].
A wrong sign, a swapped parity or a missing twiddle in either direction fails
these checks (the cases below perturb each in turn).
"""
import numpy as np
import pytest

M, H = 256, 128


def _omega(e):
    return np.exp(-2j * np.pi * e / M)


def split_forward(z, sign_fix=1, twiddle=True):
    nu = np.arange(H)
    Z = np.empty((M, M), complex)
    for a in (0, 1):
        for b in (0, 1):
            y = sum(((-1) ** (a * p + b * q)) * z[H * p:H * p + H, H * q:H * q + H]
                    for p in (0, 1) for q in (0, 1))
            if twiddle:
                y = y * _omega(sign_fix * a * nu)[:, None] * _omega(sign_fix * b * nu)[None, :]
            Z[a::2, b::2] = np.fft.fft2(y) / M
    return Z


def split_inverse(U, parity_swap=False):
    nu = np.arange(H)
    c = np.zeros((M, M), complex)
    for a in (0, 1):
        for b in (0, 1):
            ua, ub = (b, a) if parity_swap else (a, b)
            R = np.fft.ifft2(U[ua::2, ub::2]) * (H * H)          # raw inverse
            R = R * _omega(-a * nu)[:, None] * _omega(-b * nu)[None, :]
            for p in (0, 1):
                for q in (0, 1):
                    c[H * p:H * p + H, H * q:H * q + H] += ((-1) ** (a * p + b * q)) * R / M
    return c


def _frame(seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))


def test_forward_split_is_the_unitary_transform():
    z = _frame(1)
    Z = np.fft.fft2(z) / M                     # unitary 256^2 transform
    assert np.abs(split_forward(z) - Z).max() < 1e-12 * np.abs(Z).max()


def test_inverse_split_is_the_unitary_inverse():
    U = _frame(2)
    c = np.fft.ifft2(U) * M                    # unitary inverse
    assert np.abs(split_inverse(U) - c).max() < 1e-12 * np.abs(c).max()


def test_round_trip_through_both_splits():
    z = _frame(3)
    assert np.abs(split_inverse(split_forward(z)) - z).max() < 1e-12 * np.abs(z).max()


@pytest.mark.parametrize("case", ["twiddle sign", "no twiddle", "parity swap"])
def test_plausible_mistakes_fail(case):
    z = _frame(4)
    Z = np.fft.fft2(z) / M
    if case == "twiddle sign":
        bad = split_forward(z, sign_fix=-1)
        assert np.abs(bad - Z).max() > 1e-3 * np.abs(Z).max()
    elif case == "no twiddle":
        bad = split_forward(z, twiddle=False)
        assert np.abs(bad - Z).max() > 1e-3 * np.abs(Z).max()
    else:
        c = np.fft.ifft2(Z) * M
        bad = split_inverse(Z, parity_swap=True)
        assert np.abs(bad - c).max() > 1e-3 * np.abs(c).max()
