"""The scale of the intermediate between a transform's two contractions in the
FP16-scaled tensor-core mode (Eq. 2 as a contraction with the unitary
128-point DFT matrix F): every component of F z is at most sqrt(2 * 128) = 16
times the largest component of z, so an operand whose largest component is
below 2^15 stays below 2^15 after F and a factor 2^-4.  An adversarial input
comes within 10 % of the bound, so a factor 2^-3 could leave FP16's range
(65504).
"""
import numpy as np

N = 128


def unitary_dft(n):
    k = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(k, k) / n) / np.sqrt(n)


def max_component(x):
    return max(np.abs(x.real).max(), np.abs(x.imag).max())


def test_bound_holds_for_random_columns():
    F = unitary_dft(N)
    rng = np.random.default_rng(7)
    for _ in range(20):
        z = rng.uniform(-1, 1, (N, N)) + 1j * rng.uniform(-1, 1, (N, N))
        assert max_component(F @ z) <= 16.0 * max_component(z)


def test_adversarial_column_comes_close_to_the_bound():
    F = unitary_dft(N)
    k = 1
    # real part of (F z)_k = sum_n (Re F_kn Re z_n - Im F_kn Im z_n), maximised
    # by z_n = sign(Re F_kn) - i sign(Im F_kn)
    z = np.sign(F[k].real) - 1j * np.sign(F[k].imag)
    ratio = abs((F @ z)[k].real) / max_component(z)
    assert 14.0 < ratio <= 16.0
    # 2^15 scaled by 2^-3 would reach 2^15 * 14 / 8 > 65504
    assert 2.0 ** 15 * ratio / 8.0 > 65504.0
    assert 2.0 ** 15 * 16.0 / 16.0 <= 2.0 ** 15
