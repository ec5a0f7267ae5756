"""The scale of the intermediate between a transform's two contractions in the
FP16-scaled tensor-core mode (Eq. 2 as a contraction with the unitary
128-point DFT matrix F): every component of F z is at most
128 * sqrt(2) / sqrt(128) = sqrt(2 * 128) = 16 times the largest component of
z (|Re F| + |Im F| <= sqrt(2 / 128)), so an operand whose largest component
is below 2^15 stays below 2^15 after F and a factor 2^-4.  The largest ratio
an input attains is about 4 sqrt(128) / pi = 14.4 (the mean of
|cos| + |sin| is 4 / pi), within 10 % of the bound.  FP16 rounding is
relative, so the spare range costs no precision.
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


def test_adversarial_columns_stay_below_the_bound():
    F = unitary_dft(N)
    worst = 0.0
    for k in range(N):
        # Re (F z)_k = sum_n (Re F_kn Re z_n - Im F_kn Im z_n) is largest for
        # z_n = sign(Re F_kn) - i sign(Im F_kn); Im (F z)_k likewise
        zr = np.sign(F[k].real) - 1j * np.sign(F[k].imag)
        zi = np.sign(F[k].imag) + 1j * np.sign(F[k].real)
        for z in (zr, zi):
            y = (F @ z)[k]
            worst = max(worst, max(abs(y.real), abs(y.imag)) / max_component(z))
    assert worst <= 16.0
    assert abs(worst - 4.0 * np.sqrt(N) / np.pi) < 0.05       # k = 1: 14.40
    # with inputs below 2^15 and the factor 2^-4 the operand stays below 2^15
    assert 2.0 ** 15 * worst / 16.0 < 2.0 ** 15
