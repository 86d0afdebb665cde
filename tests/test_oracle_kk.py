"""Pins of the Kramers-Kronig front-end oracle against closed forms, a
library routine and the minimum-phase condition (no GPU)."""
import math

import numpy as np
import pytest

import rxsim
from oracle import kk_oracle as K


def multitone(n, N, A, tones):
    """E_t = A + sum_k B_k exp(j 2 pi m_k t / N): N-periodic, spectrum on the
    positive side of the real carrier A."""
    t = np.arange(n)
    E = np.full(n, A, dtype=np.complex128)
    for m, B in tones:
        E += B * np.exp(2j * math.pi * m * t / N)
    return E


@pytest.mark.parametrize("N", [1024, 2048, 4096])
def test_minimum_phase_multitone_is_reconstructed_exactly(N):
    """sum |B_k| < A: ln E = ln A + sum_n c_n e^{j n w t} has only positive
    frequencies, so phi = H{ln|E|} is arg E exactly; with tones at 1, 3 and
    7 periods per block the harmonics that alias are below 1e-30.  Interior
    blocks hold a whole period, so overlap-save is exact there."""
    n = 8 * N
    E = multitone(n, N, 1.0, [(1, 0.3), (3, 0.2j), (7, -0.1)])
    for nu in (0.0, 0.129):
        got = K.kk_field_from_intensity(np.abs(E) ** 2, 1e-300, N, nu)
        want = E * np.exp(-2j * math.pi * nu * np.arange(n))
        sl = slice(N // 2, n - N)
        assert np.max(np.abs(got[sl] - want[sl])) < 1e-12


def test_reconstruction_fails_without_the_minimum_phase_condition():
    N = 1024
    n = 8 * N
    E = multitone(n, N, 1.0, [(3, 1.5)])  # |B| > A: the field winds round 0
    got = K.kk_field_from_intensity(np.abs(E) ** 2, 1e-300, N, 0.0)
    sl = slice(N // 2, n - N)
    assert np.linalg.norm(got[sl] - E[sl]) / np.linalg.norm(E[sl]) > 0.3


def test_overlap_save_hilbert_equals_the_whole_array_transform_on_periodic_input():
    """scipy.signal.hilbert (one FFT over the whole array) of an N-periodic
    real signal equals the block-wise transform on samples whose block lies
    inside the stream."""
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(4)
    N = 1024
    period = rng.standard_normal(N)
    u = np.tile(period, 6)
    got = K.ols_hilbert(u, N)
    want = np.imag(signal.hilbert(u))
    sl = slice(N // 2, u.size - N)
    assert np.max(np.abs(got[sl] - want[sl])) < 1e-12


def test_hilbert_multiplier_turns_cos_into_sin():
    N = 64
    t = np.arange(N)
    for m in (1, 5, 31):
        x = np.cos(2 * math.pi * m * t / N)
        h = np.real(np.fft.ifft(np.fft.fft(x) * K.hilbert_multiplier(N)))
        assert np.max(np.abs(h - np.sin(2 * math.pi * m * t / N))) < 1e-13
    # DC and Nyquist components carry no Hilbert transform
    x = 1.0 + np.cos(math.pi * t)
    assert np.max(np.abs(np.fft.ifft(np.fft.fft(x) * K.hilbert_multiplier(N)))) < 1e-13


def test_adc_conversion_and_floor():
    codes = np.array([0, 1, 7, 4095, 2048], dtype=np.int16)
    I = K.adc_to_intensity(codes, 0.25, 3.0)
    assert np.allclose(I, [-0.75, -0.5, 1.0, 1023.0, 511.25], rtol=0, atol=1e-15)
    u = K.log_amplitude(I, 0.125)
    assert np.allclose(np.exp(2 * u), [0.125, 0.125, 1.0, 1023.0, 511.25], rtol=1e-15)


def test_simulated_link_is_reconstructed_better_at_higher_cspr():
    """The paper's signal (1 GBd, 1 % roll-off, 4 GS/s, tone 0.516 GHz from
    the signal centre), noiseless: the downshifted field approaches the
    transmitted carrier plus signal as the CSPR grows (the minimum-phase
    condition is violated less often)."""
    errs = []
    for cspr in (8.0, 14.0):
        d = rxsim.simulate_kk(rxsim.KKLinkConfig(n_sym=1 << 13, snr_db=None, cspr_db=cspr))
        nu = d["f_c"] / d["fs"]
        E = K.kk_field(d["codes"], d["gain"], d["offset"], 1024, nu)
        ref = d["field"] * np.exp(-2j * math.pi * nu * np.arange(E.size))
        sl = slice(1024, E.size - 1024)
        errs.append(np.linalg.norm(E[sl] - ref[sl]) / np.linalg.norm(ref[sl]))
    assert errs[1] < 5e-3 < errs[0] < 5e-2


def test_impulse_response_follows_the_block_geometry():
    """u = delta at p: segment b (outputs [bL, bL + L), L = N/2) sees it only
    when its block [bL - N/4, bL + 3N/4) holds p, and there the circular
    Hilbert transform of a delta is (2/N) cot(pi m / N) for odd m = t - p
    and 0 for even m."""
    N = 256
    L = N // 2
    n = 10 * L
    for p in (0, 5, 300, 383, 384, 700):
        u = np.zeros(n)
        u[p] = 1.0
        phi = K.ols_hilbert(u, N)
        want = np.zeros(n)
        for t in range(n):
            b = t // L
            if b * L - N // 4 <= p < b * L + 3 * N // 4:
                m = t - p
                if m % 2:
                    want[t] = 2.0 / N / math.tan(math.pi * m / N)
        assert np.max(np.abs(phi - want)) < 1e-13, p
