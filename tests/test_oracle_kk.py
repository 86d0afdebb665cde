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


def test_rrc_amplitude_values():
    f = np.array([0.0, 0.3, 0.494, 0.5, 0.506, 2.0]) * 1e9
    h = K.rrc_amplitude(f, 1e9, 0.01)
    assert np.allclose(h, [1.0, 1.0, 1.0, math.sqrt(0.5), 0.0, 0.0], atol=1e-12)


def test_static_eq_with_unit_response_decimates_a_band_limited_signal():
    """Tones on the block's bin grid inside |f| < fs/4: every interior block
    sees whole periods, and cutting the band then halving the DFT size is
    exact decimation, x2[m] = x4[2m]."""
    rng = np.random.default_rng(8)
    N4 = 1024
    n4 = 12 * N4
    t = np.arange(n4)
    x4 = np.zeros(n4, dtype=np.complex128)
    for k in rng.integers(-N4 // 4 + 1, N4 // 4, 12):
        x4 += (rng.standard_normal() + 1j * rng.standard_normal()) * np.exp(2j * math.pi * k * t / N4)
    x2 = K.static_eq_resample(x4, np.ones(N4 // 2, dtype=np.complex128))
    sl = slice(N4 // 4, x2.size - N4 // 2)
    assert np.max(np.abs(x2[sl] - x4[::2][sl])) < 1e-11


def test_static_eq_undoes_the_simulated_dispersion():
    """The simulator's field (dispersed with the carrier at DC) downshifted:
    with the matched filter made all-pass (a symbol rate far above the band)
    the equaliser is the CD compensation alone (about a sample of spread and
    a 0.56-sample delay from the carrier offset at 2,000 km; overlap-save
    leaves the ringing of the phase's band-edge step, ~1e-3), and it returns
    the undispersed carrier tone plus signal at every other sample
    (whole-array reference); no compensation, or the opposite sign, is two
    orders of magnitude worse."""
    d = rxsim.simulate_kk(rxsim.KKLinkConfig(n_sym=1 << 12, snr_db=None, fiber_len_m=2000e3, seed=5))
    fs, fc = d["fs"], d["f_c"]
    t = np.arange(d["field"].size)
    down = np.exp(-2j * math.pi * fc / fs * t)
    b2 = rxsim.beta2_from_dispersion(17.0, 1550e-9)
    N4 = 1024
    H = K.static_eq_response(N4, fs, 1e12, 0.01, b2, 2000e3, fc)
    x2 = K.static_eq_resample(d["field"] * down, H)
    ref = ((d["carrier"] + d["signal"] * np.exp(2j * math.pi * fc / fs * t)) * down)[::2]
    sl = slice(N4 // 2, x2.size - N4)
    top = np.max(np.abs(ref))
    assert np.max(np.abs(x2[sl] - ref[sl])) < 2e-3 * top
    x0 = K.static_eq_resample(d["field"] * down, np.ones(N4 // 2, dtype=np.complex128))
    assert np.max(np.abs(x0[sl] - ref[sl])) > 0.1 * top
    xm = K.static_eq_resample(d["field"] * down, K.static_eq_response(N4, fs, 1e12, 0.01, b2, -2000e3, fc))
    assert np.max(np.abs(xm[sl] - ref[sl])) > 0.1 * top


def ideal_2sps(n_sym, bits_per_sym, seed):
    """Raised-cosine (RRC x RRC, roll-off 0.5) QPSK/16QAM at 2 samples per
    symbol, symbols at the even samples; returns (signal, symbols)."""
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 2, n_sym * bits_per_sym).astype(np.uint8)
    sym = rxsim.gray_map(bits, bits_per_sym)
    up = np.zeros(2 * n_sym, dtype=np.complex128)
    up[::2] = sym
    f = np.fft.fftfreq(2 * n_sym, d=0.5)
    x = np.fft.ifft(np.fft.fft(up) * K.rrc_amplitude(f, 1.0, 0.5) ** 2) * 2
    return x, sym


def test_widely_linear_equaliser_removes_iq_imbalance():
    """x = s + beta conj(s) (modulator IQ imbalance): the widely-linear DD-LMS
    drives the residual far below |beta|^2, where a strictly linear one
    (h2 = 0) stays (the conjugate term is orthogonal to every linear
    filter of s); a sign error in either gradient would not converge."""
    x, sym = ideal_2sps(1 << 14, 2, 11)
    beta = 0.12 * np.exp(0.7j)
    xi = x + beta * np.conj(x)
    res = {}
    for lin in (False, True):
        y, _ = K.wl_equalise(xi, sym.size, 2, 5e-2, 64, 512, 1 << 13, 8192, linear_only=lin)
        res[lin] = float(np.mean(np.abs(y[8192:] - sym[8192:]) ** 2))
    assert res[False] < 2e-4
    assert abs(res[True] - abs(beta) ** 2) < 0.1 * abs(beta) ** 2


def test_widely_linear_equaliser_keeps_an_ideal_input():
    x, sym = ideal_2sps(1 << 13, 4, 12)
    y, chains = K.wl_equalise(x, sym.size, 4, 2e-3, 64, 512, 1 << 12, 4096)
    assert np.max(np.abs(y - sym)) < 1e-6
    h1, h2 = chains[0]
    assert abs(h1[K.WL_CENTRE] - 1) < 1e-6 and np.max(np.abs(h2)) < 1e-6


def test_noiseless_kk_link_decodes_without_errors():
    d = rxsim.simulate_kk(rxsim.KKLinkConfig(n_sym=1 << 14, snr_db=None, cspr_db=14.0, fiber_len_m=1000e3,
                                             seed=13, prbs_seed=13))
    b2 = rxsim.beta2_from_dispersion(17.0, 1550e-9)
    r = K.kk_receive(d["codes"], d["gain"], d["offset"], d["fs"], d["f_c"], 1024, 1024, 1e9, 0.01, b2, 1000e3,
                     2, 5e-3, 64, 512, 1 << 13, 4096)
    # the first and last 64 symbols see blocks that run past the stream's
    # ends (zero-padded log amplitude and field)
    a, e = 2 * 64, r["bits"].size - 2 * 64
    assert np.array_equal(r["bits"][a:e], d["bits"][a:e])
