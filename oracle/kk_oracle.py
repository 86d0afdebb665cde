"""FP64 oracle of the Kramers-Kronig front end -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The product path never does.

The steps (paper Sec. II, the real-time KK receiver; field reconstruction
after Mecozzi et al.):

  k1  ADC codes to intensity: I_t = gain (code_t - offset) (12-bit fixed
      point to floating point); the log amplitude u_t = ln sqrt(max(I_t, I_min))
      = ln(max(I_t, I_min)) / 2 with I_min = gain / 2 (half a code step, so
      that the log of an empty sample stays finite).
  k2  phase retrieval by a frequency-domain Hilbert transform of u in
      100 % overlap-save blocks of N samples (paper: N = 1024): segment b
      holds output samples [b N/2, (b+1) N/2); its block is the input
      u over [b N/2 - N/4, b N/2 + 3N/4) (zero outside the stream), whose
      DFT is multiplied by -j sgn(k) (0 at k = 0 and k = N/2), transformed
      back, and samples N/4 .. 3N/4 - 1 of the real part are the segment's
      phase phi.
  k3  field reconstruction E_t = exp(u_t + j phi_t) = sqrt(max(I_t, I_min))
      e^{j phi_t}, then the downshift to DC: E_t exp(-j 2 pi nu t) with
      nu = f_shift / f_s and t the absolute sample index.

  k4  static equaliser and resampling: 100 % overlap-save at 4 samples per
      symbol, each block's DFT cut to the 2-samples-per-symbol band and
      multiplied by the CD compensation times the RRC matched filter, then an
      inverse DFT of half the size.
  k5  widely-linear DD-LMS, 4 taps at 2 samples per symbol on x and on
      conj(x) (it corrects IQ imbalance of the modulator), block-LMS on the
      dual-polarisation equaliser's schedule (acquisition chain, then
      segment chains continued from frame to frame).
  k6  hard decisions and Gray demapping.

Every number is FP64.  Library primitives used: numpy FFT, matrix products.
"""
from __future__ import annotations

import math

import numpy as np

from .rx_oracle import decide, demap

PIN_STATUS = {
    "adc_to_intensity": "pinned: codes map linearly; codes at or below the offset give the floor",
    "ols_hilbert": "pinned: equals scipy's whole-array FFT Hilbert transform on an N-periodic input",
    "kk_field": "pinned: exact reconstruction of minimum-phase multitones (1e-10); fails without the "
                "minimum-phase condition; the downshift moves the tone at nu to DC",
    "rrc_amplitude": "pinned: 1 in the passband, 0 in the stopband, sqrt(1/2) at Rs/2",
    "static_eq_resample": "pinned: H = 1 on a band-limited input is x4[2m] exactly; with the CD response it "
                          "undoes the simulator's dispersion (whole-array reference)",
    "wl_equalise": "pinned: removes an IQ imbalance a strictly linear equaliser cannot; keeps an ideal "
                   "input; the noiseless KK link decodes without errors",
}


def adc_to_intensity(codes: np.ndarray, gain: float, offset: float) -> np.ndarray:
    """I_t = gain (code_t - offset)."""
    return gain * (codes.astype(np.float64) - offset)


def log_amplitude(I: np.ndarray, I_min: float) -> np.ndarray:
    """u_t = ln(max(I_t, I_min)) / 2."""
    return 0.5 * np.log(np.maximum(I, I_min))


def hilbert_multiplier(N: int) -> np.ndarray:
    """-j sgn(k) over the N DFT bins (k < N/2 positive, k > N/2 negative);
    0 at DC and at the Nyquist bin."""
    h = np.zeros(N, dtype=np.complex128)
    h[1:N // 2] = -1j
    h[N // 2 + 1:] = 1j
    return h


def ols_hilbert(u: np.ndarray, N: int) -> np.ndarray:
    """phi over every sample of u by 100 % overlap-save blocks of N (k2)."""
    n = u.size
    L = N // 2
    H = hilbert_multiplier(N)
    phi = np.empty(n)
    for b in range((n + L - 1) // L):
        lo = b * L - N // 4
        blk = np.zeros(N)
        a, e = max(lo, 0), min(lo + N, n)
        blk[a - lo:e - lo] = u[a:e]
        ph = np.real(np.fft.ifft(np.fft.fft(blk) * H))
        m = min(L, n - b * L)
        phi[b * L:b * L + m] = ph[N // 4:N // 4 + m]
    return phi


def kk_field_from_intensity(I: np.ndarray, I_min: float, N: int, nu: float, t0: int = 0) -> np.ndarray:
    """k1 (after the ADC) to k3: the downshifted field of samples t0, t0 + 1, ..."""
    u = log_amplitude(I, I_min)
    phi = ols_hilbert(u, N)
    t = t0 + np.arange(I.size)
    return np.exp(u + 1j * phi) * np.exp(-2j * math.pi * nu * t)


def kk_field(codes: np.ndarray, gain: float, offset: float, N: int, nu: float) -> np.ndarray:
    """The KK front end from ADC codes to the downshifted field."""
    return kk_field_from_intensity(adc_to_intensity(codes, gain, offset), 0.5 * gain, N, nu)


# --------------------------------------------------------------------------
# k4 frequency-domain static equaliser with 4 -> 2 samples per symbol,
# k5 widely-linear DD-LMS, k6 decisions (paper Sec. II)
# --------------------------------------------------------------------------

def rrc_amplitude(f: np.ndarray, Rs: float, rho: float) -> np.ndarray:
    """Root-raised-cosine amplitude response, 1 in the passband."""
    a = np.abs(f) / Rs
    h = np.zeros_like(a)
    h[a <= (1 - rho) / 2] = 1.0
    mid = (a > (1 - rho) / 2) & (a <= (1 + rho) / 2)
    h[mid] = np.sqrt(0.5 * (1.0 + np.cos(math.pi / rho * (a[mid] - (1 - rho) / 2))))
    return h


def static_eq_response(N4: int, fs: float, Rs: float, rho: float, beta2: float, L: float, f_c: float) -> np.ndarray:
    """H over the N4/2 bins of the 2-sample-per-symbol band, in the order of
    an N4/2-point DFT (k = 0 .. N4/4 - 1, then -N4/4 .. -1; f_k = k fs / N4):
    CD compensation exp(+j beta2 L w^2 / 2) at w = 2 pi (f_k + f_c) (the
    dispersion acted on the field with the carrier at DC, the signal f_c
    above it) times the RRC matched filter; the phase is reduced mod 2 pi
    in FP64."""
    k = np.concatenate([np.arange(N4 // 4), np.arange(-(N4 // 4), 0)])
    f = k * fs / N4
    w = 2.0 * math.pi * (f + f_c)
    ph = np.mod(beta2 * L * w * w / 2.0, 2.0 * math.pi)
    return np.exp(1j * ph) * rrc_amplitude(f, Rs, rho)


def static_eq_resample(E4: np.ndarray, H2: np.ndarray) -> np.ndarray:
    """k4: 100 % overlap-save at 4 samples per symbol, blocks of N4 = 2 H2.size
    advancing by N4/2; each block's N4-point DFT is cut to the 2-sps band
    (bins -N4/4 .. N4/4 - 1), multiplied by H2 and transformed back with an
    N4/2-point inverse DFT (x2[m] = x4[2m] for a band-limited x4, hence the
    factor 1/2); block b gives 2-sps outputs [b N4/4, (b+1) N4/4) from its
    samples N4/8 .. 3 N4/8 - 1 (the block spans 4-sps input
    [b N4/2 - N4/4, b N4/2 + 3 N4/4), zero outside the stream)."""
    N4 = 2 * H2.size
    L4, L2 = N4 // 2, N4 // 4
    n4 = E4.size
    n2 = n4 // 2
    out = np.empty(n2, dtype=np.complex128)
    for b in range((n2 + L2 - 1) // L2):
        lo = b * L4 - N4 // 4
        blk = np.zeros(N4, dtype=np.complex128)
        a, e = max(lo, 0), min(lo + N4, n4)
        blk[a - lo:e - lo] = E4[a:e]
        X = np.fft.fft(blk)
        X2 = np.concatenate([X[:N4 // 4], X[N4 - N4 // 4:]]) * H2
        y = np.fft.ifft(X2) / 2.0
        m = min(L2, n2 - b * L2)
        out[b * L2:b * L2 + m] = y[N4 // 8:N4 // 8 + m]
    return out


WL_TAPS = 4        # taps per filter at 2 samples per symbol (paper: 4-tap equaliser)
WL_CENTRE = 1      # tap t reads x[2k + t - WL_CENTRE]


def wl_fir(h1: np.ndarray, h2: np.ndarray, x: np.ndarray, k0: int, k1: int):
    """y_k = sum_t h1[t] x[2k+t-c] + h2[t] conj(x[2k+t-c]) for k0 <= k < k1
    (x = 0 outside the stream); returns y and the tap inputs X[k, t]."""
    n = x.size
    k = np.arange(k0, k1)
    idx = 2 * k[:, None] + np.arange(WL_TAPS)[None, :] - WL_CENTRE
    X = np.where((idx >= 0) & (idx < n), x[np.clip(idx, 0, n - 1)], 0.0)
    return X @ h1 + np.conj(X) @ h2, X


def wl_sub_block(h1, h2, x, k0, k1, mu, bits_per_sym):
    """One block-LMS step of the widely-linear DD equaliser over [k0, k1):
    outputs with fixed taps, e = y - dec(y), g1[t] = mean e conj(X[:, t]),
    g2[t] = mean e X[:, t] (the gradients of |e|^2 / 2 with respect to
    conj(h1), conj(h2)), h <- h - mu g."""
    y, X = wl_fir(h1, h2, x, k0, k1)
    e = y - decide(y, bits_per_sym)
    K = k1 - k0
    g1 = (e[:, None] * np.conj(X)).sum(axis=0) / K
    g2 = (e[:, None] * X).sum(axis=0) / K
    return h1 - mu * g1, h2 - mu * g2, y


def wl_equalise(x2: np.ndarray, n_sym: int, bits_per_sym: int, mu: float, K: int, S: int, F: int,
                acq_syms: int, linear_only: bool = False):
    """k5 on the same schedule as the dual-polarisation equaliser: one
    sequential chain of sub-blocks of K symbols over the first acq_syms
    symbols (from h1 = unit tap at offset 0, h2 = 0), then every frame of F
    symbols is cut into segments of S and segment j continues the taps of
    segment j of the previous frame (frame 0: the acquisition's taps).
    Returns the equalised symbols of the segment passes and the final taps.
    linear_only keeps h2 at 0 (a strictly linear equaliser, for the pins)."""
    h1 = np.zeros(WL_TAPS, dtype=np.complex128)
    h1[WL_CENTRE] = 1.0
    h2 = np.zeros(WL_TAPS, dtype=np.complex128)

    def step(a, b, k0, k1):
        a, b, y = wl_sub_block(a, b, x2, k0, k1, mu, bits_per_sym)
        return a, (b * 0 if linear_only else b), y

    acq = min(acq_syms, n_sym)
    for k0 in range(0, acq, K):
        h1, h2, _ = step(h1, h2, k0, min(k0 + K, acq))
    y_all = np.zeros(n_sym, dtype=np.complex128)
    chains = {}
    for f0 in range(0, n_sym, F):
        Ff = min(F, n_sym - f0)
        for j in range((Ff + S - 1) // S):
            a, b = chains.get(j, (h1, h2))
            for k0 in range(f0 + j * S, min(f0 + (j + 1) * S, f0 + Ff), K):
                k1 = min(k0 + K, f0 + (j + 1) * S, f0 + Ff)
                a, b, y = step(a, b, k0, k1)
                y_all[k0:k1] = y
            chains[j] = (a, b)
    return y_all, chains


def kk_receive(codes, gain, offset, fs, f_c, N, N4, Rs, rho, beta2, L, bits_per_sym, mu, K, S, F, acq_syms):
    """The whole KK chain of the paper: field (k1-k3), static equaliser and
    resampling (k4), widely-linear DD-LMS (k5), decisions and Gray demap
    (k6: bits per symbol, I bits then Q bits, MSB first)."""
    E4 = kk_field(codes, gain, offset, N, f_c / fs)
    x2 = static_eq_resample(E4, static_eq_response(N4, fs, Rs, rho, beta2, L, f_c))
    n_sym = x2.size // 2
    y, chains = wl_equalise(x2, n_sym, bits_per_sym, mu, K, S, F, acq_syms)
    return {"field": E4, "x2": x2, "y": y, "bits": demap(y, bits_per_sym).reshape(-1), "chains": chains}
