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

Every number is FP64.  Library primitive used: numpy FFT.
"""
from __future__ import annotations

import math

import numpy as np

PIN_STATUS = {
    "adc_to_intensity": "pinned: codes map linearly; codes at or below the offset give the floor",
    "ols_hilbert": "pinned: equals scipy's whole-array FFT Hilbert transform on an N-periodic input",
    "kk_field": "pinned: exact reconstruction of minimum-phase multitones (1e-10); fails without the "
                "minimum-phase condition; the downshift moves the tone at nu to DC",
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
