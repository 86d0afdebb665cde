"""Forward model of the paper's single-polarisation minimum-phase link for a
Kramers-Kronig receiver (FP64, numpy; paper Sec. II, Fig. 1).

Circular (full-length FFT) operations over the whole sequence, so the
generated stream is periodic in the sample count.  Steps, in order:

1. payload bits: PRBS-31 (the dual-polarisation simulator's x sequence);
2. Gray mapping (QPSK / 16QAM, unit mean symbol energy);
3. `sps` samples per symbol, root-raised-cosine pulse shaping in the
   frequency domain (paper: 1 GBd, 1 % roll-off, 4 GS/s);
4. the signal is placed f_c above a real, positive carrier tone of power
   CSPR x signal power: E(t) = A + s(t) exp(j 2 pi f_c t) (the carrier frame;
   paper: signal up to 0.505 GHz, tone 0.516 GHz from the signal centre);
5. chromatic dispersion exp(-j beta2 L w^2 / 2) on the whole field;
6. complex AWGN of per-sample variance Ps / SNR (optical noise);
7. square-law detection I = |E|^2 and a 12-bit ADC:
   code = clip(round(I / gain + offset), 0, 4095), gain chosen so that the
   largest intensity sits 2 % below full scale.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .channel import _fftn, _ifftn, _rrc_amplitude, beta2_from_dispersion, gray_map, pol_seed_state, prbs31


@dataclasses.dataclass
class KKLinkConfig:
    baud_hz: float = 1e9
    sps: int = 4
    bits_per_sym: int = 2
    n_sym: int = 1 << 16
    rolloff: float = 0.01
    f_c_hz: float = 0.516e9          # signal centre above the carrier
    cspr_db: float = 10.0            # carrier to signal power ratio
    fiber_len_m: float = 0.0
    D_ps_nm_km: float = 17.0
    lambda_m: float = 1550e-9
    snr_db: float | None = 25.0      # signal power / noise power per sample; None: noiseless
    adc_offset: float = 0.0          # code of zero intensity
    prbs_seed: int = 1
    seed: int = 0


def simulate_kk(cfg: KKLinkConfig) -> dict:
    rng = np.random.default_rng(cfg.seed)
    n = cfg.n_sym * cfg.sps
    fs = cfg.baud_hz * cfg.sps
    bits = prbs31(pol_seed_state(cfg.prbs_seed, 0), cfg.n_sym * cfg.bits_per_sym)
    sym = gray_map(bits, cfg.bits_per_sym)
    up = np.zeros(n, dtype=np.complex128)
    up[::cfg.sps] = sym
    f = np.fft.fftfreq(n, d=1.0 / fs)
    s = _ifftn(_fftn(up) * _rrc_amplitude(f, cfg.baud_hz, cfg.rolloff)) * cfg.sps
    ps = float(np.mean(np.abs(s) ** 2))
    A = math.sqrt(ps * 10.0 ** (cfg.cspr_db / 10.0))
    t = np.arange(n)
    E = A + s * np.exp(2j * math.pi * (cfg.f_c_hz / fs) * t)
    if cfg.fiber_len_m:
        b2 = beta2_from_dispersion(cfg.D_ps_nm_km, cfg.lambda_m)
        w = 2.0 * math.pi * f
        E = _ifftn(_fftn(E) * np.exp(-1j * b2 * cfg.fiber_len_m * w * w / 2.0))
    if cfg.snr_db is not None:
        sig = math.sqrt(ps / 10.0 ** (cfg.snr_db / 10.0) / 2.0)
        E = E + sig * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    inten = np.abs(E) ** 2
    gain = float(inten.max()) / (0.98 * (4095.0 - cfg.adc_offset))
    codes = np.clip(np.rint(inten / gain + cfg.adc_offset), 0, 4095).astype(np.int16)
    return {"codes": codes, "gain": gain, "offset": cfg.adc_offset, "fs": fs, "f_c": cfg.f_c_hz,
            "field": E, "carrier": A, "signal": s, "symbols": sym, "bits": bits}
