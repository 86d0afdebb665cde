"""Forward model of a dual-polarisation coherent optical link (FP64, numpy).

The transmitter, fibre and receiver front end are simulated with circular
(full-length FFT) operations over the whole sequence, so the generated
stream is periodic in the symbol count.  Steps, in order:

1. payload bits: PRBS-31 per polarisation (recurrence b[n] = b[n-28] ^ b[n-31],
   first 31 bits = the seed state, LSB first);
2. Gray mapping per dimension (QPSK {0:+1, 1:-1}; 16QAM levels
   {-3,-1,+1,+3} <- {00,01,11,10}), unit mean symbol energy;
3. 2 samples/symbol, root-raised-cosine pulse shaping in the frequency domain;
4. Haar-random 2x2 unitary polarisation rotation;
5. chromatic dispersion exp(-j*beta2*L*w^2/2) (w = 2*pi*f);
6. a fractional sampling delay tau (exp(-j*w*tau));
7. frequency offset and Wiener laser phase noise, common to both polarisations;
8. complex AWGN with per-sample variance 2*Ps/SNR (Es/N0 = SNR per polarisation).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

try:  # multithreaded FFTs for the large streams when scipy is present
    import scipy.fft as _fft

    def _fftn(x):
        return _fft.fft(x, axis=-1, workers=-1)

    def _ifftn(x):
        return _fft.ifft(x, axis=-1, workers=-1)
except ImportError:  # pragma: no cover - numpy fallback
    def _fftn(x):
        return np.fft.fft(x, axis=-1)

    def _ifftn(x):
        return np.fft.ifft(x, axis=-1)

C_LIGHT = 299792458.0  # m/s


def beta2_from_dispersion(D_ps_nm_km: float, lambda_m: float) -> float:
    """Group-velocity dispersion beta2 [s^2/m] from the dispersion parameter D."""
    D = D_ps_nm_km * 1e-12 / (1e-9 * 1e3)  # s/m^2
    return -D * lambda_m ** 2 / (2.0 * math.pi * C_LIGHT)


def pol_seed_state(seed: int, pol: int) -> int:
    """31-bit non-zero PRBS start state of polarisation ``pol`` for ``seed``:
    v = (seed + off_pol) mod (2^31 - 1), state = (v * 1103515245 mod (2^31 - 1)) + 1
    with off = 0 for x and 0x2545F491 for y (the multiplier spreads small
    seeds over the 31 bits, so the sequence does not start in a run of zeros)."""
    m = (1 << 31) - 1
    off = 0 if pol == 0 else 0x2545F491
    v = (int(seed) + off) % m
    return (v * 1103515245) % m + 1


def prbs31(state: int, nbits: int) -> np.ndarray:
    """PRBS-31 bits (uint8) from a 31-bit start state.

    b[i] = (state >> i) & 1 for i < 31, then b[n] = b[n-28] ^ b[n-31].
    Generated by repeated squaring of the recurrence: the sequence also obeys
    b[n] = b[n-28m] ^ b[n-31m] for m = 2^k, so each pass extends it by 28m.
    """
    if not 0 < state < (1 << 31):
        raise ValueError("PRBS-31 state must be a non-zero 31-bit value")
    out = np.zeros(max(nbits, 31) + 31 * 64, dtype=np.uint8)
    out[:31] = [(state >> i) & 1 for i in range(31)]
    n = 31
    while n < nbits:
        m = 1
        while 31 * m * 2 <= n:
            m *= 2
        step = 28 * m
        hi = min(n + step, out.size)
        cnt = hi - n
        out[n:hi] = out[n - 28 * m:n - 28 * m + cnt] ^ out[n - 31 * m:n - 31 * m + cnt]
        n = hi
        if n >= out.size and n < nbits:  # grow the buffer
            out = np.concatenate([out, np.zeros(nbits + 31 * 64 - out.size, np.uint8)])
    return out[:nbits].copy()


def gray_map(bits: np.ndarray, bits_per_sym: int) -> np.ndarray:
    """Gray-coded square QAM symbols of unit mean energy (bits LSB-stream order)."""
    b = bits.reshape(-1, bits_per_sym).astype(np.int64)
    if bits_per_sym == 2:
        return ((1 - 2 * b[:, 0]) + 1j * (1 - 2 * b[:, 1])) / math.sqrt(2.0)
    if bits_per_sym == 4:
        lut = np.array([-3.0, -1.0, 3.0, 1.0])  # index = 2*msb + lsb: 00,01,10,11
        i = lut[2 * b[:, 0] + b[:, 1]]
        q = lut[2 * b[:, 2] + b[:, 3]]
        return (i + 1j * q) / math.sqrt(10.0)
    raise ValueError("bits_per_sym must be 2 (QPSK) or 4 (16QAM)")


def _rrc_amplitude(f: np.ndarray, Rs: float, rho: float) -> np.ndarray:
    """Root-raised-cosine amplitude response (peak 1)."""
    a = np.abs(f) / Rs
    h = np.zeros_like(a)
    h[a <= (1 - rho) / 2] = 1.0
    if rho > 0:
        mid = (a > (1 - rho) / 2) & (a <= (1 + rho) / 2)
        h[mid] = np.sqrt(0.5 * (1.0 + np.cos(math.pi / rho * (a[mid] - (1 - rho) / 2))))
    return h


def haar_unitary(rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed 2x2 unitary (QR of a complex Gaussian, phase-fixed)."""
    z = (rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))[None, :]


@dataclasses.dataclass
class LinkConfig:
    baud_hz: float = 28e9
    bits_per_sym: int = 2            # 2 = QPSK, 4 = 16QAM
    n_sym: int = 1 << 16             # symbols per polarisation
    fiber_len_m: float = 1000e3
    D_ps_nm_km: float = 17.0
    lambda_m: float = 1550e-9
    rolloff: float = 0.1
    snr_db: float | None = 12.0      # Es/N0 per polarisation; None = noiseless
    fo_hz: float = 100e6
    linewidth_hz: float = 100e3
    rotate: bool = True              # Haar-random polarisation rotation
    delay_frac: float | None = None  # sampling delay in symbols; None = U[0,1)
    phase0: float | None = None      # initial carrier phase; None = U[0,2pi)
    prbs_seed: int = 1
    seed: int = 1000
    out_dtype: str = "c128"          # c128 | c64 | c16 (interleaved float16 re/im)
    phase_jumps: tuple = ()          # ((sample index, radians), ...) carrier phase steps


def simulate(cfg: LinkConfig) -> dict:
    """Generate one received stream.  Returns a dict with

    ``rx``: samples, shape [2, 2*n_sym] (complex128/complex64) or
    [2, 2*n_sym, 2] float16 for c16; ``tx_bits`` [2, n_sym*bits_per_sym]
    uint8; ``tx_syms`` [2, n_sym] complex128; and the drawn impairments
    (``U``, ``tau_s``, ``phase0``)."""
    sps = 2
    Rs = float(cfg.baud_hz)
    fs = sps * Rs
    n = int(cfg.n_sym)
    ns = sps * n
    rng = np.random.default_rng(cfg.seed)

    bits = np.stack([prbs31(pol_seed_state(cfg.prbs_seed, p), n * cfg.bits_per_sym)
                     for p in range(2)])
    syms = np.stack([gray_map(bits[p], cfg.bits_per_sym) for p in range(2)])

    f = np.fft.fftfreq(ns, d=1.0 / fs)
    up = np.zeros((2, ns), dtype=np.complex128)
    up[:, ::sps] = syms
    X = _fftn(up) * _rrc_amplitude(f, Rs, cfg.rolloff)[None, :]
    x = _ifftn(X)
    x /= np.sqrt(np.mean(np.abs(x) ** 2, axis=1, keepdims=True))
    Ps = 1.0

    U = haar_unitary(rng) if cfg.rotate else np.eye(2, dtype=np.complex128)
    x = U @ x

    w = 2.0 * math.pi * f
    b2 = beta2_from_dispersion(cfg.D_ps_nm_km, cfg.lambda_m)
    delay_frac = float(rng.uniform(0.0, 1.0)) if cfg.delay_frac is None else float(cfg.delay_frac)
    tau = delay_frac / Rs
    cd_phase = np.mod(b2 * cfg.fiber_len_m * w ** 2 / 2.0, 2.0 * math.pi)
    Hch = np.exp(-1j * cd_phase) * np.exp(-1j * w * tau)
    x = _ifftn(_fftn(x) * Hch[None, :])

    phase0 = float(rng.uniform(0, 2 * math.pi)) if cfg.phase0 is None else float(cfg.phase0)
    nidx = np.arange(ns, dtype=np.float64)
    ph = phase0 + 2.0 * math.pi * cfg.fo_hz * nidx / fs
    if cfg.linewidth_hz > 0:
        inc = rng.standard_normal(ns) * math.sqrt(2.0 * math.pi * cfg.linewidth_hz / fs)
        inc[0] = 0.0
        ph = ph + np.cumsum(inc)
    for n_j, rad in cfg.phase_jumps:
        ph[int(n_j):] += float(rad)
    x = x * np.exp(1j * ph)[None, :]

    if cfg.snr_db is not None:
        snr = 10.0 ** (cfg.snr_db / 10.0)
        sigma2 = Ps * sps / snr
        x = x + math.sqrt(sigma2 / 2.0) * (rng.standard_normal((2, ns)) + 1j * rng.standard_normal((2, ns)))

    if cfg.out_dtype == "c128":
        rx = x
    elif cfg.out_dtype == "c64":
        rx = x.astype(np.complex64)
    elif cfg.out_dtype == "c16":
        rx = np.stack([x.real, x.imag], axis=-1).astype(np.float16)
    else:
        raise ValueError("out_dtype must be c128, c64 or c16")
    return {"rx": rx, "tx_bits": bits, "tx_syms": syms, "U": U, "tau_s": tau,
            "delay_frac": delay_frac, "phase0": phase0, "fs": fs, "beta2": b2}
