"""FP64 oracle of the receiver chain -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The product path never does.

The chain (per stream, both polarisations processed jointly):

  a1  overlap-save chromatic-dispersion compensation (paper Sec. II: 100 %
      overlap-save frequency-domain processing, the overlap with the
      previous buffer carried so the stream is contiguous; CD compensated in
      the frequency domain).  H = exp(+j*beta2*L*w^2/2) * RRC matched filter
      * exp(+j*w*tau_f) (timing advance of the frame).
  a3  timing: Godard band-edge spectral correlation of the compensated
      spectrum, tau_{f+1} = tau_f + gain * residual; frame 0 is first
      estimated with tau = 0 (acquisition pass).
  a2  frequency offset: Welch-averaged periodogram of the 4th power of the
      symbol-spaced compensated samples, argmax + 3-point refine on the log
      (a frame shorter than 4096 symbols keeps the previous estimate);
      removed with a phase-continuous rotation together with the frame AGC.
  a4  2x2 butterfly FIR, T taps at T/2 spacing, one output per symbol.
  a5  block-LMS adaptation, one tap update per sub-block of K symbols with
      the gradient averaged over the sub-block (taps fixed inside it):
      CMA during acquisition, then decision-directed LMS (paper Sec. II uses a
      DD-LMS time-domain equaliser) with a 4th-power block phase reference.
      Acquisition is one sequential chain over the first symbols of the
      stream; afterwards every frame is cut into segments of S symbols and
      segment j continues the chain of segment j of the previous frame.
  a6  blind phase search over B test angles with a (2W+1)-symbol window and
      pi/2 unwrapping; reduced-cost form: the same window costs at the B/S
      coarse angles only, the fine index from the parabola through the
      coarse minimum and its two neighbours.
  a7  hard decision and Gray demapping (paper Sec. II: decisions demapped).
  a8  BER against the known PRBS-31 payload after a one-time sync (delay,
      polarisation order, quadrant), with cycle-slip re-resolution; Q-factor
      from BER (paper Sec. III: Q estimated from BER).

Every number is FP64.  Library primitives used: numpy FFT, matrix products.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

C_LIGHT = 299792458.0
FOE_MIN_SYMS = 4096  # a frame shorter than this keeps the previous FO estimate

# Which functions are pinned by independent checks (tests/test_oracle_*.py).
PIN_STATUS = {
    "cd_frequency_response": "pinned: channel round trip to 1e-12; Nyquist ISI-free symbols",
    "ols_cd": "pinned: equals the full-length circular filter on interior samples",
    "godard_sum": "pinned: injected delay recovered (noiseless) to <1% of T",
    "foe_from_periodogram": "pinned: injected offset recovered within a tenth of a bin",
    "mimo_fir": "pinned: brute-force convolution sums; inverse of a known unitary",
    "sub_block_update": "pinned: CMA converges to the inverse of a known unitary",
    "bps": "pinned: constant injected phase recovered modulo pi/2 to grid resolution",
    "two_stage_index": "pinned: vertex of exact parabolas (wrapping included) recovered to the nearest fine index",
    "bps_two_stage": "pinned: equals bps for S = 1; off-grid constant phase recovered to one fine step",
    "unwrap_increments": "pinned: phase ramp across quadrants tracked without slips",
    "decide/demap": "pinned: exhaustive constellation round trip, Gray neighbour property",
    "prbs31_bits": "pinned: independent generator agreement, recurrence, balance",
    "ber_count": "pinned: AWGN BER inside the 99% Clopper-Pearson interval of the Q-function; "
                 "quarter-turn carrier steps counted as slips with hand-counted errors",
    "cma_radius": "pinned: QPSK 1 and 16QAM 1.32 from the constellation's moduli by hand",
    "acquire": "pinned: CMA inverts a known unitary (QPSK and 16QAM, < -30 dB) with unit output power",
    "dd_phase": "pinned: constant phase of the whole constellation recovered to 1e-12, quarter turns ignored",
    "q_factor_db": "pinned: BER = Q(x) of a Gaussian tail gives 20 log10(x) to 1e-9",
}


# --------------------------------------------------------------------------
# configuration and geometry
# --------------------------------------------------------------------------

@dataclasses.dataclass
class RxConfig:
    baud_hz: float = 28e9
    bits_per_sym: int = 2                 # 2 QPSK, 4 16QAM
    fiber_len_m: float = 1000e3
    D_ps_nm_km: float = 17.0
    lambda_m: float = 1550e-9
    rrc_rolloff: float = 0.1              # < 0: no matched filter
    fft_n: int = 0                        # 0: auto
    cd_halo: int = 0                      # M-1; 0: auto
    mimo_taps: int = 15
    bps_angles: int = 64
    bps_half_window: int = 16
    bps_coarse_stride: int = 1            # S > 1: two-stage search over B/S coarse angles
    sub_block_syms: int = 64
    seg_syms: int = 512
    frame_syms: int = 1 << 16
    cma_syms: int = 16384
    acq_syms: int = 20480
    mu_cma: float = 3e-2
    mu_dd: float = 5e-3
    timing_gain: float = 0.5
    prbs_seed: int = 0                    # 0: no BER counting
    ber_skip_syms: int = 16384
    sync_syms: int = 4096
    sync_max_delay: int = 32
    slip_window: int = 1024


@dataclasses.dataclass
class Geometry:
    fs: float
    beta2: float
    cd_memory: float      # CD impulse-response length in samples
    halo: int             # M - 1 (even)
    h: int                # halo / 2
    N: int                # OLS FFT size
    L: int                # kept samples per OLS block
    c: int                # FIR centre tap (T-1)/2


def beta2(cfg: RxConfig) -> float:
    """beta2 = -D lambda^2 / (2 pi c), D converted from ps/(nm km) to s/m^2."""
    D = cfg.D_ps_nm_km * 1e-6
    return -D * cfg.lambda_m ** 2 / (2.0 * math.pi * C_LIGHT)


def geometry(cfg: RxConfig) -> Geometry:
    """OLS sizes.  CD memory = |D| L (lambda^2 Rs (1+rho) / c) fs samples;
    halo M-1 = ceil(1.1 * memory) rounded up to even; N = smallest power of
    two >= max(1024, 4 (M-1)), at most 16384, doubled to 32768 when 16384
    points would keep less than half of each block (M-1 > 8192), unless
    given."""
    fs = 2.0 * cfg.baud_hz
    rho = max(cfg.rrc_rolloff, 0.0)
    D = abs(cfg.D_ps_nm_km) * 1e-6
    dlam = cfg.lambda_m ** 2 * cfg.baud_hz * (1.0 + rho) / C_LIGHT
    mem = D * cfg.fiber_len_m * dlam * fs
    halo = cfg.cd_halo if cfg.cd_halo > 0 else int(math.ceil(1.1 * mem))
    halo += halo & 1
    halo = max(halo, 2)
    if cfg.fft_n > 0:
        N = cfg.fft_n
    else:
        N = 1024
        while N < 4 * halo and N < 16384:
            N *= 2
        if 2 * halo > N:
            N *= 2
    if N - halo < 2:
        raise ValueError("fft_n too small for the CD halo")
    return Geometry(fs=fs, beta2=beta2(cfg), cd_memory=mem, halo=halo, h=halo // 2,
                    N=N, L=N - halo, c=(cfg.mimo_taps - 1) // 2)


# --------------------------------------------------------------------------
# a1: chromatic dispersion compensation by overlap-save
# --------------------------------------------------------------------------

def _rrc(f: np.ndarray, Rs: float, rho: float) -> np.ndarray:
    """Root-raised-cosine amplitude: 1 in |f| <= (1-rho)Rs/2, cosine roll-off
    sqrt((1+cos(pi/rho (|f|/Rs - (1-rho)/2)))/2) up to (1+rho)Rs/2, 0 beyond."""
    a = np.abs(f) / Rs
    out = np.where(a <= (1 - rho) / 2, 1.0, 0.0)
    if rho > 0:
        band = (a > (1 - rho) / 2) & (a <= (1 + rho) / 2)
        arg = math.pi / rho * (a - (1 - rho) / 2)
        out = np.where(band, np.sqrt(0.5 * (1.0 + np.cos(arg))), out)
    return out


def bin_freqs(N: int, fs: float) -> np.ndarray:
    """FFT bin frequencies: k fs/N for k < N/2, (k-N) fs/N otherwise."""
    k = np.arange(N)
    return np.where(k < N // 2, k, k - N) * (fs / N)


def cd_frequency_response(cfg: RxConfig, N: int) -> np.ndarray:
    """H[k] = exp(+j beta2 L w_k^2 / 2) * RRC(f_k), w_k = 2 pi f_k (FP64; the
    phase is reduced modulo 2 pi before the exponential)."""
    g = geometry(cfg)
    f = bin_freqs(N, g.fs)
    w = 2.0 * math.pi * f
    ph = np.mod(g.beta2 * cfg.fiber_len_m * w ** 2 / 2.0, 2.0 * math.pi)
    H = np.exp(1j * ph)
    if cfg.rrc_rolloff >= 0:
        H = H * _rrc(f, cfg.baud_hz, cfg.rrc_rolloff)
    return H


def timing_response(N: int, fs: float, tau: float) -> np.ndarray:
    """exp(+j w_k tau): advances the signal by tau seconds."""
    return np.exp(1j * 2.0 * math.pi * bin_freqs(N, fs) * tau)


def full_length_cd(x: np.ndarray, cfg: RxConfig) -> np.ndarray:
    """Test mode: the CD/matched filter applied as one circular filter over
    the whole record (one FFT of the record length)."""
    H = cd_frequency_response(cfg, x.shape[-1])
    return np.fft.ifft(np.fft.fft(x, axis=-1) * H, axis=-1)


def ols_cd(x: np.ndarray, s0: int, s1: int, H: np.ndarray, h: int, N: int, L: int,
           n_valid: int, on_block=None) -> np.ndarray:
    """Overlap-save: output samples [s0, s1) of one polarisation.

    Block j keeps outputs [s0 + jL, s0 + (j+1)L) (the last one clipped) from
    the circular filtering of the input window [s0 + jL - h, +N): samples
    outside [0, n_valid) are zero.  ``on_block(Y, z_kept, a, lo)`` is called
    per block with the filtered spectrum, the kept outputs, the index of the
    first kept sample and the index of the window's first sample."""
    out = np.zeros(s1 - s0, dtype=np.complex128)
    j = 0
    while s0 + j * L < s1:
        a = s0 + j * L
        win = np.zeros(N, dtype=np.complex128)
        lo, hi = a - h, a - h + N
        clo, chi = max(lo, 0), min(hi, n_valid)
        if chi > clo:
            win[clo - lo:chi - lo] = x[clo:chi]
        Y = np.fft.fft(win) * H
        z = np.fft.ifft(Y)
        keep = min(L, s1 - a)
        out[a - s0:a - s0 + keep] = z[h:h + keep]
        if on_block is not None:
            on_block(Y, z[h:h + keep], a, lo)
        j += 1
    return out


# --------------------------------------------------------------------------
# a3 timing, a2 frequency offset
# --------------------------------------------------------------------------

def godard_sum(Y: np.ndarray, n0: int = 0) -> complex:
    """Band-edge spectral correlation (-1)^n0 sum_{k<N/2} Y[k] conj(Y[k+N/2]):
    the bins Rs apart at 2 samples/symbol; its argument is -2 pi Rs times the
    residual delay.  n0 is the absolute index of the block's first sample: a
    window start shifted by n0 samples turns the product by exp(j pi n0)."""
    N = Y.shape[-1]
    sgn = -1.0 if (n0 & 1) else 1.0
    return sgn * complex(np.sum(Y[:N // 2] * np.conj(Y[N // 2:])))


def timing_residual(C: complex, Rs: float) -> float:
    """Residual delay -arg(C) / (2 pi Rs), in (-T/2, T/2]."""
    if C == 0:
        return 0.0
    return -math.atan2(C.imag, C.real) / (2.0 * math.pi * Rs)


def foe_block_periodogram(z_even: np.ndarray, N: int) -> np.ndarray:
    """|FFT_{N/2}(z^4)|^2 of one block's symbol-spaced samples, zero-padded."""
    u = np.zeros(N // 2, dtype=np.complex128)
    u[:z_even.size] = z_even ** 4
    return np.abs(np.fft.fft(u)) ** 2


def foe_from_periodogram(P: np.ndarray, Rs: float) -> float:
    """Frequency offset from the summed 4th-power periodogram (N/2 bins at
    1 sample/symbol): argmax (lowest index on ties), then a parabola through
    the logarithms of the peak and its two cyclic neighbours (Gaussian
    interpolation), offset = bin frequency / 4.  No refinement if a
    neighbour is zero or the parabola is flat."""
    n = P.size
    k = int(np.argmax(P))
    pm, p0, pp = P[(k - 1) % n], P[k], P[(k + 1) % n]
    d = 0.0
    if pm > 0 and pp > 0 and p0 > 0:
        lm, l0, lp = math.log(pm), math.log(p0), math.log(pp)
        den = lm - 2.0 * l0 + lp
        if den < 0:
            d = 0.5 * (lm - lp) / den
    ks = k if k < n // 2 else k - n
    return (ks + d) * (Rs / n) / 4.0


# --------------------------------------------------------------------------
# constellation, decision, demapping
# --------------------------------------------------------------------------

def levels(bits_per_sym: int) -> np.ndarray:
    """Per-dimension amplitude levels in increasing order (unit symbol energy)."""
    if bits_per_sym == 2:
        return np.array([-1.0, 1.0]) / math.sqrt(2.0)
    return np.array([-3.0, -1.0, 1.0, 3.0]) / math.sqrt(10.0)


def level_bits(bits_per_sym: int) -> np.ndarray:
    """Gray bit label (MSB first) of each level index: QPSK {-:1, +:0};
    16QAM {-3:00, -1:01, +1:11, +3:10}."""
    if bits_per_sym == 2:
        return np.array([[1], [0]], dtype=np.uint8)
    return np.array([[0, 0], [0, 1], [1, 1], [1, 0]], dtype=np.uint8)


def const_map(bits: np.ndarray, bits_per_sym: int) -> np.ndarray:
    """Bits (I bits then Q bits per symbol) -> constellation points."""
    lv = levels(bits_per_sym)
    lb = level_bits(bits_per_sym)
    h = bits_per_sym // 2
    b = bits.reshape(-1, 2, h)
    code = {tuple(lb[i]): i for i in range(lv.size)}
    iI = np.array([code[tuple(r)] for r in b[:, 0, :]])
    iQ = np.array([code[tuple(r)] for r in b[:, 1, :]])
    return lv[iI] + 1j * lv[iQ]


def level_index(x: np.ndarray, bits_per_sym: int) -> np.ndarray:
    """Nearest level per dimension; a value exactly on a threshold takes the
    larger level."""
    lv = levels(bits_per_sym)
    thr = 0.5 * (lv[1:] + lv[:-1])
    return np.searchsorted(thr, x, side="right")


def decide(z: np.ndarray, bits_per_sym: int) -> np.ndarray:
    """Hard decision: nearest constellation point."""
    lv = levels(bits_per_sym)
    return lv[level_index(z.real, bits_per_sym)] + 1j * lv[level_index(z.imag, bits_per_sym)]


def demap(z: np.ndarray, bits_per_sym: int) -> np.ndarray:
    """Decision + Gray demap: [n] complex -> [n, bits_per_sym] bits."""
    lb = level_bits(bits_per_sym)
    return np.concatenate([lb[level_index(z.real, bits_per_sym)],
                           lb[level_index(z.imag, bits_per_sym)]], axis=1)


def cma_radius(bits_per_sym: int) -> float:
    """R2 = E|s|^4 / E|s|^2 of the unit-energy constellation."""
    lv = levels(bits_per_sym)
    pts = (lv[:, None] + 1j * lv[None, :]).ravel()
    return float(np.mean(np.abs(pts) ** 4) / np.mean(np.abs(pts) ** 2))


# --------------------------------------------------------------------------
# a4/a5: butterfly FIR and block-LMS
# --------------------------------------------------------------------------

def mimo_fir(w: np.ndarray, r: np.ndarray, k0: int, k1: int) -> np.ndarray:
    """y_p[k] = sum_q sum_t w[p,q,t] r_q[2k + t] for k in [k0, k1) (r is the
    frame buffer whose index 2k + t is sample 2k + t - c of the frame)."""
    T = w.shape[-1]
    X = [np.stack([r[q, 2 * k:2 * k + T] for k in range(k0, k1)]) for q in range(2)]
    return np.stack([X[0] @ w[p, 0] + X[1] @ w[p, 1] for p in range(2)]), X


def dd_phase(y: np.ndarray) -> float:
    """4th-power block phase reference: arg(-sum y^4) / 4 (square QAM has
    E[s^4] < 0), 0 if the sum is zero."""
    s = -np.sum(y ** 4)
    if s == 0:
        return 0.0
    return math.atan2(s.imag, s.real) / 4.0


def sub_block_update(w, r, k0, k1, mode, mu, R2, bits_per_sym):
    """One block-LMS step over symbols [k0, k1): outputs with fixed taps,
    error (CMA: e = y(|y|^2 - R2); DD: e = y - e^{j phi} dec(e^{-j phi} y),
    phi from dd_phase), gradient g[p,q,t] = (1/K) sum_k e_p[k] conj(r_q[2k+t]),
    then w <- w - mu g.  Returns (new taps, outputs)."""
    y, X = mimo_fir(w, r, k0, k1)
    K = k1 - k0
    e = np.empty_like(y)
    for p in range(2):
        if mode == "cma":
            e[p] = y[p] * (np.abs(y[p]) ** 2 - R2)
        else:
            ph = dd_phase(y[p])
            rot = np.exp(1j * ph)
            e[p] = y[p] - rot * decide(y[p] / rot, bits_per_sym)
    g = np.empty_like(w)
    for p in range(2):
        for q in range(2):
            g[p, q] = X[q].conj().T @ e[p] / K
    return w - mu * g, y


def centre_spike(T: int) -> np.ndarray:
    """Initial taps: w_xx[c] = w_yy[c] = 1, all others 0."""
    w = np.zeros((2, 2, T), dtype=np.complex128)
    w[0, 0, (T - 1) // 2] = 1.0
    w[1, 1, (T - 1) // 2] = 1.0
    return w


def acquire(r: np.ndarray, n_sym: int, cfg: RxConfig):
    """Sequential acquisition over symbols [0, min(acq_syms, n_sym)) of the
    first frame: sub-blocks of K; CMA while the sub-block starts before
    cma_syms, DD afterwards.  At the CMA->DD switch, if the lag-0 correlation
    of the two outputs over the last min(1024, cma) CMA symbols exceeds 0.5,
    the y row is replaced by the conjugate-orthogonal of the x row."""
    T, K = cfg.mimo_taps, cfg.sub_block_syms
    R2 = cma_radius(cfg.bits_per_sym)
    w = centre_spike(T)
    n_acq = min(cfg.acq_syms, n_sym)
    ys = []
    reinit = False
    k0 = 0
    was_cma = False
    while k0 < n_acq:
        k1 = min(k0 + K, n_acq)
        mode = "cma" if k0 < cfg.cma_syms else "dd"
        if mode == "dd" and was_cma:
            yy = np.concatenate(ys, axis=1)
            nc = min(1024, yy.shape[1])
            yx, yv = yy[0, -nc:], yy[1, -nc:]
            den = math.sqrt(float(np.sum(np.abs(yx) ** 2) * np.sum(np.abs(yv) ** 2)))
            rho = abs(np.sum(yx * np.conj(yv))) / den if den > 0 else 0.0
            if rho > 0.5:
                w[1, 0] = -np.conj(w[0, 1][::-1])
                w[1, 1] = np.conj(w[0, 0][::-1])
                reinit = True
        mu = cfg.mu_cma if mode == "cma" else cfg.mu_dd
        w, y = sub_block_update(w, r, k0, k1, mode, mu, R2, cfg.bits_per_sym)
        if mode == "cma":
            ys.append(y)
        was_cma = mode == "cma"
        k0 = k1
    return w, reinit


# --------------------------------------------------------------------------
# a6 blind phase search, a7 decisions
# --------------------------------------------------------------------------

def bps_angles(B: int) -> np.ndarray:
    """phi_b = (b/B - 1/2) pi/2, b = 0..B-1."""
    return (np.arange(B) / B - 0.5) * (math.pi / 2.0)


def bps_costs(y: np.ndarray, phi: np.ndarray, W: int, bits_per_sym: int, a: int, b: int) -> np.ndarray:
    """D_{k,i} = sum_{|m|<=W, 0<=k+m<n} |z - dec(z)|^2, z = y_{k+m} exp(-j phi_i),
    for the symbols a <= k < b (rows) and the listed test angles (columns)."""
    n = y.size
    lo, hi = max(a - W, 0), min(b + W, n)
    z = y[lo:hi, None] * np.exp(-1j * phi)[None, :]
    d = np.abs(z - decide(z, bits_per_sym)) ** 2
    D = np.zeros((b - a, phi.size))
    for i in range(-W, W + 1):
        src_lo, src_hi = a + i, b + i
        clo, chi = max(src_lo, 0), min(src_hi, n)
        if chi > clo:
            D[clo - src_lo:chi - src_lo] += d[clo - lo:chi - lo]
    return D


def bps(y: np.ndarray, B: int, W: int, bits_per_sym: int, chunk: int = 1 << 15) -> np.ndarray:
    """b_k = argmin_b sum_{|i|<=W, 0<=k+i<n} |z_{k+i,b} - dec(z_{k+i,b})|^2,
    z_{k,b} = y_k exp(-j phi_b); lowest b on exact ties.  Computed in chunks
    of symbols (each output is the same sum, in the same order)."""
    n = y.size
    phi = bps_angles(B)
    out = np.empty(n, dtype=np.int64)
    for a in range(0, n, chunk):
        b = min(a + chunk, n)
        out[a:b] = np.argmin(bps_costs(y, phi, W, bits_per_sym, a, b), axis=1)
    return out


def two_stage_index(Dc: np.ndarray, S: int, B: int) -> np.ndarray:
    """Fine angle index from the window costs Dc[k, j] of the C = B/S coarse
    angles b = S j: j* = argmin_j (lowest j on ties); with the cyclic
    neighbours D-, D0, D+ of j* (the cost is pi/2-periodic in the angle, so
    coarse index C wraps to 0), c = D- - 2 D0 + D+ (>= 0 at a minimum) and
    delta = (D- - D+) / (2c) in [-1/2, 1/2] (0 if c = 0) is the vertex of
    the parabola through the three costs in units of the coarse step;
    b = (S j* + floor(S delta + 1/2)) mod B."""
    C = Dc.shape[1]
    k = np.arange(Dc.shape[0])
    j = np.argmin(Dc, axis=1)
    Dm, D0, Dp = Dc[k, (j - 1) % C], Dc[k, j], Dc[k, (j + 1) % C]
    c = Dm - 2.0 * D0 + Dp
    delta = np.where(c > 0, (Dm - Dp) / (2.0 * np.where(c > 0, c, 1.0)), 0.0)
    delta = np.clip(delta, -0.5, 0.5)
    r = np.floor(S * delta + 0.5).astype(np.int64)
    return (S * j + r) % B


def bps_two_stage(y: np.ndarray, B: int, W: int, bits_per_sym: int, S: int,
                  chunk: int = 1 << 15) -> np.ndarray:
    """Reduced-cost blind phase search: the window costs of the same
    definition as bps() at the B/S coarse angles b = S j only, then the fine
    index on the B-angle grid from two_stage_index (S = 1 is bps())."""
    n = y.size
    phi = bps_angles(B)[::S]
    out = np.empty(n, dtype=np.int64)
    for a in range(0, n, chunk):
        b = min(a + chunk, n)
        out[a:b] = two_stage_index(bps_costs(y, phi, W, bits_per_sym, a, b), S, B)
    return out


def unwrap_increments(bhat: np.ndarray, B: int) -> np.ndarray:
    """m_0 = 0, m_k = m_{k-1} + round((phi_{k-1} - phi_k) / (pi/2)) with
    round(x) = floor(x + 1/2); since (phi_{k-1}-phi_k)/(pi/2) = (b_{k-1}-b_k)/B
    the increment is floor((2(b_{k-1} - b_k) + B) / (2B)) in exact integers."""
    m = np.zeros(bhat.size, dtype=np.int64)
    if bhat.size > 1:
        inc = (2 * (bhat[:-1] - bhat[1:]) + B) // (2 * B)
        m[1:] = np.cumsum(inc)
    return m


# --------------------------------------------------------------------------
# a8 BER
# --------------------------------------------------------------------------

def prbs31_bits(state: int, nbits: int) -> np.ndarray:
    """PRBS-31: b[i] = (state >> i) & 1 for i < 31, b[n] = b[n-28] ^ b[n-31];
    the recurrence is applied 28 bits at a time (each of those bits depends
    only on the 31 before the group)."""
    b = np.zeros(max(nbits, 31) + 28, dtype=np.uint8)
    for i in range(31):
        b[i] = (state >> i) & 1
    n = 31
    while n < nbits:
        b[n:n + 28] = b[n - 28:n] ^ b[n - 31:n - 3]
        n += 28
    return b[:nbits]


def prbs_state(seed: int, pol: int) -> int:
    """Start state of polarisation pol: v = (seed + off_pol) mod (2^31-1),
    state = ((v * 1103515245) mod (2^31-1)) + 1; off = 0 for x and
    0x2545F491 for y."""
    p = (1 << 31) - 1
    v = (int(seed) + (0 if pol == 0 else 0x2545F491)) % p
    return (v * 1103515245) % p + 1


def rotate_quadrants(lI: np.ndarray, lQ: np.ndarray, q: int, nl: int):
    """Level indices of s * j^q (j: (I, Q) -> (-Q, I); negation l -> nl-1-l)."""
    for _ in range(q % 4):
        lI, lQ = nl - 1 - lQ, lI
    return lI, lQ


def _bits_from_levels(lI, lQ, bits_per_sym):
    lb = level_bits(bits_per_sym)
    return np.concatenate([lb[lI], lb[lQ]], axis=1)


def ber_sync(lv_idx, ref_bits, cfg: RxConfig, k_s: int, n_sync: int):
    """Search delay d in [-Dmax, Dmax], polarisation order (identity, swap) and
    per-polarisation quadrant q on symbols [k_s, k_s + n_sync): rx symbol k
    of pol p is compared with tx symbol k - d of pol perm[p].  Minimum total
    errors wins; ties keep the first candidate in (d ascending, identity
    before swap, q ascending) order."""
    nl = 1 << (cfg.bits_per_sym // 2)
    bps_ = cfg.bits_per_sym
    best = None
    for d in range(-cfg.sync_max_delay, cfg.sync_max_delay + 1):
        for perm in (0, 1):
            tot = 0
            qs = []
            for p in range(2):
                tp = p ^ perm
                lI, lQ = lv_idx[p][0][k_s:k_s + n_sync], lv_idx[p][1][k_s:k_s + n_sync]
                ref = ref_bits[tp][(k_s - d) * bps_:(k_s - d + n_sync) * bps_].reshape(n_sync, bps_)
                errs = []
                for q in range(4):
                    a, b = rotate_quadrants(lI, lQ, q, nl)
                    errs.append(int(np.sum(_bits_from_levels(a, b, bps_) != ref)))
                qb = int(np.argmin(errs))
                qs.append(qb)
                tot += errs[qb]
            if best is None or tot < best[0]:
                best = (tot, d, perm, qs)
    return {"errors": best[0], "delay": best[1], "perm": best[2], "quadrant": best[3]}


def ber_count(lv_idx, ref_bits, cfg: RxConfig, sync: dict, k_s: int, k_end: int):
    """Count bit errors on symbols [k_s, k_end) per polarisation with the sync
    delay/permutation.  Windows of slip_window symbols from k_s: if the
    window's errors under the current quadrant exceed a quarter of its bits,
    the quadrant becomes the window's best (lowest q on ties) and a slip is
    counted; the window's errors are counted under the quadrant then in use."""
    nl = 1 << (cfg.bits_per_sym // 2)
    bps_ = cfg.bits_per_sym
    d, perm = sync["delay"], sync["perm"]
    errors, bits, slips = 0, 0, 0
    for p in range(2):
        q = sync["quadrant"][p]
        tp = p ^ perm
        a = k_s
        while a < k_end:
            b = min(a + cfg.slip_window, k_end)
            n = b - a
            lI, lQ = lv_idx[p][0][a:b], lv_idx[p][1][a:b]
            ref = ref_bits[tp][(a - d) * bps_:(b - d) * bps_].reshape(n, bps_)
            errs = []
            for qq in range(4):
                u, v = rotate_quadrants(lI, lQ, qq, nl)
                errs.append(int(np.sum(_bits_from_levels(u, v, bps_) != ref)))
            if errs[q] * 4 > n * bps_:
                q = int(np.argmin(errs))
                slips += 1
            errors += errs[q]
            bits += n * bps_
            a = b
    return {"errors": errors, "bits": bits, "slips": slips}


def q_factor_db(ber: float) -> float:
    """Q = 20 log10(sqrt(2) erfcinv(2 BER))."""
    from scipy.special import erfcinv
    if ber <= 0 or ber >= 0.5:
        return float("inf") if ber <= 0 else 0.0
    return 20.0 * math.log10(math.sqrt(2.0) * float(erfcinv(2.0 * ber)))


# --------------------------------------------------------------------------
# the whole stream
# --------------------------------------------------------------------------

class Receiver:
    """Runs the chain over one complete stream x [2, n_samp] (complex)."""

    def __init__(self, cfg: RxConfig):
        self.cfg = cfg
        self.g = geometry(cfg)
        if cfg.mimo_taps % 2 != 1:
            raise ValueError("mimo_taps must be odd")
        self.Hcd = cd_frequency_response(cfg, self.g.N)

    def _cd_frame(self, x, n_samp, s0, s1, tau, f0, f1, collect):
        """OLS over [s0, s1) of both pols with timing tau.  Accumulates the
        Godard sum; if collect, also the in-frame power and the FOE
        periodogram of even in-frame samples [f0, f1)."""
        g = self.g
        H = self.Hcd * timing_response(g.N, g.fs, tau)
        acc = {"C": 0j, "P": 0.0, "S": np.zeros(g.N // 2)}

        def on_block(Y, z, a, lo):
            acc["C"] += godard_sum(Y, lo)
            if collect:
                n = a + np.arange(z.size)
                inf = (n >= f0) & (n < f1)
                acc["P"] += float(np.sum(np.abs(z[inf]) ** 2))
                sel = inf & (n % 2 == 0)
                if np.any(sel):
                    acc["S"] += foe_block_periodogram(z[sel], g.N)

        z = np.stack([ols_cd(x[p], s0, s1, H, g.h, g.N, g.L, n_samp, on_block) for p in range(2)])
        return z, acc

    def run(self, x: np.ndarray, tx_ref: bool = True) -> dict:
        cfg, g = self.cfg, self.g
        x = np.asarray(x, dtype=np.complex128)
        n_samp = x.shape[1]
        n_sym = n_samp // 2
        F, S, T, c = cfg.frame_syms, cfg.seg_syms, cfg.mimo_taps, g.c
        Rs = cfg.baud_hz
        n_frames = (n_sym + F - 1) // F
        G = (F + S - 1) // S
        y_all = np.zeros((2, n_sym), dtype=np.complex128)
        tau, theta = 0.0, 0.0
        chains = None
        trace = {"tau": [], "dfo": [], "gain": [], "theta": [], "C": []}
        w_acq, reinit = None, False
        for f in range(n_frames):
            Ff = min(F, n_sym - f * F)
            s0, s1 = 2 * f * F - c, 2 * (f * F + Ff) + c
            f0, f1 = 2 * f * F, 2 * (f * F + Ff)
            if f == 0:
                _, acc0 = self._cd_frame(x, n_samp, s0, s1, 0.0, f0, f1, False)
                tau = timing_residual(acc0["C"], Rs)
            z, acc = self._cd_frame(x, n_samp, s0, s1, tau, f0, f1, True)
            dfo = foe_from_periodogram(acc["S"], Rs)
            if f > 0 and Ff < FOE_MIN_SYMS:  # too short for its own estimate
                dfo = trace["dfo"][-1]
            P = acc["P"] / (2.0 * (f1 - f0))
            gain = 1.0 / math.sqrt(P) if P > 0 else 1.0
            om = 2.0 * math.pi * dfo / g.fs
            n = np.arange(s0, s1) - f0
            r = gain * z * np.exp(-1j * (theta + om * n))[None, :]
            trace["tau"].append(tau)
            trace["dfo"].append(dfo)
            trace["gain"].append(gain)
            trace["theta"].append(theta)
            trace["C"].append(acc["C"])
            if f == 0:
                w_acq, reinit = acquire(r, Ff, cfg)
                chains = [w_acq.copy() for _ in range(G)]
            R2 = cma_radius(cfg.bits_per_sym)
            for j in range((Ff + S - 1) // S):
                w = chains[j]
                a = j * S
                e = min(a + S, Ff)
                k0 = a
                while k0 < e:
                    k1 = min(k0 + cfg.sub_block_syms, e)
                    w, yb = sub_block_update(w, r, k0, k1, "dd", cfg.mu_dd, R2, cfg.bits_per_sym)
                    y_all[:, f * F + k0:f * F + k1] = yb
                    k0 = k1
                chains[j] = w
            theta = math.fmod(theta + om * (f1 - f0), 2.0 * math.pi)
            tau = tau + cfg.timing_gain * timing_residual(acc["C"], Rs)
        res = {"y": y_all, "trace": trace, "w_acq": w_acq, "reinit": reinit,
               "chains": chains, "n_sym": n_sym}
        # a6/a7
        B, W = cfg.bps_angles, cfg.bps_half_window
        phi = bps_angles(B)
        if cfg.bps_coarse_stride > 1:
            bh = np.stack([bps_two_stage(y_all[p], B, W, cfg.bits_per_sym, cfg.bps_coarse_stride) for p in range(2)])
        else:
            bh = np.stack([bps(y_all[p], B, W, cfg.bits_per_sym) for p in range(2)])
        m = np.stack([unwrap_increments(bh[p], B) for p in range(2)])
        phat = phi[bh] + m * (math.pi / 2.0)
        zc = y_all * np.exp(-1j * phat)
        lvi = [(level_index(zc[p].real, cfg.bits_per_sym), level_index(zc[p].imag, cfg.bits_per_sym))
               for p in range(2)]
        bits = np.stack([demap(zc[p], cfg.bits_per_sym) for p in range(2)])  # [2, n, bps]
        res.update({"bhat": bh, "m": m, "phase": phat, "zc": zc, "levels": lvi, "bits": bits})
        # a8
        res["ber"] = None
        if cfg.prbs_seed != 0:
            k_s = cfg.ber_skip_syms
            tail = (g.h + 1) // 2 + T + W
            k_end = n_sym - tail
            if k_s + cfg.sync_syms <= k_end and k_s > cfg.sync_max_delay:
                nb = (n_sym + cfg.sync_max_delay + 1) * cfg.bits_per_sym
                ref = [prbs31_bits(prbs_state(cfg.prbs_seed, p), nb) for p in range(2)]
                sync = ber_sync(lvi, ref, cfg, k_s, cfg.sync_syms)
                cnt = ber_count(lvi, ref, cfg, sync, k_s, k_end)
                lv = levels(cfg.bits_per_sym)
                dec = np.stack([lv[lvi[p][0]] + 1j * lv[lvi[p][1]] for p in range(2)])
                evm = float(np.sum(np.abs(zc[:, k_s:k_end] - dec[:, k_s:k_end]) ** 2)
                            / np.sum(np.abs(dec[:, k_s:k_end]) ** 2))
                ber = cnt["errors"] / cnt["bits"] if cnt["bits"] else 0.0
                res["ber"] = dict(cnt, sync=sync, ber=ber, evm=evm, k_s=k_s, k_end=k_end)
        return res
