"""Planted mistakes: each oracle function listed in PIN_STATUS is replaced by
a plausible wrong version (a flipped sign, a dropped factor, a transposed
operand, a wrong index or window) and at least one of its pins must then
fail.  This shows the pins constrain the function and do not merely
restate it.  CPU only; the real oracle is restored after each case."""
import math

import numpy as np
import pytest

import test_oracle_pins as P
from oracle import rx_oracle as O

ORIG = {k: getattr(O, k) for k in ("cd_frequency_response", "ols_cd", "godard_sum", "foe_from_periodogram",
                                   "mimo_fir", "sub_block_update", "bps", "bps_angles", "two_stage_index",
                                   "bps_two_stage", "unwrap_increments", "level_bits", "prbs31_bits",
                                   "ber_count", "cma_radius", "dd_phase", "q_factor_db", "acquire")}


# ---------------------------------------------------------------- mistakes --

def cd_conjugated(cfg, N):
    """Receiver applies the fibre's own phase (sign of beta2 L w^2 / 2 flipped)."""
    return np.conj(ORIG["cd_frequency_response"](cfg, N))


def ols_kept_window_off_by_one(x, s0, s1, H, h, N, L, n_valid, on_block=None):
    """Keeps z[h+1 : h+1+L] instead of z[h : h+L]: every output one sample late."""
    out = ORIG["ols_cd"](x, s0 + 1, s1 + 1, H, h, N, L, n_valid, on_block)
    return out


def godard_without_window_sign(Y, n0=0):
    """Drops the (-1)^n0 factor of a window starting at an odd sample."""
    return ORIG["godard_sum"](Y, 0)


def foe_without_quarter(Pw, Rs):
    """Forgets to divide the 4th-power tone frequency by 4."""
    return 4.0 * ORIG["foe_from_periodogram"](Pw, Rs)


def mimo_transposed(w, r, k0, k1):
    """Uses w[q, p] for the output p from input q (transposed butterfly)."""
    return ORIG["mimo_fir"](np.swapaxes(w, 0, 1), r, k0, k1)


def sub_block_cma_sign_flipped(w, r, k0, k1, mode, mu, R2, bits_per_sym):
    """CMA error y (R2 - |y|^2) instead of y (|y|^2 - R2): gradient ascent."""
    return ORIG["sub_block_update"](w, r, k0, k1, mode, -mu if mode == "cma" else mu, R2, bits_per_sym)


def bps_maximises(y, B, W, bits_per_sym, chunk=1 << 15):
    """argmax of the window cost instead of argmin."""
    n = y.size
    phi = ORIG["bps_angles"](B)
    out = np.empty(n, dtype=np.int64)
    for a in range(0, n, chunk):
        b = min(a + chunk, n)
        out[a:b] = np.argmax(O.bps_costs(y, phi, W, bits_per_sym, a, b), axis=1)
    return out


def two_stage_parabola_sign_flipped(Dc, S, B):
    """Vertex delta = (D+ - D-) / (2c): the refinement steps away from the minimum."""
    C = Dc.shape[1]
    k = np.arange(Dc.shape[0])
    j = np.argmin(Dc, axis=1)
    Dm, D0, Dp = Dc[k, (j - 1) % C], Dc[k, j], Dc[k, (j + 1) % C]
    c = Dm - 2.0 * D0 + Dp
    delta = np.where(c > 0, (Dp - Dm) / (2.0 * np.where(c > 0, c, 1.0)), 0.0)
    r = np.floor(S * np.clip(delta, -0.5, 0.5) + 0.5).astype(np.int64)
    return (S * j + r) % B


def two_stage_wrong_coarse_grid(y, B, W, bits_per_sym, S, chunk=1 << 15):
    """Coarse angles b = S j + 1 while the index is still read as S j."""
    n = y.size
    phi = ORIG["bps_angles"](B)[1::S]
    out = np.empty(n, dtype=np.int64)
    for a in range(0, n, chunk):
        b = min(a + chunk, n)
        out[a:b] = O.two_stage_index(O.bps_costs(y, phi, W, bits_per_sym, a, b), S, B)
    return out


def unwrap_sign_flipped(bhat, B):
    """Increment from (b_k - b_{k-1}) instead of (b_{k-1} - b_k)."""
    return ORIG["unwrap_increments"](-bhat, B)


def natural_binary_labels(bits_per_sym):
    """16QAM levels labelled 00, 01, 10, 11 (natural binary, not Gray)."""
    if bits_per_sym == 2:
        return ORIG["level_bits"](2)
    return np.array([[0, 0], [0, 1], [1, 0], [1, 1]], dtype=np.uint8)


def prbs_wrong_tap(state, nbits):
    """b[n] = b[n-27] ^ b[n-31] (a neighbouring, wrong feedback tap)."""
    b = np.zeros(max(nbits, 31) + 27, dtype=np.uint8)
    for i in range(31):
        b[i] = (state >> i) & 1
    n = 31
    while n < nbits:
        b[n:n + 27] = b[n - 27:n] ^ b[n - 31:n - 4]
        n += 27
    return b[:nbits]


def ber_count_old_quadrant(lv_idx, ref_bits, cfg, sync, k_s, k_end):
    """Counts a slipped window's errors under the quadrant it slipped from."""
    nl = 1 << (cfg.bits_per_sym // 2)
    bps_ = cfg.bits_per_sym
    d, perm = sync["delay"], sync["perm"]
    errors, bits, slips = 0, 0, 0
    for p in range(2):
        q = sync["quadrant"][p]
        a = k_s
        while a < k_end:
            b = min(a + cfg.slip_window, k_end)
            n = b - a
            lI, lQ = lv_idx[p][0][a:b], lv_idx[p][1][a:b]
            ref = ref_bits[p ^ perm][(a - d) * bps_:(b - d) * bps_].reshape(n, bps_)
            errs = []
            for qq in range(4):
                u, v = O.rotate_quadrants(lI, lQ, qq, nl)
                errs.append(int(np.sum(O._bits_from_levels(u, v, bps_) != ref)))
            counted = errs[q]
            if errs[q] * 4 > n * bps_:
                q = int(np.argmin(errs))
                slips += 1
            errors += counted
            bits += n * bps_
            a = b
    return {"errors": errors, "bits": bits, "slips": slips}


def cma_radius_second_moment(bits_per_sym):
    """E|s|^2 (= 1) instead of E|s|^4 / E|s|^2."""
    lv = O.levels(bits_per_sym)
    pts = (lv[:, None] + 1j * lv[None, :]).ravel()
    return float(np.mean(np.abs(pts) ** 2))


def dd_phase_without_minus(y):
    """arg(sum y^4) / 4: misses the pi of E[s^4] < 0 (a pi/4 offset)."""
    s = np.sum(y ** 4)
    return 0.0 if s == 0 else math.atan2(s.imag, s.real) / 4.0


def q_factor_without_sqrt2(ber):
    """20 log10(erfcinv(2 BER)): the sqrt 2 of Q = sqrt(2) erfcinv(2 BER) dropped."""
    from scipy.special import erfcinv
    return 20.0 * math.log10(float(erfcinv(2.0 * ber)))


def acquire_without_reinit_rule_or_cma(r, n_sym, cfg):
    """Acquisition that never leaves the centre spike (the update step skipped)."""
    return O.centre_spike(cfg.mimo_taps), False


CASES = [
    ("cd_frequency_response", cd_conjugated, lambda: P.test_cd_round_trip_1e12(1000e3)),
    ("ols_cd", ols_kept_window_off_by_one, P.test_ols_exact_for_filters_inside_the_halo),
    ("godard_sum", godard_without_window_sign, P.test_godard_block_sign_for_odd_window_start),
    ("foe_from_periodogram", foe_without_quarter, lambda: P.test_foe_recovers_injected_offset(100e6)),
    ("mimo_fir", mimo_transposed, P.test_mimo_fir_single_tap_is_a_shift),
    ("sub_block_update", sub_block_cma_sign_flipped, P.test_cma_converges_to_inverse_rotation),
    ("bps", bps_maximises, lambda: P.test_bps_recovers_constant_phase_mod_half_pi(2)),
    ("two_stage_index", two_stage_parabola_sign_flipped, P.test_two_stage_refinement_finds_the_vertex_of_a_parabola),
    ("bps_two_stage", two_stage_wrong_coarse_grid, lambda: P.test_two_stage_recovers_an_off_grid_phase_to_one_fine_step(2)),
    ("unwrap_increments", unwrap_sign_flipped, P.test_unwrap_follows_a_ramp_across_quadrants),
    ("level_bits", natural_binary_labels, lambda: P.test_demap_exhaustive_and_gray(4)),
    ("prbs31_bits", prbs_wrong_tap, P.test_prbs_independent_generators_agree),
    ("ber_count", ber_count_old_quadrant, P.test_quarter_turn_phase_jumps_are_counted_as_slips),
    ("cma_radius", cma_radius_second_moment, P.test_cma_radius_values),
    ("dd_phase", dd_phase_without_minus, lambda: P.test_dd_phase_recovers_a_constant_phase(2)),
    ("q_factor_db", q_factor_without_sqrt2, lambda: P.test_q_factor_of_a_gaussian_tail(3.0)),
    ("acquire", acquire_without_reinit_rule_or_cma, P.test_cma_converges_to_inverse_rotation_16qam),
]


@pytest.mark.parametrize("name,bad,pin", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_its_pin(monkeypatch, name, bad, pin):
    pin()  # the real oracle passes
    monkeypatch.setattr(O, name, bad)
    with pytest.raises(AssertionError):
        pin()


def test_every_pinned_function_has_a_planted_case():
    planted = {c[0] for c in CASES}
    for key in O.PIN_STATUS:
        names = {"decide/demap": "level_bits"}.get(key, key)
        assert names in planted, key
