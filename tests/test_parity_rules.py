"""The GPU parity rules themselves, on the CPU: an error confined to one
overlap-save block of a long record must fail the equalised-symbol check
even when the record's overall relative RMS stays inside the bound."""
import numpy as np
import pytest

from parity_util import Y_TOL, check_equalised


def record(n_sym, seed=1):
    rng = np.random.default_rng(seed)
    return (rng.choice([-1.0, 1.0], (2, n_sym)) + 1j * rng.choice([-1.0, 1.0], (2, n_sym))) / np.sqrt(2)


def test_fp32_rounding_passes():
    y = record(1 << 20)
    g = (y.astype(np.complex64)).astype(np.complex128)
    rep = check_equalised(g, y, 1 << 20, 7000)
    assert rep["y_rel_rms_block_max"] < 1e-6


def test_error_in_one_block_of_a_2_21_sample_record_fails():
    """2^20 symbols per polarisation (2^21 samples), one 7,000-symbol block
    (the kept outputs of a 16384-point block with a 2.3k halo, in symbols)
    off by 1e-3: overall rel RMS ~8e-5 < 1e-4, the block's 1e-3 > 1e-4."""
    n, blk = 1 << 20, 7000
    y = record(n)
    g = y.copy()
    a = 5 * blk
    g[:, a:a + blk] *= 1.0 + 1e-3
    glob = np.linalg.norm(g - y) / np.linalg.norm(y)
    assert glob < Y_TOL
    with pytest.raises(AssertionError, match="block"):
        check_equalised(g, y, n, blk)


def test_error_in_one_frame_fails():
    n, F = 1 << 18, 1 << 15
    y = record(n, 2)
    g = y.copy()
    g[:, 3 * F:4 * F] *= 1.0 + 2e-4
    with pytest.raises(AssertionError):
        check_equalised(g, y, F, 1 << 14)


def test_oracle_settings_drop_launch_only_fields():
    """Launch tiles, storage type and block sizes are not method settings:
    the oracle's configuration is built without them."""
    from oracle import rx_oracle as O
    from paper_2108_07001_gb300.workloads import oracle_kwargs
    kw = oracle_kwargs(dict(fiber_len_m=1000e3, modulation=4, mimo_block_warps=2, bps_block_runs=4,
                            storage_dtype=1, max_block_samples=1 << 15))
    cfg = O.RxConfig(**kw)
    assert cfg.bits_per_sym == 4 and cfg.fiber_len_m == 1000e3
