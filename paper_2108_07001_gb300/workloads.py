"""Named synthetic workloads: link (simulator) and receiver settings.

Each entry gives the channel the seeded simulator draws and the receiver
configuration the library and the oracle both run with.  Seeds follow
seed = 1000 + index; stream s of a multi-stream workload uses
seed * 1000 + s.
"""
from __future__ import annotations

DP_QPSK_1000KM = dict(
    name="dp-qpsk-28gbd-1000km-2^16sym",
    link=dict(baud_hz=28e9, bits_per_sym=2, n_sym=1 << 16, fiber_len_m=1000e3, D_ps_nm_km=17.0,
              snr_db=12.0, fo_hz=100e6, linewidth_hz=100e3, rotate=True, prbs_seed=1000, seed=1000,
              out_dtype="c128"),
    rx=dict(baud_hz=28e9, modulation=2, fiber_len_m=1000e3, mimo_taps=15, bps_angles=64,
            bps_half_window=16, frame_syms=1 << 16, prbs_seed=1000),
)

DP_QPSK_10000KM_STREAM = dict(
    name="dp-qpsk-28gbd-10000km-stream-2^24sym",
    link=dict(baud_hz=28e9, bits_per_sym=2, n_sym=1 << 24, fiber_len_m=10000e3, D_ps_nm_km=17.0,
              snr_db=10.0, fo_hz=100e6, linewidth_hz=100e3, rotate=True, prbs_seed=1001, seed=1001,
              out_dtype="c64"),
    rx=dict(baud_hz=28e9, modulation=2, fiber_len_m=10000e3, mimo_taps=15, bps_angles=64,
            bps_half_window=16, frame_syms=1 << 20, seg_syms=512, prbs_seed=1001,
            max_block_samples=1 << 17),
    push_syms=1 << 16,
)

DP_QPSK_64GBD_10000KM_STREAM = dict(
    name="dp-qpsk-64gbd-10000km-stream",
    link=dict(baud_hz=64e9, bits_per_sym=2, n_sym=1 << 22, fiber_len_m=10000e3, D_ps_nm_km=17.0,
              snr_db=12.0, fo_hz=100e6, linewidth_hz=100e3, rotate=True, prbs_seed=1005, seed=1005,
              out_dtype="c64"),
    rx=dict(baud_hz=64e9, modulation=2, fiber_len_m=10000e3, mimo_taps=15, bps_angles=64,
            bps_half_window=16, frame_syms=1 << 20, seg_syms=512, prbs_seed=1005,
            max_block_samples=1 << 17),
    push_syms=1 << 16,
)

DP_16QAM_5000KM = dict(
    name="dp-16qam-32gbd-5000km-2^22sym",
    link=dict(baud_hz=32e9, bits_per_sym=4, n_sym=1 << 22, fiber_len_m=5000e3, D_ps_nm_km=17.0,
              snr_db=18.0, fo_hz=100e6, linewidth_hz=100e3, rotate=True, prbs_seed=1002, seed=1002,
              out_dtype="c16"),
    rx=dict(baud_hz=32e9, modulation=4, fiber_len_m=5000e3, mimo_taps=25, bps_angles=32,
            bps_half_window=32, frame_syms=1 << 20, prbs_seed=1002, mu_dd=2e-3),
)

ALL = [DP_QPSK_1000KM, DP_QPSK_10000KM_STREAM, DP_16QAM_5000KM, DP_QPSK_64GBD_10000KM_STREAM]
STREAMS = {w["name"]: w for w in (DP_QPSK_10000KM_STREAM, DP_QPSK_64GBD_10000KM_STREAM)}


def oracle_kwargs(rx: dict) -> dict:
    """The receiver settings in the oracle's field names."""
    m = dict(rx)
    m.pop("max_block_samples", None)
    m.pop("storage_dtype", None)
    m.pop("mimo_block_warps", None)  # launch tiles: no effect on any result
    m.pop("bps_block_runs", None)
    if "modulation" in m:
        m["bits_per_sym"] = m.pop("modulation")
    return m
