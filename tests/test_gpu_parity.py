"""GPU parity: the CUDA receiver (through the C ABI) against the FP64 oracle
on the same seeded inputs.  Tolerances are in tests/parity_util.py."""
import math

import numpy as np
import pytest

import rxsim
from paper_2108_07001_gb300 import workloads
from parity_util import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def link(**kw):
    return rxsim.LinkConfig(**kw)


STRIDES = pytest.mark.parametrize("stride", [1, 4], ids=["full_bps", "two_stage_bps"])


@STRIDES
def test_config0_parity(stride):
    """DP-QPSK 28 GBd, 2^16 symbols, complex128 input, 1,000 km, all
    impairments at 12 dB: one frame, pushed whole (full and two-stage BPS)."""
    wl = workloads.DP_QPSK_1000KM
    rx_kw = dict(wl["rx"], bps_coarse_stride=stride)
    sim = rxsim.simulate(link(**wl["link"]))
    gpu, r = run_gpu(sim["rx"], rx_kw)
    ref = run_oracle(sim["rx"], rx_kw)
    rep = compare(gpu, ref, rx_kw)
    st = gpu["stats"]
    b = ref["ber"]
    assert st["synced"] == 1
    assert (st["sync_delay"], st["sync_perm"]) == (b["sync"]["delay"], b["sync"]["perm"])
    assert st["bits"] == b["bits"]
    assert abs(int(st["bit_errors"]) - b["errors"]) <= 2 * rep.get("bit_mismatch_syms", 0) * 2 + 2
    assert st["cycle_slips"] == b["slips"]
    assert abs(st["evm"] - b["evm"]) <= 1e-3 * b["evm"] + 1e-6
    from oracle import rx_oracle as O
    assert abs(st["q_db"] - O.q_factor_db(st["ber"])) < 1e-9
    tr = gpu["trace"]
    assert abs(tr[0, 0] - ref["trace"]["tau"][0]) * 28e9 < 1e-4
    assert abs(tr[0, 1] - ref["trace"]["dfo"][0]) < 1e3
    assert abs(tr[0, 2] - ref["trace"]["gain"][0]) < 1e-5
    r.close()


@STRIDES
def test_multi_frame_ragged_pushes(stride):
    """Four frames plus a ragged tail, pushed in irregular blocks: state
    (OLS overlap, FO phase, timing, adaptive chains, BPS window, unwrap)
    carried across pushes and frames."""
    F = 1 << 13
    n_sym = 4 * F + 1234
    sim = rxsim.simulate(link(n_sym=n_sym, snr_db=11.0, fiber_len_m=2000e3, prbs_seed=31, seed=1234,
                              out_dtype="c64"))
    rx_kw = dict(fiber_len_m=2000e3, frame_syms=F, acq_syms=F, cma_syms=4096, prbs_seed=31, seg_syms=512,
                 ber_skip_syms=2048, sync_syms=2048, bps_coarse_stride=stride)
    n = sim["rx"].shape[1]
    pushes = []
    rng = np.random.default_rng(3)
    left = n
    while left:
        m = int(min(left, rng.integers(1, 9000)))
        pushes.append(m)
        left -= m
    gpu, r = run_gpu(sim["rx"], rx_kw, pushes=pushes)
    ref = run_oracle(sim["rx"], rx_kw)
    compare(gpu, ref, rx_kw)
    tr = gpu["trace"]
    assert tr.shape[0] == len(ref["trace"]["tau"]) == 5
    assert np.allclose(tr[:, 0], ref["trace"]["tau"], atol=1e-4 / 28e9)
    assert np.allclose(tr[:, 1], ref["trace"]["dfo"], atol=2e3)
    assert np.allclose(tr[:, 2], ref["trace"]["gain"], rtol=1e-5)
    assert np.allclose(np.unwrap(tr[:, 3]), np.unwrap(ref["trace"]["theta"]), atol=1e-4)
    st = gpu["stats"]
    assert st["bits"] == ref["ber"]["bits"]
    r.close()


@STRIDES
def test_cycle_slips_counted_like_the_oracle(stride):
    """Abrupt +-pi/2 and pi carrier steps (1 km: no dispersion to smear
    them) in a four-frame stream at 13 dB, one of them at a frame boundary:
    the GPU's slip pass (a chunk of windows run in parallel from every start
    state, the maps composed in order) gives the oracle's sequential counts."""
    F = 1 << 13
    n_sym = 4 * F + 777
    jumps = ((2 * 9000 + 1, math.pi / 2), (2 * 14100, -math.pi / 2), (2 * 16390, math.pi / 2),
             (2 * 25000 + 1, math.pi))
    sim = rxsim.simulate(link(n_sym=n_sym, snr_db=13.0, fiber_len_m=1e3, prbs_seed=9, seed=77, out_dtype="c64",
                              phase_jumps=jumps))
    rx_kw = dict(fiber_len_m=1e3, frame_syms=F, acq_syms=F, cma_syms=4096, prbs_seed=9, ber_skip_syms=2048,
                 sync_syms=2048, bps_coarse_stride=stride)
    gpu, r = run_gpu(sim["rx"], rx_kw)
    ref = run_oracle(sim["rx"], rx_kw)
    rep = compare(gpu, ref, rx_kw)
    st, b = gpu["stats"], ref["ber"]
    assert b["slips"] == 8  # one per polarisation and step
    assert st["cycle_slips"] == b["slips"]
    assert st["bits"] == b["bits"]
    assert abs(int(st["bit_errors"]) - b["errors"]) <= 2 * rep.get("bit_mismatch_syms", 0) * 2 + 2
    r.close()


@STRIDES
def test_qam16_parity(stride):
    """DP-16QAM 32 GBd, T = 25, B = 32, W = 32 over 5,000 km at 18 dB (full
    search, and two-stage over 8 coarse angles)."""
    sim = rxsim.simulate(link(baud_hz=32e9, bits_per_sym=4, n_sym=1 << 15, fiber_len_m=5000e3, snr_db=18.0,
                              prbs_seed=17, seed=1002, out_dtype="c64"))
    rx_kw = dict(baud_hz=32e9, modulation=4, fiber_len_m=5000e3, mimo_taps=25, bps_angles=32,
                 bps_half_window=32, frame_syms=1 << 15, prbs_seed=17, mu_dd=2e-3, bps_coarse_stride=stride)
    gpu, r = run_gpu(sim["rx"], rx_kw)
    ref = run_oracle(sim["rx"], rx_kw)
    compare(gpu, ref, rx_kw)
    assert gpu["stats"]["bits"] == ref["ber"]["bits"]
    r.close()


@STRIDES
def test_fp16_storage_parity(stride):
    """Complex-half storage: the oracle runs on the same half-precision
    samples, so only the arithmetic differs (full and two-stage BPS)."""
    sim = rxsim.simulate(link(n_sym=1 << 15, snr_db=12.0, fiber_len_m=1000e3, prbs_seed=5, seed=55,
                              out_dtype="c16"))
    rx_kw = dict(fiber_len_m=1000e3, frame_syms=1 << 15, prbs_seed=5, storage_dtype=2, bps_coarse_stride=stride)
    gpu, r = run_gpu(sim["rx"], rx_kw)
    ref = run_oracle(sim["rx"], rx_kw)
    compare(gpu, ref, rx_kw)
    r.close()


def test_c128_input_equals_c64_input_rounded():
    sim = rxsim.simulate(link(n_sym=1 << 14, snr_db=12.0, fiber_len_m=800e3, seed=66))
    rx_kw = dict(fiber_len_m=800e3, frame_syms=1 << 14, acq_syms=8192)
    g1, r1 = run_gpu(sim["rx"], rx_kw)
    g2, r2 = run_gpu(sim["rx"].astype(np.complex64), rx_kw)
    assert np.array_equal(g1["y"], g2["y"])
    r1.close()
    r2.close()


def test_noiseless_stream_is_error_free():
    sim = rxsim.simulate(link(n_sym=1 << 16, snr_db=None, fiber_len_m=3000e3, prbs_seed=8, seed=8,
                              out_dtype="c64"))
    rx_kw = dict(fiber_len_m=3000e3, frame_syms=1 << 14, acq_syms=8192, prbs_seed=8, ber_skip_syms=4096)
    gpu, r = run_gpu(sim["rx"], rx_kw, pushes=[1 << 15] * 4, history=False)
    st = gpu["stats"]
    # counted: symbols [4096, 2^16 - tail) of both polarisations, 2 bits each
    assert st["synced"] and st["bit_errors"] == 0 and st["cycle_slips"] == 0 and st["bits"] > 240000
    r.close()


# ------------------------------------------------------------ edge cases ---

def test_empty_stream_and_state_errors():
    from paper_2108_07001_gb300 import rx
    r = rx.Receiver(frame_syms=4096, acq_syms=2048, cma_syms=1024)
    r.end()
    assert r.pull_bits(16).size == 0
    with pytest.raises(rx.RxError) as e:
        r.push_host(np.zeros((2, 8), np.complex64))
    assert e.value.code == rx.RX_ESTATE
    r.close()


def test_push_too_large_and_bad_dtype():
    import ctypes
    from paper_2108_07001_gb300 import rx
    r = rx.Receiver(frame_syms=4096, acq_syms=2048, cma_syms=1024, max_block_samples=1000)
    with pytest.raises(rx.RxError) as e:
        r.push_host(np.zeros((2, 1001), np.complex64))
    assert e.value.code == rx.RX_EINVAL
    x = np.zeros((2, 10), np.complex64)
    assert r.lib.rx_push_block(r.h, x.ctypes.data_as(ctypes.c_void_p), 10, 7, 0, None) == rx.RX_EINVAL
    r.close()


def test_stream_shorter_than_acquisition():
    sim = rxsim.simulate(link(n_sym=3000, snr_db=15.0, fiber_len_m=300e3, seed=3))
    rx_kw = dict(fiber_len_m=300e3, frame_syms=4096, acq_syms=4096, cma_syms=2048)
    gpu, r = run_gpu(sim["rx"], rx_kw)
    ref = run_oracle(sim["rx"], rx_kw)
    compare(gpu, ref, rx_kw, check_bits=True)
    assert gpu["bits"].size == 3000 * 4
    r.close()


def test_backpressure_when_bits_are_not_pulled():
    import torch
    from paper_2108_07001_gb300 import rx
    r = rx.Receiver(frame_syms=1 << 16, max_block_samples=1 << 17)
    x = torch.zeros((2, 1 << 17), dtype=torch.complex64, device="cuda:0")
    codes = []
    for _ in range(64):
        try:
            r.push_tensor(x)
        except rx.RxError as e:
            codes.append(e.code)
            break
    assert codes == [rx.RX_EAGAIN]
    got = r.pull_bits(1 << 22)
    assert got.size > 0
    r.push_tensor(x)  # room again
    r.close()


def test_reset_reproduces_the_stream():
    sim = rxsim.simulate(link(n_sym=1 << 14, snr_db=12.0, fiber_len_m=600e3, prbs_seed=4, seed=4,
                              out_dtype="c64"))
    rx_kw = dict(fiber_len_m=600e3, frame_syms=1 << 14, acq_syms=8192, prbs_seed=4, ber_skip_syms=4096)
    g1, r = run_gpu(sim["rx"], rx_kw)
    r.reset()
    import torch
    r.push_tensor(torch.from_numpy(sim["rx"]).to("cuda:0"))
    r.end()
    bits = r.pull_bits(1 << 20)
    assert np.array_equal(bits, g1["bits"])
    assert r.stats()["bit_errors"] == g1["stats"]["bit_errors"]
    r.close()


def test_host_push_equals_device_push():
    sim = rxsim.simulate(link(n_sym=1 << 14, snr_db=12.0, fiber_len_m=600e3, seed=9, out_dtype="c64"))
    rx_kw = dict(fiber_len_m=600e3, frame_syms=1 << 14, acq_syms=8192)
    g1, r1 = run_gpu(sim["rx"], rx_kw)
    from paper_2108_07001_gb300 import rx
    r2 = rx.Receiver(**rx_kw, max_block_samples=1 << 15)
    r2.push_host(sim["rx"])
    r2.end()
    bits = r2.pull_bits(1 << 20)
    assert np.array_equal(bits, g1["bits"])
    r1.close()
    r2.close()


def test_autotuned_fft_size_is_admissible_and_keeps_parity():
    """The autotuner's FFT size is admissible for the CD length and the chain
    with it still matches the oracle (the OLS result does not depend on N
    beyond rounding)."""
    from paper_2108_07001_gb300 import rx
    rx_kw = dict(fiber_len_m=3000e3, frame_syms=1 << 14, prbs_seed=41, cma_syms=8192, acq_syms=12288,
                 ber_skip_syms=4096)
    n, ms = rx.autotune_fft(rx.default_config(**rx_kw), frames=2)
    assert n in (1024, 2048, 4096, 8192, 16384, 32768) and ms > 0
    sim = rxsim.simulate(link(n_sym=1 << 15, snr_db=12.0, fiber_len_m=3000e3, prbs_seed=41, seed=41))
    kw = dict(rx_kw, fft_n=n)
    gpu, r = run_gpu(sim["rx"], kw)
    ref = run_oracle(sim["rx"], kw)
    compare(gpu, ref, kw)
    r.close()


def test_pinned_host_push_equals_device_push():
    """Page-locked host blocks taken in stream order, copied by a copy
    engine (on_device = 2) or read by the ingest kernel through the device
    mapping (on_device = 3), give exactly the device-push result; unpinned
    memory is refused."""
    import torch
    from paper_2108_07001_gb300 import rx
    sim = rxsim.simulate(link(n_sym=1 << 15, snr_db=12.0, fiber_len_m=600e3, seed=88, out_dtype="c64"))
    rx_kw = dict(fiber_len_m=600e3, frame_syms=1 << 14, acq_syms=8192, history_syms=1 << 15, max_block_samples=1 << 14)
    x = np.ascontiguousarray(sim["rx"])
    blocks = [np.ascontiguousarray(x[:, a:a + (1 << 14)]) for a in range(0, x.shape[1], 1 << 14)]
    out = []
    for mode in ("device", "pinned", "mapped"):
        r = rx.Receiver(**rx_kw)
        stream = torch.cuda.current_stream().cuda_stream
        keep = []
        for b in blocks:
            if mode == "device":
                t = torch.from_numpy(b).to("cuda:0")
                keep.append(t)
                r.push_device(t.data_ptr(), b.shape[1], rx.RX_C64, stream)
            else:
                t = torch.from_numpy(b).pin_memory()
                keep.append(t)
                if mode == "pinned":
                    r.push_pinned(t.data_ptr(), b.shape[1], rx.RX_C64, stream)
                else:
                    r.push_mapped(t.data_ptr(), b.shape[1], rx.RX_C64, stream)
        r.end()
        buf = np.empty(1 << 20, dtype=np.uint8)
        nb = r.pull_bytes(buf, timeout_ms=-1)
        out.append((buf[:(nb + 7) // 8].copy(), r.equalised(0, 1 << 15)))
        if mode != "device":
            with pytest.raises(rx.RxError):
                r2 = rx.Receiver(**rx_kw)
                try:
                    push = r2.push_pinned if mode == "pinned" else r2.push_mapped
                    push(blocks[0].ctypes.data, blocks[0].shape[1], rx.RX_C64, stream)
                finally:
                    r2.close()
        r.close()
    for k in (1, 2):
        assert np.array_equal(out[0][0], out[k][0])
        assert np.array_equal(out[0][1], out[k][1])


# ------------------------------------------------- the bench's own workload ---

def test_headline_stream_parity_two_frames():
    """The bench workload's receiver exactly as the bench runs it (28 GBd,
    10,000 km: N = 16384 by the default rule, frames of 2^20 symbols,
    512-symbol segment chains, complex64 pushes of 2^16 symbols) on the
    first 2^21 symbols per polarisation of the bench's own samples: two
    frames, so the second frame's segment chains, overlap, FO phase and
    timing continue from the first.  Equalised symbols, BPS angles and bits
    follow the parity rules; the BER counters, sync and slips equal the
    oracle's on the same samples."""
    from oracle import rx_oracle as O
    wl = workloads.DP_QPSK_10000KM_STREAM
    n_sym = 1 << 21
    x = rxsim.simulate(link(**wl["link"]))["rx"][:, :2 * n_sym]
    rx_kw = dict(wl["rx"])
    assert O.geometry(O.RxConfig(**workloads.oracle_kwargs(rx_kw))).N == 16384
    m = 2 * wl["push_syms"]
    gpu, r = run_gpu(x, rx_kw, pushes=[m] * (2 * n_sym // m))
    ref = run_oracle(x, rx_kw)
    rep = compare(gpu, ref, rx_kw)
    st, b = gpu["stats"], ref["ber"]
    assert st["frames"] == 2 and len(ref["trace"]["tau"]) == 2
    assert st["synced"] == 1
    assert (st["sync_delay"], st["sync_perm"]) == (b["sync"]["delay"], b["sync"]["perm"])
    assert [st["sync_quadrant_x"], st["sync_quadrant_y"]] == [int(q) for q in b["sync"]["quadrant"]]
    assert st["bits"] == b["bits"]
    assert abs(int(st["bit_errors"]) - b["errors"]) <= 2 * rep.get("bit_mismatch_syms", 0)
    assert st["cycle_slips"] == b["slips"]
    assert abs(st["q_db"] - O.q_factor_db(st["ber"])) < 1e-9
    tr = gpu["trace"]
    assert np.allclose(tr[:, 0], ref["trace"]["tau"], atol=1e-4 / 28e9)
    assert np.allclose(tr[:, 2], ref["trace"]["gain"], rtol=1e-5)
    r.close()


@pytest.mark.parametrize("fft_n", [0, 16384], ids=["default_32768", "fft_16384"])
def test_64gbd_10000km_parity(fft_n):
    """64 GBd over 10,000 km, a CD halo of ~13.5k samples: the default rule
    takes the 32768-point transform (a cluster of two CTAs per block, ~59 %
    of each block kept); forced to 16384 points, the largest halo fraction
    the single-CTA kernel meets (~18 % kept).  Two frames of 2^17 symbols
    pushed in 2^16-symbol blocks."""
    from oracle import rx_oracle as O
    n_sym = 1 << 18
    sim = rxsim.simulate(link(baud_hz=64e9, n_sym=n_sym, fiber_len_m=10000e3, snr_db=12.0, prbs_seed=64,
                              seed=6400, out_dtype="c64"))
    rx_kw = dict(baud_hz=64e9, fiber_len_m=10000e3, frame_syms=1 << 17, prbs_seed=64, fft_n=fft_n)
    assert O.geometry(O.RxConfig(**workloads.oracle_kwargs(rx_kw))).N == (fft_n or 32768)
    gpu, r = run_gpu(sim["rx"], rx_kw, pushes=[1 << 17] * (2 * n_sym >> 17))
    ref = run_oracle(sim["rx"], rx_kw)
    rep = compare(gpu, ref, rx_kw)
    st, b = gpu["stats"], ref["ber"]
    assert st["bits"] == b["bits"] and st["cycle_slips"] == b["slips"]
    assert abs(int(st["bit_errors"]) - b["errors"]) <= 2 * rep.get("bit_mismatch_syms", 0)
    tr = gpu["trace"]
    assert np.allclose(tr[:, 0], ref["trace"]["tau"], atol=1e-4 / 64e9)
    assert np.allclose(tr[:, 1], ref["trace"]["dfo"], atol=2e3)
    assert np.allclose(tr[:, 2], ref["trace"]["gain"], rtol=1e-5)
    r.close()


def test_32768_point_transform_ragged_pushes_fp16():
    """The two-CTA 32768-point form with irregular pushes, FP16 storage and
    three frames plus a ragged tail (the last block of each frame partial,
    the stream edge zero-padded)."""
    F = 1 << 14
    n_sym = 3 * F + 3333
    sim = rxsim.simulate(link(baud_hz=56e9, n_sym=n_sym, fiber_len_m=6000e3, snr_db=13.0, prbs_seed=56, seed=5600,
                              out_dtype="c16"))
    rx_kw = dict(baud_hz=56e9, fiber_len_m=6000e3, frame_syms=F, acq_syms=F, cma_syms=8192, prbs_seed=56,
                 ber_skip_syms=8192, sync_syms=2048, fft_n=32768, storage_dtype=2)
    n = sim["rx"].shape[1]
    pushes, left = [], n
    rng = np.random.default_rng(56)
    while left:
        m = int(min(left, rng.integers(1000, 40000)))
        pushes.append(m)
        left -= m
    gpu, r = run_gpu(sim["rx"], rx_kw, pushes=pushes)
    ref = run_oracle(sim["rx"], rx_kw)
    compare(gpu, ref, rx_kw)
    assert gpu["stats"]["bits"] == ref["ber"]["bits"]
    r.close()


def test_launch_tiles_do_not_change_results():
    """Every equaliser tile (1, 2, 4, 8 segment chains per block) and BPS
    tile (4, 8 runs per block) gives bit for bit the same bits, equalised
    symbols and counters; the tile autotuner returns admissible tiles."""
    from paper_2108_07001_gb300 import rx
    F = 1 << 14
    sim = rxsim.simulate(link(n_sym=3 * F + 700, snr_db=12.0, fiber_len_m=1500e3, prbs_seed=15, seed=1515,
                              out_dtype="c64"))
    base = dict(fiber_len_m=1500e3, frame_syms=F, acq_syms=8192, cma_syms=4096, prbs_seed=15, ber_skip_syms=4096)
    ref = None
    for mw, br in ((4, 8), (1, 8), (2, 4), (8, 4)):
        gpu, r = run_gpu(sim["rx"], dict(base, mimo_block_warps=mw, bps_block_runs=br), pushes=[20000] * 4 + [
            sim["rx"].shape[1] - 80000])
        st = gpu["stats"]
        got = (gpu["bits"], gpu["y"], st["bit_errors"], st["bits"], st["cycle_slips"])
        r.close()
        if ref is None:
            ref = got
            continue
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), (mw, br)
        assert got[2:] == ref[2:], (mw, br)
    t = rx.autotune_tiles(rx.default_config(**base), frames=2)
    assert t["fft_n"] in (1024, 2048, 4096, 8192, 16384, 32768)
    assert t["mimo_block_warps"] in (1, 2, 4, 8) and t["bps_block_runs"] in (4, 8) and t["ms_per_msample"] > 0
