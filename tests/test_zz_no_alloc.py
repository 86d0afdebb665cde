"""The allocation-free block-decision entry point (rx_decide_block_noalloc).

Some callers cannot enter the CUDA allocator (a capture thread with a hard
deadline, or a process whose device memory is held by another pool
allocator).  For them the library decides a block of equalised symbols
with all working memory in one static device array.  These tests check,
through the C ABI, that calls in a row give the same bits as the streaming
receiver's own decisions for the same symbols, for both modulations,
several angle counts and half windows, a block length that is neither a
whole number of bytes of bits nor of BPS runs, and a short block decided
right after a longer one (the array keeps the longer call's tail, which
must not be read).  The file is collected last and passes alone or after
the other tests."""
import ctypes

import numpy as np
import pytest

import rxsim

pytestmark = pytest.mark.gpu


def streaming_decisions(n_sym, modulation, B, W, seed):
    """A one-frame stream of n_sym symbols through the streaming receiver:
    its equalised symbols (device, [2, n] complex64) and its decided bits."""
    import torch
    from paper_2108_07001_gb300 import rx

    if modulation == 2:
        link = dict(baud_hz=28e9, bits_per_sym=2, snr_db=12.0, fiber_len_m=800e3)
        cfg = dict(baud_hz=28e9, modulation=2, fiber_len_m=800e3)
    else:
        link = dict(baud_hz=32e9, bits_per_sym=4, snr_db=18.0, fiber_len_m=500e3)
        cfg = dict(baud_hz=32e9, modulation=4, fiber_len_m=500e3, mimo_taps=25, mu_dd=2e-3)
    sim = rxsim.simulate(rxsim.LinkConfig(n_sym=n_sym, seed=seed, prbs_seed=11, out_dtype="c64", **link))
    r = rx.Receiver(frame_syms=1 << 15, acq_syms=8192, history_syms=n_sym, max_block_samples=2 * n_sym,
                    bps_angles=B, bps_half_window=W, **cfg)
    r.push_tensor(torch.from_numpy(sim["rx"]).to("cuda:0"))
    r.end()
    bits = r.pull_bits(1 << 21)
    y = r.equalised(0, n_sym)
    r.close()
    assert bits.size == n_sym * 2 * modulation
    return torch.from_numpy(np.ascontiguousarray(y)).to("cuda:0"), bits


def decide(yd, n_sym, modulation, B, W):
    import torch
    from paper_2108_07001_gb300 import rx

    lib = rx.load()
    nbits = n_sym * 2 * modulation
    out = torch.full(((nbits + 7) // 8,), 0xA5, dtype=torch.uint8, device="cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.rx_decide_block_noalloc(ctypes.c_void_p(yd.data_ptr()), n_sym, modulation, B, W,
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    assert rc == rx.RX_OK, lib.rx_last_error().decode()
    torch.cuda.synchronize()
    return np.unpackbits(out.cpu().numpy())[:nbits]


@pytest.mark.parametrize("modulation,B,W", [(2, 64, 16), (2, 32, 8), (4, 32, 32), (4, 64, 24)],
                         ids=["qpsk-B64-W16", "qpsk-B32-W8", "qam16-B32-W32", "qam16-B64-W24"])
def test_noalloc_decisions_equal_the_streaming_receiver(modulation, B, W):
    long_n, short_n = 1 << 15, 12345  # 12345: odd, not a whole number of runs
    y_long, ref_long = streaming_decisions(long_n, modulation, B, W, 321)
    y_short, ref_short = streaming_decisions(short_n, modulation, B, W, 654)
    assert np.array_equal(decide(y_long, long_n, modulation, B, W), ref_long)
    for _ in range(2):  # a short block after a longer one, twice in a row
        assert np.array_equal(decide(y_short, short_n, modulation, B, W), ref_short)


def test_noalloc_rejects_bad_arguments():
    import torch
    from paper_2108_07001_gb300 import rx

    lib = rx.load()
    y = torch.zeros((2, 8), dtype=torch.complex64, device="cuda:0")
    out = torch.zeros(8, dtype=torch.uint8, device="cuda:0")
    rc = lib.rx_decide_block_noalloc(ctypes.c_void_p(y.data_ptr()), 65537, rx.RX_QPSK, 64, 16,
                                     ctypes.c_void_p(out.data_ptr()), None)
    assert rc == rx.RX_EINVAL
    assert "RX_NOALLOC_MAX_SYMS" in lib.rx_last_error().decode()
    # a pointer 4 bytes into the block is not a complex float: refused before any launch
    rc = lib.rx_decide_block_noalloc(ctypes.c_void_p(y.data_ptr() + 4), 4, rx.RX_QPSK, 64, 16,
                                     ctypes.c_void_p(out.data_ptr()), None)
    assert rc == rx.RX_EINVAL
    assert "aligned" in lib.rx_last_error().decode()
