"""The allocation-free block-decision entry point (rx_decide_block_noalloc).

Some callers cannot enter the CUDA allocator (a capture thread with a hard
deadline, or a process whose device memory is held by another pool
allocator).  For them the library decides a block of equalised symbols
with all working memory in one static device array.  This test checks,
through the C ABI, that two calls in a row give the same bits as the
streaming receiver's own decisions for the same symbols.  It lives in its
own file, collected last, and passes alone or after the other tests."""
import ctypes

import numpy as np
import pytest

import rxsim

pytestmark = pytest.mark.gpu


def test_noalloc_decisions_equal_the_streaming_receiver():
    import torch
    from paper_2108_07001_gb300 import rx

    n_sym = 1 << 14
    sim = rxsim.simulate(rxsim.LinkConfig(n_sym=n_sym, snr_db=12.0, fiber_len_m=800e3, seed=321,
                                          prbs_seed=11, out_dtype="c64"))
    r = rx.Receiver(fiber_len_m=800e3, frame_syms=n_sym, acq_syms=8192, history_syms=n_sym,
                    max_block_samples=2 * n_sym)
    r.push_tensor(torch.from_numpy(sim["rx"]).to("cuda:0"))
    r.end()
    ref = r.pull_bits(1 << 20)            # the streaming receiver's decisions
    y = r.equalised(0, n_sym)             # the symbols it decided, [2, n] complex64
    r.close()
    assert ref.size == n_sym * 4

    lib = rx.load()
    yd = torch.from_numpy(np.ascontiguousarray(y)).to("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    nbytes = n_sym * 4 // 8
    for _ in range(2):                    # the array keeps the previous call's contents
        out = torch.full((nbytes,), 0xA5, dtype=torch.uint8, device="cuda:0")
        rc = lib.rx_decide_block_noalloc(ctypes.c_void_p(yd.data_ptr()), n_sym, rx.RX_QPSK, 64, 16,
                                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert rc == rx.RX_OK, lib.rx_last_error().decode()
        torch.cuda.synchronize()
        got = np.unpackbits(out.cpu().numpy())[:ref.size]
        assert np.array_equal(got, ref)


def test_noalloc_rejects_oversized_blocks():
    import torch
    from paper_2108_07001_gb300 import rx

    lib = rx.load()
    y = torch.zeros((2, 8), dtype=torch.complex64, device="cuda:0")
    out = torch.zeros(8, dtype=torch.uint8, device="cuda:0")
    rc = lib.rx_decide_block_noalloc(ctypes.c_void_p(y.data_ptr()), 65537, rx.RX_QPSK, 64, 16,
                                     ctypes.c_void_p(out.data_ptr()), None)
    assert rc == rx.RX_EINVAL
    assert "RX_NOALLOC_MAX_SYMS" in lib.rx_last_error().decode()
