"""GPU parity of the KK receiver chain (rx_kkrx_*: KK field, static
equaliser with 4 -> 2 samples per symbol, widely-linear DD-LMS, decisions)
against the FP64 oracle on the same seeded ADC codes.

Tolerances: equalised symbols relative RMS <= 1e-4 (the FP32 chain of two
overlap-save stages and a block-LMS whose taps follow the oracle's schedule;
rounding perturbs them at ~1e-6); decided bits identical except for symbols
whose oracle value lies within 1e-3 of a decision threshold."""
import numpy as np
import pytest

import rxsim
from oracle import kk_oracle as K
from oracle import rx_oracle as O
from paper_2108_07001_gb300 import rx

pytestmark = pytest.mark.gpu

Y_TOL = 1e-4
BOUNDARY = 1e-3
B2 = rxsim.beta2_from_dispersion(17.0, 1550e-9)


def case(bits_per_sym, n_sym, seed, cspr, snr, L=1000e3):
    d = rxsim.simulate_kk(rxsim.KKLinkConfig(n_sym=n_sym, bits_per_sym=bits_per_sym, fiber_len_m=L, cspr_db=cspr,
                                             snr_db=snr, seed=seed, prbs_seed=seed))
    return d


def chain_cfg(d, bits_per_sym, F, S=512, acq=4096, mu=5e-3, L=1000e3, block=1 << 16, hist=0):
    return rx.default_kkrx_config(
        dict(fs_hz=d["fs"], f_shift_hz=d["f_c"], adc_gain=d["gain"], adc_offset=d["offset"], fft_n=1024,
             max_block_samples=block),
        baud_hz=1e9, modulation=bits_per_sym, fiber_len_m=L, rrc_rolloff=0.01, eq_fft_n=1024, mu=mu, seg_syms=S,
        frame_syms=F, acq_syms=acq, history_syms=hist)


def run_chain(d, cfg, sizes, host_every=0):
    import torch
    codes = d["codes"]
    n_sym = codes.size // 4
    nbytes = (n_sym * cfg.modulation + 7) // 8
    dev = torch.device("cuda:0")
    dc = torch.from_numpy(codes).to(dev)
    bits = torch.zeros(nbytes + 64, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    nb_total = 0
    with rx.KKReceiver(cfg) as r:
        a = 0
        for i, m in enumerate(sizes):
            off = nb_total // 8
            if host_every and i % host_every == 0:
                nb = r.push_host(codes[a:a + m], bits.data_ptr() + off, bits.numel() - off, stream)
            else:
                nb = r.push_device(dc.data_ptr() + 2 * a, m, bits.data_ptr() + off, bits.numel() - off, stream)
            assert nb % 8 == 0
            nb_total += nb
            a += m
        nb_total += r.end(bits.data_ptr() + nb_total // 8, bits.numel() - nb_total // 8, stream)
        torch.cuda.synchronize()
        y = r.equalised(0, cfg.history_syms) if cfg.history_syms else None
    assert nb_total == n_sym * cfg.modulation
    return np.unpackbits(bits.cpu().numpy())[:nb_total], y


def oracle(d, cfg):
    return K.kk_receive(d["codes"], d["gain"], d["offset"], d["fs"], d["f_c"], 1024, cfg.eq_fft_n, 1e9,
                        cfg.rrc_rolloff, B2, cfg.fiber_len_m, cfg.modulation, cfg.mu, 64, cfg.seg_syms,
                        cfg.frame_syms, cfg.acq_syms)


def compare(bits, y, ref, bits_per_sym):
    n = ref["y"].size
    rel = float(np.linalg.norm(y - ref["y"]) / np.linalg.norm(ref["y"]))
    assert rel <= Y_TOL, rel
    lv = O.levels(bits_per_sym)
    thr = 0.5 * (lv[1:] + lv[:-1])
    near = np.zeros(n, dtype=bool)
    for t in thr:
        near |= (np.abs(ref["y"].real - t) < BOUNDARY) | (np.abs(ref["y"].imag - t) < BOUNDARY)
    mism = np.any(bits.reshape(n, bits_per_sym) != ref["bits"].reshape(n, bits_per_sym), axis=1)
    assert not (mism & ~near).any(), int((mism & ~near).sum())
    return rel, int(mism.sum())


def ragged(n, seed, hi):
    rng = np.random.default_rng(seed)
    sizes, left = [], n
    while left:
        m = int(min(left, rng.integers(1, hi)))
        sizes.append(m)
        left -= m
    return sizes


@pytest.mark.parametrize("bits_per_sym,cspr,snr,mu", [(2, 12.0, 7.0, 5e-3), (4, 16.0, 13.0, 2e-3)],
                         ids=["qpsk", "16qam"])
def test_chain_matches_the_oracle(bits_per_sym, cspr, snr, mu):
    """Three 8192-symbol frames and a ragged tail, ragged pushes mixing host
    and device memory, at an SNR that leaves a BER of 1e-3 to 2e-3 (SNR per
    4-sps sample over the whole band): symbols and bits against the oracle;
    the bits' errors against the transmitted PRBS are the oracle's."""
    F = 1 << 13
    n_sym = 3 * F + 1111
    d = case(bits_per_sym, n_sym, 61 + bits_per_sym, cspr, snr)
    cfg = chain_cfg(d, bits_per_sym, F, mu=mu, hist=n_sym)
    bits, y = run_chain(d, cfg, ragged(d["codes"].size, 5, 30000), host_every=4)
    ref = oracle(d, cfg)
    rel, mism = compare(bits, y, ref, bits_per_sym)
    tx = d["bits"][:bits.size]
    a, e = 2 * 1024 * bits_per_sym, bits.size - 2 * 64 * bits_per_sym
    err_gpu = int(np.sum(bits[a:e] != tx[a:e]))
    err_orc = int(np.sum(ref["bits"][a:e] != tx[a:e]))
    assert abs(err_gpu - err_orc) <= bits_per_sym * mism
    assert err_orc / (e - a) < 1e-2


def test_push_sizes_and_memory_do_not_change_the_result():
    F = 1 << 12
    d = case(2, 2 * F + 321, 71, 12.0, 22.0)
    cfg = chain_cfg(d, 2, F, acq=2048, hist=0)
    n = d["codes"].size
    b1, _ = run_chain(d, cfg, [n])
    b2, _ = run_chain(d, cfg, ragged(n, 6, 5000))
    b3, _ = run_chain(d, cfg, ragged(n, 7, 9000), host_every=1)
    assert np.array_equal(b1, b2) and np.array_equal(b1, b3)


def test_paper_buffers_as_frames():
    """Frames of 2^20 symbols = one 2^22-sample ADC buffer each (the
    paper's buffer), two buffers plus a ragged tail pushed whole: the bits
    equal the oracle's except near-threshold symbols."""
    F = 1 << 20
    n_sym = 2 * F + 5000
    d = case(2, n_sym, 73, 12.0, 7.0)
    cfg = chain_cfg(d, 2, F, acq=8192, block=1 << 22, hist=n_sym)
    n = d["codes"].size
    bits, y = run_chain(d, cfg, [1 << 22, 1 << 22, n - (2 << 22)])
    ref = oracle(d, cfg)
    compare(bits, y, ref, 2)


def test_short_streams():
    """A stream shorter than the acquisition, and one shorter than a
    block: every symbol is decided, as by the oracle."""
    for n_sym in (3000, 100):
        d = case(2, n_sym, 75, 12.0, 22.0)
        cfg = chain_cfg(d, 2, 1 << 12, acq=4096, hist=n_sym)
        bits, y = run_chain(d, cfg, [d["codes"].size])
        ref = oracle(d, cfg)
        compare(bits, y, ref, 2)


def test_reset_reproduces_the_stream():
    """A second stream on the same handle after rx_kkrx_reset gives the same
    bits as the first (every stage's positions, carries and taps restart)."""
    import torch
    F = 1 << 12
    d = case(4, 2 * F + 99, 77, 16.0, 14.0)
    cfg = chain_cfg(d, 4, F, acq=2048, mu=2e-3)
    codes = torch.from_numpy(d["codes"]).cuda()
    n = codes.numel()
    nbytes = (n // 4 * 4 + 7) // 8
    outs = []
    stream = torch.cuda.current_stream().cuda_stream
    with rx.KKReceiver(cfg) as r:
        for _ in range(2):
            bits = torch.zeros(nbytes + 64, dtype=torch.uint8, device="cuda")
            nb = 0
            for a in range(0, n, 7000):
                m = min(7000, n - a)
                nb += r.push_device(codes.data_ptr() + 2 * a, m, bits.data_ptr() + nb // 8, bits.numel() - nb // 8,
                                    stream)
            nb += r.end(bits.data_ptr() + nb // 8, bits.numel() - nb // 8, stream)
            torch.cuda.synchronize()
            outs.append((nb, bits.cpu().numpy()))
            r.reset()
    assert outs[0][0] == outs[1][0] == (n // 4) * 4
    assert np.array_equal(outs[0][1], outs[1][1])


def test_batch_push_equals_single_pushes():
    """Five receivers (different links, QPSK) pushed together, one front-end
    graph and one equaliser graph per round, uneven lengths per channel and
    round (including none), 4096-symbol frames completing at different
    rounds: bit for bit the bits of the same pushes one receiver at a time,
    the streams' ends included."""
    import torch
    F = 1 << 12
    rng = np.random.default_rng(91)
    links = [case(2, 3 * F + 200 * c, 90 + c, 12.0, 9.0) for c in range(5)]
    n = [d["codes"].size for d in links]
    dev = torch.device("cuda:0")
    codes = [torch.from_numpy(d["codes"]).to(dev) for d in links]
    nbytes = [(m // 4 * 2 + 7) // 8 + 64 for m in n]
    out = {k: [torch.zeros(nbytes[c], dtype=torch.uint8, device=dev) for c in range(5)] for k in ("batch", "single")}
    rxs = {k: [rx.KKReceiver(chain_cfg(d, 2, F, acq=2048, block=20000)) for d in links] for k in out}
    pos = [0] * 5
    nb = {k: [0] * 5 for k in out}
    stream = torch.cuda.current_stream().cuda_stream
    with rx.KKReceiverBatch(rxs["batch"]) as batch:
        for r in range(12):
            sizes = [int(min(n[c] - pos[c], rng.choice([0, 5, 700, 3000, 12000, 20000]))) for c in range(5)]
            got = batch.push([codes[c].data_ptr() + 2 * pos[c] for c in range(5)], sizes,
                             [out["batch"][c].data_ptr() + nb["batch"][c] // 8 for c in range(5)],
                             [nbytes[c] - nb["batch"][c] // 8 for c in range(5)], stream)
            for c in range(5):
                k = rxs["single"][c].push_device(codes[c].data_ptr() + 2 * pos[c], sizes[c],
                                                 out["single"][c].data_ptr() + nb["single"][c] // 8,
                                                 nbytes[c] - nb["single"][c] // 8, stream)
                assert got[c] == k
                nb["batch"][c] += got[c]
                nb["single"][c] += k
                pos[c] += sizes[c]
    for key in out:
        for c in range(5):
            r = rxs[key][c]
            if n[c] > pos[c]:
                nb[key][c] += r.push_device(codes[c].data_ptr() + 2 * pos[c], n[c] - pos[c],
                                            out[key][c].data_ptr() + nb[key][c] // 8, nbytes[c] - nb[key][c] // 8,
                                            stream)
            nb[key][c] += r.end(out[key][c].data_ptr() + nb[key][c] // 8, nbytes[c] - nb[key][c] // 8, stream)
            r.close()
    torch.cuda.synchronize()
    for c in range(5):
        assert nb["batch"][c] == nb["single"][c] == (n[c] // 4) * 2
        assert torch.equal(out["batch"][c], out["single"][c]), c
