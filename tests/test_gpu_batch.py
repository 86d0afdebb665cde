"""Batched pushes of many dual-polarisation streams (rx_batch_*): one
launch per stage and frame ordinal over every stream's frames gives what
the same blocks pushed stream by stream give.

The batched kernels inline the same stage bodies into other kernels, and
the compiler may fuse a different multiply into an FMA there, so soft
values agree to FP32 rounding rather than bit for bit: both paths are
deterministic, and 1-ulp differences in the CD output show up downstream as
differences of order 1e-6 of the unit-power symbols (bound used: 1e-4,
room for the adaptive equaliser to carry them over a few frames).  A
decision within rounding of a threshold (or a BPS near-tie) can then come
out differently, so the bits of both runs are held to the oracle parity
rules on the same samples (identical except near a threshold or at a
near-tie); frame, sync and slip counters must be equal."""
import numpy as np
import pytest

import rxsim
from paper_2108_07001_gb300 import rx
from parity_util import compare, run_oracle

pytestmark = pytest.mark.gpu

F = 1 << 13


def stream_case(kind, seed):
    """A short stream and its receiver configuration; the kinds differ in
    FFT size, tap count, BPS form, modulation, storage type and launch
    tiles, so the batch runs several launch groups per stage."""
    if kind == "qpsk1000":
        link = dict(baud_hz=28e9, bits_per_sym=2, n_sym=4 * F + 999, fiber_len_m=1000e3, snr_db=12.0)
        cfg = dict(baud_hz=28e9, modulation=2, fiber_len_m=1000e3)
    elif kind == "qpsk3000_fft8192":
        link = dict(baud_hz=32e9, bits_per_sym=2, n_sym=3 * F + 77, fiber_len_m=3000e3, snr_db=11.0)
        cfg = dict(baud_hz=32e9, modulation=2, fiber_len_m=3000e3, fft_n=8192, mimo_block_warps=2, bps_block_runs=4)
    elif kind == "qpsk64_fft32768":
        link = dict(baud_hz=64e9, bits_per_sym=2, n_sym=3 * F + 1000, fiber_len_m=4000e3, snr_db=13.0)
        cfg = dict(baud_hz=64e9, modulation=2, fiber_len_m=4000e3, fft_n=32768)
    elif kind == "qpsk_two_stage_fp16":
        link = dict(baud_hz=28e9, bits_per_sym=2, n_sym=5 * F, fiber_len_m=1500e3, snr_db=12.0)
        cfg = dict(baud_hz=28e9, modulation=2, fiber_len_m=1500e3, bps_coarse_stride=4,
                   storage_dtype=rx.RX_C16)
    else:
        link = dict(baud_hz=32e9, bits_per_sym=4, n_sym=3 * F + 500, fiber_len_m=500e3, snr_db=18.0)
        cfg = dict(baud_hz=32e9, modulation=4, fiber_len_m=500e3, mimo_taps=25, bps_angles=32, bps_half_window=32,
                   mu_dd=2e-3, mimo_block_warps=8)
    sim = rxsim.simulate(rxsim.LinkConfig(**link, prbs_seed=seed, seed=seed, out_dtype="c64"))
    n_sym = link["n_sym"]
    cfg.update(frame_syms=F, acq_syms=F, cma_syms=4096, prbs_seed=seed, ber_skip_syms=2048, sync_syms=2048,
               history_syms=n_sym, max_block_samples=1 << 15)
    x = sim["rx"]
    rng = np.random.default_rng(seed)
    cuts, left = [], x.shape[1]
    while left:
        m = int(min(left, rng.choice([0, 1000, 5000, 1 << 14, 1 << 15, int(rng.integers(1, 1 << 15))])))
        cuts.append(m)
        left -= m
    blocks, a = [], 0
    for m in cuts:
        blocks.append(np.ascontiguousarray(x[:, a:a + m]))
        a += m
    return cfg, blocks, n_sym


KINDS = ("qpsk1000", "qpsk3000_fft8192", "qpsk_two_stage_fp16", "qam16", "qpsk64_fft32768")


@pytest.fixture(scope="module")
def cases():
    return [stream_case(k, 900 + i) for i, k in enumerate(KINDS)]


def results(r, n_sym):
    buf = np.empty(1 << 22, dtype=np.uint8)
    nb = r.pull_bytes(buf, timeout_ms=-1)
    bhat, m = r.phase(0, n_sym)
    return buf[:(nb + 7) // 8].copy(), nb, r.equalised(0, n_sym), r.stats(), \
        {"bhat": bhat, "m": m, "trace": r.frame_trace()}


def oracle_input(x, cfg):
    """The samples as the receiver stores them (FP16 storage: rounded to
    half precision, as the parity tests feed the oracle)."""
    if cfg.get("storage_dtype") == rx.RX_C16:
        return np.stack([x.real, x.imag], axis=-1).astype(np.float16)
    return x


def plain(cases):
    import torch
    out = []
    s = torch.cuda.current_stream().cuda_stream
    for cfg, blocks, n_sym in cases:
        r = rx.Receiver(**cfg)
        for b in blocks:
            if b.shape[1]:
                t = torch.from_numpy(b).cuda()
                r.push_device(t.data_ptr(), b.shape[1], rx.RX_C64, s)
                torch.cuda.current_stream().synchronize()
        r.end()
        out.append(results(r, n_sym))
        r.close()
    return out


@pytest.mark.parametrize("graph", [False, True], ids=["streams", "graph_replay"])
def test_batch_equals_plain_pushes(cases, graph):
    """Uneven rounds (some streams idle in a round), one stream's block of
    round 2 pushed through its own call in the middle of the batch's
    rounds, one stream ended through its own call, the others by the
    batch: bits, equalised symbols and counters equal the plain pushes',
    with the stages launched on the batch's streams or replayed as one
    captured graph per call."""
    import torch
    want = plain(cases)
    s = torch.cuda.current_stream().cuda_stream
    recs = [rx.Receiver(**cfg) for cfg, _, _ in cases]
    dev = [[torch.from_numpy(b).cuda() for b in blocks] for _, blocks, _ in cases]
    dummy = torch.zeros(16, dtype=torch.complex64, device="cuda")  # a non-null pointer for "nothing"
    n_rounds = max(len(b) for b in dev)
    with rx.Batch(recs, graph=graph) as batch:
        for j in range(n_rounds):
            ptrs, ns = [], []
            for c, blocks in enumerate(dev):
                if j < len(blocks) and blocks[j].shape[1] and not (c == 1 and j == 2):
                    ptrs.append(blocks[j].data_ptr())
                    ns.append(blocks[j].shape[1])
                else:
                    ptrs.append(dummy.data_ptr())
                    ns.append(0)
            if n_rounds > 2 and j == 2 and len(dev[1]) > 2 and dev[1][2].shape[1]:
                recs[1].push_device(dev[1][2].data_ptr(), dev[1][2].shape[1], rx.RX_C64, s)
            batch.push(ptrs, ns, rx.RX_C64, s)
        recs[0].end()
        with pytest.raises(rx.RxError) as e:  # stream 0 has ended: the whole call is refused
            batch.end(s)
        assert e.value.code == rx.RX_ESTATE
        ptrs = [dummy.data_ptr()] + [None] * (len(recs) - 1)
        batch.push(ptrs, [0] * len(recs), rx.RX_C64, s)
        info = batch.info()
        ginfo = batch.graph_info()
    got = [results(r, n_sym) for r, (_, _, n_sym) in zip(recs, cases)]
    for r in recs:
        r.close()
    frames = 0
    for k, (a, b) in enumerate(zip(want, got)):
        bits0, n0, y0, s0, _ = a
        bits1, n1, y1, s1, _ = b
        assert n0 == n1 > 0, KINDS[k]
        assert np.abs(y0 - y1).max() <= 1e-4, KINDS[k]
        for f in ("bits", "cycle_slips", "synced", "frames", "sync_delay", "sync_perm"):
            assert s0[f] == s1[f], (KINDS[k], f)
        nd = int(np.count_nonzero(np.unpackbits(bits0) != np.unpackbits(bits1)))
        assert abs(s0["bit_errors"] - s1["bit_errors"]) <= nd, KINDS[k]
        assert s1["synced"] == 1 and s1["ber"] < 1e-2, KINDS[k]
        assert s1["evm"] == pytest.approx(s0["evm"], rel=1e-4)
        frames += s1["frames"]
        # both runs against the FP64 oracle on the same samples (FP16 storage:
        # the half-precision samples): equalised symbols, BPS angles, bits
        # and BER counters under the single-stream parity rules
        cfg, blocks, n_sym = cases[k]
        ocfg = {key: v for key, v in cfg.items() if key != "history_syms"}
        ref = run_oracle(oracle_input(np.concatenate(blocks, axis=1), cfg), ocfg)
        for bits, nb, y, st, ph in (a, b):
            rep = compare(dict(ph, y=y, bits=np.unpackbits(bits)[:nb]), ref, ocfg)
            assert st["bits"] == ref["ber"]["bits"] and st["cycle_slips"] == ref["ber"]["slips"], KINDS[k]
            assert abs(int(st["bit_errors"]) - ref["ber"]["errors"]) <= 2 * rep.get("bit_mismatch_syms", 0)
    assert 0 < info["frames"] <= frames
    assert info["calls"] == n_rounds + 1
    assert info["launches"] > 0
    if graph:
        assert ginfo["nodes"] > 0 and 0 < ginfo["replays"] <= info["calls"]
    else:
        assert ginfo == {"replays": 0, "nodes": 0}


def test_graph_mode_is_set_before_the_first_push(cases):
    """rx_batch_set_graph is refused once the batch has pushed, and a graph
    batch can be switched back to the stream mode before it pushes."""
    import torch
    cfg, blocks, _ = cases[0]
    r = rx.Receiver(**cfg)
    lib = rx.load()
    with rx.Batch([r], graph=True) as batch:
        assert batch.graph_info()["nodes"] > 0
        assert lib.rx_batch_set_graph(batch.b, 0) == rx.RX_OK
        assert batch.graph_info()["nodes"] == 0
        assert lib.rx_batch_set_graph(batch.b, 1) == rx.RX_OK
        t = torch.from_numpy(blocks[0]).cuda() if blocks[0].shape[1] else torch.zeros((2, 1), dtype=torch.complex64,
                                                                                      device="cuda")
        batch.push([t.data_ptr()], [t.shape[1]], rx.RX_C64, torch.cuda.current_stream().cuda_stream)
        assert lib.rx_batch_set_graph(batch.b, 0) == rx.RX_ESTATE
        assert lib.rx_batch_set_graph(batch.b, 1) == rx.RX_ESTATE
        torch.cuda.synchronize()
    r.close()


def test_refused_batch_push_changes_nothing(cases):
    import torch
    cfg, blocks, _ = cases[0]
    s = torch.cuda.current_stream().cuda_stream
    r0, r1 = rx.Receiver(**cfg), rx.Receiver(**cfg)
    t = torch.from_numpy(next(b for b in blocks if b.shape[1])).cuda()
    big = torch.zeros((2, (1 << 15) + 1), dtype=torch.complex64, device="cuda")
    with rx.Batch([r0, r1]) as batch:
        with pytest.raises(rx.RxError) as e:  # stream 1's block exceeds max_block_samples
            batch.push([t.data_ptr(), big.data_ptr()], [t.shape[1], big.shape[1]], rx.RX_C64, s)
        assert e.value.code == rx.RX_EINVAL
        assert batch.info()["calls"] == 0
        with pytest.raises(rx.RxError):
            batch.push([t.data_ptr(), t.data_ptr()], [t.shape[1], t.shape[1]], rx.RX_C64, s, on_device=0)
        batch.push([t.data_ptr(), t.data_ptr()], [t.shape[1], t.shape[1]], rx.RX_C64, s)
        batch.end(s)
    a, b = results(r0, 1000), results(r1, 1000)
    assert a[1] == b[1] and np.array_equal(a[0], b[0])
    r0.close()
    r1.close()


def test_batch_from_page_locked_host_memory_equals_device_memory(cases):
    """Blocks in page-locked host memory, read by the batched ingest
    through the device mapping (on_device = 2), give bit for bit what the
    same blocks in device memory give (the same batched kernels)."""
    import torch
    s = torch.cuda.current_stream().cuda_stream
    sel = [cases[0], cases[2]]
    out = []
    for mode in ("device", "pinned"):
        recs = [rx.Receiver(**cfg) for cfg, _, _ in sel]
        keep = [[torch.from_numpy(b).cuda() if mode == "device" else torch.from_numpy(b).pin_memory()
                 for b in blocks if b.shape[1]] for _, blocks, _ in sel]
        dummy = keep[0][0]
        with rx.Batch(recs) as batch:
            for j in range(max(len(k) for k in keep)):
                ptrs = [k[j].data_ptr() if j < len(k) else dummy.data_ptr() for k in keep]
                ns = [k[j].shape[1] if j < len(k) else 0 for k in keep]
                batch.push(ptrs, ns, rx.RX_C64, s, on_device=1 if mode == "device" else 2)
            batch.end(s)
        out.append([results(r, n_sym)[:3] for r, (_, _, n_sym) in zip(recs, sel)])
        for r in recs:
            r.close()
    for (b0, n0, y0), (b1, n1, y1) in zip(out[0], out[1]):
        assert n0 == n1 > 0
        assert np.array_equal(b0, b1)
        assert np.array_equal(y0, y1)


def test_plain_pushes_after_the_batch_is_destroyed(cases):
    """Streams pushed through a batch, then (after rx_batch_destroy) through
    their own calls, give what plain pushes throughout give: the plain path
    no longer refers to the batch's streams."""
    import torch
    s = torch.cuda.current_stream().cuda_stream
    sel = [cases[0], cases[3]]
    want = plain(sel)
    recs = [rx.Receiver(**cfg) for cfg, _, _ in sel]
    dev = [[torch.from_numpy(b).cuda() for b in blocks if b.shape[1]] for _, blocks, _ in sel]
    with rx.Batch(recs) as batch:
        batch.push([d[0].data_ptr() for d in dev], [d[0].shape[1] for d in dev], rx.RX_C64, s)
    for r, d in zip(recs, dev):  # the batch is gone
        for t in d[1:]:
            r.push_device(t.data_ptr(), t.shape[1], rx.RX_C64, s)
        r.end()
    got = [results(r, n_sym) for r, (_, _, n_sym) in zip(recs, sel)]
    for r in recs:
        r.close()
    for (cfg, blocks, n_sym), a, b in zip(sel, want, got):
        (b0, n0, y0, s0, _), (b1, n1, y1, s1, ph1) = a, b
        assert n0 == n1 > 0
        assert np.abs(y0 - y1).max() <= 1e-4
        for f in ("frames", "synced", "cycle_slips"):
            assert s0[f] == s1[f], f
        # decided bits: equal, or a difference explained under the oracle's rules
        if not np.array_equal(b0, b1):
            ocfg = {key: v for key, v in cfg.items() if key != "history_syms"}
            ref = run_oracle(oracle_input(np.concatenate(blocks, axis=1), cfg), ocfg)
            compare(dict(ph1, y=y1, bits=np.unpackbits(b1)[:n1]), ref, ocfg)
