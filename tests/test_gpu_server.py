"""Serving layer on the GPU: streams served together give exactly what each
gives alone (and what a plain receiver gives), admission by device memory,
latency statistics."""
import numpy as np
import pytest

import rxsim
from paper_2108_07001_gb300 import rx
from parity_util import compare, run_oracle

pytestmark = pytest.mark.gpu


def stream_case(kind, seed):
    """A short stream of one of three channel types and its receiver config."""
    F = 1 << 13
    if kind == "qpsk1000":
        link = dict(baud_hz=28e9, bits_per_sym=2, n_sym=4 * F + 999, fiber_len_m=1000e3, snr_db=12.0)
        cfg = dict(baud_hz=28e9, modulation=2, fiber_len_m=1000e3)
    elif kind == "qpsk2000":
        link = dict(baud_hz=32e9, bits_per_sym=2, n_sym=3 * F + 77, fiber_len_m=2000e3, snr_db=11.0)
        cfg = dict(baud_hz=32e9, modulation=2, fiber_len_m=2000e3)
    else:
        link = dict(baud_hz=32e9, bits_per_sym=4, n_sym=3 * F + 500, fiber_len_m=500e3, snr_db=18.0)
        cfg = dict(baud_hz=32e9, modulation=4, fiber_len_m=500e3, mimo_taps=25, bps_angles=32, bps_half_window=32,
                   mu_dd=2e-3)
    sim = rxsim.simulate(rxsim.LinkConfig(**link, prbs_seed=seed, seed=seed, out_dtype="c64"))
    n_sym = link["n_sym"]
    cfg.update(frame_syms=F, acq_syms=F, cma_syms=4096, prbs_seed=seed, ber_skip_syms=2048, sync_syms=2048,
               history_syms=n_sym, max_block_samples=1 << 15)
    x = sim["rx"]
    rng = np.random.default_rng(seed)
    cuts, left = [], x.shape[1]
    while left:
        m = int(min(left, rng.integers(1000, 1 << 15)))
        cuts.append(m)
        left -= m
    blocks, a = [], 0
    for m in cuts:
        blocks.append(np.ascontiguousarray(x[:, a:a + m]))
        a += m
    return cfg, blocks, n_sym


def submit(srv, sid, block, device):
    """A host block, or (device) a device copy kept alive by the caller."""
    if not device:
        srv.submit_host(sid, block)
        return None
    import torch
    t = torch.from_numpy(block).cuda()
    torch.cuda.synchronize()
    srv.submit_device(sid, t.data_ptr(), block.shape[1], rx.RX_C64)
    return t


def serve(cases, interleave=True, batch=0, device=False):
    """Runs the given streams through one server (batch = 1: batched rounds,
    device: blocks submitted from device memory); returns per-stream (bits,
    n_bits, y, stats, BPS angles/unwrap/trace) and the server statistics."""
    out = {}
    keep = []
    with rx.Server(max_streams=16, batch=batch) as srv:
        sids = {k: srv.open(**cfg) for k, (cfg, _, _) in cases.items()}
        queues = {k: list(blocks) for k, (_, blocks, _) in cases.items()}
        if interleave:
            while any(queues.values()):
                for k in cases:
                    if queues[k]:
                        keep.append(submit(srv, sids[k], queues[k].pop(0), device))
        else:
            for k in cases:
                for b in queues[k]:
                    keep.append(submit(srv, sids[k], b, device))
        for k in cases:
            srv.end(sids[k])
        for k in cases:
            srv.sync(sids[k], timeout_ms=120000)
        for k, (cfg, _, n_sym) in cases.items():
            bits, nb = srv.pull_bytes(sids[k])
            rcv = srv.receiver(sids[k])
            y = rcv.equalised(0, n_sym)
            bhat, m = rcv.phase(0, n_sym)
            out[k] = (bits, nb, y, srv.stream_stats(sids[k]), {"bhat": bhat, "m": m, "trace": rcv.frame_trace()})
        sst = srv.stats()
    return out, sst


CASES = ("qpsk1000", "qpsk2000", "qam16")


@pytest.fixture(scope="module")
def cases():
    return {k: stream_case(k, 700 + i) for i, k in enumerate(CASES)}


MODES = {"per_stream": dict(batch=0, device=False), "batched": dict(batch=1, device=True),
         "batched_graph": dict(batch=2, device=True)}


@pytest.fixture(scope="module", params=list(MODES))
def mode(request):
    return request.param


@pytest.fixture(scope="module")
def mixed(cases, mode):
    return serve(cases, interleave=True, **MODES[mode])


def test_each_stream_alone_equals_the_mix(cases, mixed, mode):
    """Bit for bit: decided bits, equalised symbols and counters of each
    stream served alone and served in the mix (per-stream pushes, and
    batched rounds where the mix shares every launch, launched on streams
    or replayed as a graph)."""
    mix, _ = mixed
    for k in CASES:
        alone, _ = serve({k: cases[k]}, **MODES[mode])
        b0, n0, y0, s0, _ = alone[k]
        b1, n1, y1, s1, _ = mix[k]
        assert n0 == n1 > 0
        assert np.array_equal(b0, b1), k
        assert np.array_equal(y0, y1), k
        for f in ("bits", "bit_errors", "cycle_slips", "synced", "frames"):
            assert s0[f] == s1[f], (k, f)


def test_served_stream_equals_a_plain_receiver(cases, mixed, mode):
    if mode != "per_stream":
        pytest.skip("batched rounds: compared with an rx_batch of the same blocks below")
    mix, _ = mixed
    k = "qpsk1000"
    cfg, blocks, n_sym = cases[k]
    r = rx.Receiver(**cfg)
    for b in blocks:
        r.push_host(b)
    r.end()
    buf = np.empty(1 << 22, dtype=np.uint8)
    nb = r.pull_bytes(buf, timeout_ms=-1)
    bits = buf[:(nb + 7) // 8]
    y = r.equalised(0, n_sym)
    st = r.stats()
    r.close()
    b1, n1, y1, s1, _ = mix[k]
    assert nb == n1
    assert np.array_equal(bits, b1)
    assert np.array_equal(y, y1)
    assert st["bit_errors"] == s1["bit_errors"] and st["bits"] == s1["bits"]


def test_batched_rounds_equal_a_batch_of_the_stream_alone(cases, mixed, mode):
    """A stream served in batched rounds gives bit for bit what its blocks
    pushed through an rx_batch of its own give (the same batched kernels)."""
    if not mode.startswith("batched"):
        pytest.skip("per-stream pushes: compared with a plain receiver above")
    import torch
    mix, sst = mixed
    assert sst["batch_calls"] > 0
    k = "qam16"
    cfg, blocks, n_sym = cases[k]
    r = rx.Receiver(**cfg)
    s = torch.cuda.current_stream().cuda_stream
    dev = [torch.from_numpy(b).cuda() for b in blocks]
    with rx.Batch([r], graph=mode == "batched_graph") as batch:
        for t in dev:
            batch.push([t.data_ptr()], [t.shape[1]], rx.RX_C64, s)
        batch.end(s)
    buf = np.empty(1 << 22, dtype=np.uint8)
    nb = r.pull_bytes(buf, timeout_ms=-1)
    y = r.equalised(0, n_sym)
    r.close()
    b1, n1, y1, s1, _ = mix[k]
    assert nb == n1 and np.array_equal(buf[:(nb + 7) // 8], b1)
    assert np.array_equal(y, y1)


def test_served_streams_match_the_oracle(cases, mixed):
    """Every stream served in the mix against the FP64 oracle on the same
    samples, under the parity rules of the single-stream tests (equalised
    symbols, BPS angles, bits, BER counters)."""
    mix, _ = mixed
    for k in CASES:
        cfg, blocks, n_sym = cases[k]
        ocfg = {key: v for key, v in cfg.items() if key != "history_syms"}
        ref = run_oracle(np.concatenate(blocks, axis=1), ocfg)
        bits, nb, y, st, ph = mix[k]
        rep = compare(dict(ph, y=y, bits=np.unpackbits(bits)[:nb]), ref, ocfg)
        assert st["bits"] == ref["ber"]["bits"] and st["cycle_slips"] == ref["ber"]["slips"], k
        assert abs(int(st["bit_errors"]) - ref["ber"]["errors"]) <= 2 * rep.get("bit_mismatch_syms", 0), k


def test_server_statistics(cases, mixed, mode):
    mix, sst = mixed
    assert (sst["batch_calls"] > 0) == mode.startswith("batched")
    n_blocks = sum(len(cases[k][1]) for k in CASES)
    assert sst["blocks_submitted"] == sst["blocks_pushed"] == n_blocks
    assert sst["blocks_queued"] == 0 and sst["worker_error"] == 0
    assert sst["samples_pushed"] == sum(2 * cases[k][2] for k in CASES)
    assert sst["frames_done"] == sum(mix[k][3]["frames"] for k in CASES)
    assert sst["latency_samples"] > 0
    assert 0 < sst["latency_p50_ms"] <= sst["latency_p99_ms"] <= sst["latency_max_ms"]
    for k in CASES:
        st = mix[k][3]
        assert st["synced"] == 1 and st["bits"] > 0 and st["ber"] < 1e-2


def test_streams_are_admitted_by_device_memory(cases):
    cfg = cases["qpsk1000"][0]
    with rx.Server(max_streams=8) as probe:
        probe.open(**cfg)
        one = probe.stats()["mem_in_use_bytes"]
    assert one > 0
    with rx.Server(max_streams=8, mem_budget_bytes=2 * one + one // 2) as srv:
        a = srv.open(**cfg)
        srv.open(**cfg)
        with pytest.raises(rx.RxError) as e:
            srv.open(**cfg)
        assert e.value.code == rx.RX_EAGAIN
        assert srv.stats()["streams_open"] == 2
        srv.close_stream(a)
        srv.open(**cfg)  # room again
        assert srv.stats()["mem_in_use_bytes"] == 2 * one


@pytest.mark.parametrize("batch", [1, 2], ids=["streams", "graph_replay"])
def test_batched_server_admits_and_retires_streams_continuously(cases, batch):
    """Batched rounds with streams opening and closing while others are on
    the GPU: a stream opened after the others have been running, and a
    stream closed (and its receiver freed) in the middle, each give what
    they give served alone (every change of membership builds a new batch,
    in graph replay a new graph)."""
    import torch
    keep = []
    got = {}
    with rx.Server(max_streams=16, batch=batch) as srv:
        a = srv.open(**cases["qpsk1000"][0])
        b = srv.open(**cases["qam16"][0])
        qa, qb = list(cases["qpsk1000"][1]), list(cases["qam16"][1])
        for _ in range(3):
            keep.append(submit(srv, a, qa.pop(0), True))
            keep.append(submit(srv, b, qb.pop(0), True))
        c = srv.open(**cases["qpsk2000"][0])  # joins while a and b are running
        qc = list(cases["qpsk2000"][1])
        while qb:
            keep.append(submit(srv, b, qb.pop(0), True))
            if qc:
                keep.append(submit(srv, c, qc.pop(0), True))
        srv.end(b)
        srv.sync(b, timeout_ms=120000)
        got["qam16"] = srv.pull_bytes(b)
        srv.close_stream(b)  # leaves while a and c keep going
        while qa or qc:
            if qa:
                keep.append(submit(srv, a, qa.pop(0), True))
            if qc:
                keep.append(submit(srv, c, qc.pop(0), True))
        for sid, k in ((a, "qpsk1000"), (c, "qpsk2000")):
            srv.end(sid)
            srv.sync(sid, timeout_ms=120000)
            got[k] = srv.pull_bytes(sid)
        assert srv.stats()["batch_calls"] > 0
    for k in ("qpsk1000", "qam16", "qpsk2000"):
        alone, _ = serve({k: cases[k]}, batch=batch, device=True)
        bits, nb = got[k]
        assert nb == alone[k][1] > 0, k
        assert np.array_equal(bits, alone[k][0]), k
