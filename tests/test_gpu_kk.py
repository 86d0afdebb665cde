"""GPU parity of the Kramers-Kronig front end (rx_kk_*) against the FP64
oracle on the same seeded ADC codes.

Tolerance: the field is computed in FP32 (log, two N-point FFTs, exp and
sincos of numbers of order 1), so each output carries a few units of
2^-24 times log2(N) in relative error: relative RMS error <= 1e-5 over the
stream and every sample within 1e-4 of the largest field magnitude."""
import math

import numpy as np
import pytest

import rxsim
from oracle import kk_oracle as K
from paper_2108_07001_gb300 import rx

pytestmark = pytest.mark.gpu

RMS_TOL = 1e-5
MAX_TOL = 1e-4


def link(n_sym, seed, **kw):
    d = rxsim.simulate_kk(rxsim.KKLinkConfig(n_sym=n_sym, seed=seed, prbs_seed=seed, fiber_len_m=100e3,
                                             cspr_db=10.0, snr_db=20.0, **kw))
    return d


def frontend(d, N, block=1 << 22):
    return rx.KKFrontEnd(fs_hz=d["fs"], f_shift_hz=d["f_c"], adc_gain=d["gain"], adc_offset=d["offset"],
                         fft_n=N, max_block_samples=block)


def expected_out(in_pos, N):
    L = N // 2
    q = in_pos - N // 4
    return q // L * L if q >= L else 0


def run_pushes(d, N, sizes, host_every=0):
    """Pushes the codes in the given sizes (every host_every-th from host
    memory); returns the whole field and the per-push output counts."""
    import torch
    codes = d["codes"]
    n = codes.size
    dev = torch.device("cuda:0")
    dc = torch.from_numpy(codes).to(dev)
    out = torch.zeros(n, dtype=torch.complex64, device=dev)
    counts = []
    with frontend(d, N, block=max(sizes)) as fe:
        a = pos = 0
        for i, m in enumerate(sizes):
            if host_every and i % host_every == 0:
                k = fe.push_host(codes[a:a + m], out[pos:].data_ptr(), n - pos,
                                 torch.cuda.current_stream().cuda_stream)
            else:
                k = fe.push_tensor(dc[a:a + m], out[pos:])
            a += m
            pos += k
            counts.append((a, pos, k))
        pos += fe.end_tensor(out[pos:])
        assert fe.position() == (n, n)
    torch.cuda.synchronize()
    assert pos == n
    return out.cpu().numpy(), counts


def check(got, want):
    err = np.abs(got - want)
    rms = float(np.linalg.norm(got - want) / np.linalg.norm(want))
    assert rms <= RMS_TOL, rms
    assert err.max() <= MAX_TOL * np.abs(want).max(), (err.max(), int(err.argmax()))
    return rms


@pytest.mark.parametrize("N", [1024, 2048, 4096])
def test_ragged_pushes_match_the_oracle(N):
    """Pushes from 1 sample to several blocks, mixing host and device memory,
    with a ragged tail: every push writes exactly the newly complete
    segments and the whole stream equals the oracle's field."""
    d = link(65536 + 333, seed=41)
    n = d["codes"].size
    rng = np.random.default_rng(N)
    sizes, left = [], n
    for m in [1, N // 8, N // 4 - 1, 3, N, 7 * N + 5]:
        sizes.append(m)
        left -= m
    while left:
        m = int(min(left, rng.integers(1, 40000)))
        sizes.append(m)
        left -= m
    got, counts = run_pushes(d, N, sizes, host_every=3)
    prev = 0
    for a, pos, k in counts:
        assert pos == expected_out(a, N) and k == pos - prev
        prev = pos
    want = K.kk_field(d["codes"], d["gain"], d["offset"], N, d["f_c"] / d["fs"])
    check(got, want)


def test_host_pushes_equal_device_pushes():
    d = link(1 << 14, seed=43)
    sizes = [5000] * (d["codes"].size // 5000) + [d["codes"].size % 5000]
    a, _ = run_pushes(d, 1024, sizes, host_every=0)
    b, _ = run_pushes(d, 1024, sizes, host_every=1)
    assert np.array_equal(a, b)


def test_paper_buffers_sampled_segments():
    """The paper's geometry: 2^22-sample buffers of 12-bit codes at 4 GS/s
    (1 GBd, 4 samples per symbol), 1024-point blocks; three buffers in
    whole pushes.  Segments spread over the stream (the last ones at
    t ~ 1.2e7, where the downshift phase has turned 1.6e6 times) are checked
    against the oracle run on each segment's block alone."""
    import torch
    N, L = 1024, 512
    buf = 1 << 22
    d = link(3 * buf // 4, seed=47)
    codes = d["codes"]
    n = codes.size
    dev = torch.device("cuda:0")
    dc = torch.from_numpy(codes).to(dev)
    out = torch.zeros(n, dtype=torch.complex64, device=dev)
    pos = 0
    with frontend(d, N, block=buf) as fe:
        for b in range(3):
            pos += fe.push_tensor(dc[b * buf:(b + 1) * buf], out[pos:])
        pos += fe.end_tensor(out[pos:])
    torch.cuda.synchronize()
    assert pos == n
    got = out.cpu().numpy()
    I = K.adc_to_intensity(codes, d["gain"], d["offset"])
    nu = d["f_c"] / d["fs"]
    rng = np.random.default_rng(5)
    segs = sorted(set([0, 1, n // L - 1] + [int(s) for s in rng.integers(0, n // L, 40)]))
    for b in segs:
        w0 = max(b - 1, 0) * L
        w1 = min(w0 + 3 * L, n)
        field = K.kk_field_from_intensity(I[w0:w1], 0.5 * d["gain"], N, nu, t0=w0)
        r = b * L - w0
        check(got[b * L:(b + 1) * L], field[r:r + L])


def test_edge_cases():
    import torch
    d = link(4096, seed=49)
    codes = torch.from_numpy(d["codes"]).cuda()
    out = torch.zeros(codes.numel(), dtype=torch.complex64, device="cuda")
    with frontend(d, 1024, block=1 << 16) as fe:
        assert fe.push_tensor(codes[:0], out) == 0          # empty push
        assert fe.push_tensor(codes[:200], out) == 0        # less than a quarter block
        with pytest.raises(rx.RxError):
            fe.push_tensor(codes[200:1000], out[:10])       # out too small for the completed segment
        assert fe.position() == (200, 0)                    # a refused push changes nothing
        assert fe.end_tensor(out) == 200                    # end: the short stream is output whole
        with pytest.raises(rx.RxError) as e:
            fe.push_tensor(codes[:10], out)
        assert e.value.code == rx.RX_ESTATE
        first = out[:200].cpu().numpy()
        fe.reset()                                          # a new stream on the same handle
        assert fe.push_tensor(codes[:200], out) == 0
        assert fe.end_tensor(out) == 200
        assert np.array_equal(out[:200].cpu().numpy(), first)
    want = K.kk_field(d["codes"][:200], d["gain"], d["offset"], 1024, d["f_c"] / d["fs"])
    check(first, want)


def test_batch_push_equals_single_pushes():
    """Six channels (different links) pushed together through one graph
    replay per round, with uneven lengths per channel and round (empty,
    below a quarter block, several blocks), give bit for bit the field of
    the same pushes one channel at a time; the streams then end alike."""
    import torch
    rng = np.random.default_rng(77)
    links = [link(4096 + 500 * c, seed=80 + c) for c in range(6)]
    n = [d["codes"].size for d in links]
    dev = torch.device("cuda:0")
    codes = [torch.from_numpy(d["codes"]).to(dev) for d in links]
    outs = {k: [torch.zeros(m, dtype=torch.complex64, device=dev) for m in n] for k in ("batch", "single")}
    fes = {k: [frontend(d, 1024, block=20000) for d in links] for k in ("batch", "single")}
    pos_in = [0] * 6
    pos_out = {k: [0] * 6 for k in outs}
    stream = torch.cuda.current_stream().cuda_stream
    with rx.KKBatch(fes["batch"]) as batch:
        for r in range(8):
            sizes = [int(min(n[c] - pos_in[c], rng.choice([0, 3, 200, 1500, 9000, 20000]))) for c in range(6)]
            got = batch.push([codes[c][pos_in[c]:].data_ptr() for c in range(6)], sizes,
                             [outs["batch"][c][pos_out["batch"][c]:].data_ptr() for c in range(6)],
                             [n[c] - pos_out["batch"][c] for c in range(6)], stream)
            for c in range(6):
                k = fes["single"][c].push_tensor(codes[c][pos_in[c]:pos_in[c] + sizes[c]],
                                                 outs["single"][c][pos_out["single"][c]:])
                assert got[c] == k
                pos_out["batch"][c] += got[c]
                pos_out["single"][c] += k
                pos_in[c] += sizes[c]
    for key in outs:
        for c in range(6):
            fe = fes[key][c]
            rest = torch.from_numpy(links[c]["codes"][pos_in[c]:]).to(dev)
            p = pos_out[key][c]
            p += fe.push_tensor(rest, outs[key][c][p:]) if rest.numel() else 0
            p += fe.end_tensor(outs[key][c][p:])
            assert p == n[c]
            fe.close()
    torch.cuda.synchronize()
    for c in range(6):
        a, b = outs["batch"][c].cpu().numpy(), outs["single"][c].cpu().numpy()
        assert np.array_equal(a, b), c
    want = K.kk_field(links[0]["codes"], links[0]["gain"], links[0]["offset"], 1024,
                      links[0]["f_c"] / links[0]["fs"])
    check(outs["batch"][0].cpu().numpy(), want)
