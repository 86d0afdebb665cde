"""Helpers shared by the GPU parity tests: run the CUDA receiver through the
C ABI and the FP64 oracle on the same seeded samples, then compare.

Tolerances (stated where used):
  equalised symbols  rel RMS <= 1e-4 (FP32 path vs FP64 oracle) over the
                     record, over every frame and over every overlap-save
                     block's worth of symbols;
  BPS angle          the GPU's angle is the oracle's, or a near-tie of it:
                     D_or[b_gpu] - min_b D_or <= 1e-4 * min_b D_or;
                     two-stage search: the GPU's index is the refinement of a
                     coarse angle that is a near-tie in the same sense, with
                     floor(S delta + 1/2) taken anywhere within
                     S delta +- 3 S 1e-4 max(D-, D0, D+) / c (the change of
                     S delta when each cost moves by up to 1e-4 of itself);
  unwrapped phase    equal wherever the angles are equal;
  bits               identical except for symbols whose oracle-corrected value
                     lies within 1e-3 of a decision threshold or whose BPS
                     angle is a near-tie.
"""
from __future__ import annotations

import math

import numpy as np

import rxsim
from oracle import rx_oracle as O

Y_TOL = 1e-4
BOUNDARY = 1e-3
TIE = 1e-4


def run_gpu(samples: np.ndarray, rx_kw: dict, pushes=None, dtype=None, history=True):
    """Push samples (host array [2, n] complex or [2, n, 2] float16) in the given
    block sizes from device memory; returns results and the receiver."""
    import torch
    from paper_2108_07001_gb300 import rx

    n = samples.shape[1]
    n_sym = n // 2
    kw = dict(rx_kw)
    if history:
        kw["history_syms"] = n_sym
    pushes = pushes or [n]
    kw.setdefault("max_block_samples", max(max(pushes), 1))
    r = rx.Receiver(**kw)
    dev = torch.from_numpy(np.ascontiguousarray(samples)).to("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    pos = 0
    bits = []
    for m in pushes:
        blk = dev[:, pos:pos + m].contiguous()
        r.push_tensor(blk, stream)
        pos += m
        bits.append(r.pull_bits(1 << 22, timeout_ms=0))
    assert pos == n
    r.end()
    bits.append(r.pull_bits(1 << 24, timeout_ms=-1))
    torch.cuda.synchronize()
    out = {"bits": np.concatenate(bits), "stats": r.stats(), "trace": r.frame_trace()}
    if history:
        out["y"] = r.equalised(0, n_sym)
        out["bhat"], out["m"] = r.phase(0, n_sym)
    return out, r


def run_oracle(samples: np.ndarray, rx_kw: dict):
    if samples.dtype == np.float16:
        x = samples[..., 0].astype(np.float64) + 1j * samples[..., 1].astype(np.float64)
    else:
        x = samples.astype(np.complex128)
    return O.Receiver(O.RxConfig(**_oracle_kw(rx_kw))).run(x)


def rel_rms(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oracle_bps_metric(y: np.ndarray, k: np.ndarray, B: int, W: int, bits_per_sym: int) -> np.ndarray:
    """D_{k,b} of the oracle's definition for the listed symbols k."""
    n = y.size
    phi = O.bps_angles(B)
    out = np.zeros((k.size, B))
    for i in range(-W, W + 1):
        kk = k + i
        ok = (kk >= 0) & (kk < n)
        z = y[np.clip(kk, 0, n - 1)][:, None] * np.exp(-1j * phi)[None, :]
        d = np.abs(z - O.decide(z, bits_per_sym)) ** 2
        out += np.where(ok[:, None], d, 0.0)
    return out


def two_stage_valid(y: np.ndarray, k: np.ndarray, b_gpu: np.ndarray, B: int, W: int, bits_per_sym: int,
                    S: int) -> np.ndarray:
    """Whether each GPU index b_gpu[i] of symbol k[i] is a valid two-stage
    result under the oracle's own costs (see the module docstring)."""
    C = B // S
    phi = O.bps_angles(B)[::S]
    ok = np.zeros(k.size, dtype=bool)
    for i, kk in enumerate(k):
        Dc = O.bps_costs(y, phi, W, bits_per_sym, int(kk), int(kk) + 1)[0]
        dmin = Dc.min()
        for j in np.nonzero(Dc - dmin <= TIE * dmin)[0]:
            Dm, D0, Dp = Dc[(j - 1) % C], Dc[j], Dc[(j + 1) % C]
            c = Dm - 2.0 * D0 + Dp
            if c > 0:
                x = S * float(np.clip((Dm - Dp) / (2.0 * c), -0.5, 0.5))
                tol = 3.0 * S * TIE * max(Dm, D0, Dp) / c
            else:
                x, tol = 0.0, 0.0
            for r in range(int(math.floor(x - tol + 0.5)), int(math.floor(x + tol + 0.5)) + 1):
                r = min(max(r, -(S // 2)), S // 2)
                if (S * j + r) % B == b_gpu[i]:
                    ok[i] = True
    return ok


def _oracle_kw(rx_kw: dict) -> dict:
    from paper_2108_07001_gb300.workloads import oracle_kwargs
    kw = oracle_kwargs(rx_kw)
    for k in ("history_syms", "profile", "device"):
        kw.pop(k, None)
    return kw


def check_equalised(y_gpu: np.ndarray, y_ref: np.ndarray, frame_syms: int, block_syms: int) -> dict:
    """Equalised symbols [2, n]: relative RMS <= Y_TOL over the whole record,
    over every frame, and over every piece of block_syms symbols (one
    overlap-save block's kept outputs; pieces start at each frame start), so
    an error confined to one block cannot hide in the norm of a long record."""
    n = y_ref.shape[1]
    glob = rel_rms(y_gpu, y_ref)
    per_frame = [rel_rms(y_gpu[:, a:a + frame_syms], y_ref[:, a:a + frame_syms]) for a in range(0, n, frame_syms)]
    worst_block, worst_at = 0.0, 0
    for f0 in range(0, n, frame_syms):
        f1 = min(f0 + frame_syms, n)
        for a in range(f0, f1, block_syms):
            b = min(a + block_syms, f1)
            den = np.linalg.norm(y_ref[:, a:b])
            e = float(np.linalg.norm(y_gpu[:, a:b] - y_ref[:, a:b]) / den) if den > 0 else 0.0
            if e > worst_block:
                worst_block, worst_at = e, a
    if glob > Y_TOL or max(per_frame) > Y_TOL or worst_block > Y_TOL:
        worst = np.argsort(-np.abs(y_gpu - y_ref).max(axis=0))[:8]
        raise AssertionError(f"equalised symbols: rel RMS {glob:.3e}, per frame {np.round(per_frame, 7).tolist()}, "
                             f"worst {block_syms}-symbol block {worst_block:.3e} at symbol {worst_at} "
                             f"(bound {Y_TOL}); worst symbols {worst.tolist()}")
    return {"y_rel_rms": glob, "y_rel_rms_frame_max": max(per_frame), "y_rel_rms_block_max": worst_block}


def compare(gpu: dict, ref: dict, rx_kw: dict, check_bits=True) -> dict:
    """All parity checks; returns a report (asserts on failure)."""
    B = rx_kw.get("bps_angles", 64)
    W = rx_kw.get("bps_half_window", 16)
    bps = rx_kw.get("modulation", 2)
    S = rx_kw.get("bps_coarse_stride", 1)
    rep = {}
    F = rx_kw.get("frame_syms", 1 << 16)
    g = O.geometry(O.RxConfig(**_oracle_kw(rx_kw)))
    try:
        rep.update(check_equalised(gpu["y"], ref["y"], F, max(g.L // 2, 1)))
    except AssertionError as e:
        tr = gpu.get("trace")
        raise AssertionError(f"{e}; gpu trace {None if tr is None else tr.tolist()}; oracle tau "
                             f"{ref['trace']['tau']} dfo {ref['trace']['dfo']} gain {ref['trace']['gain']}")

    # BPS angles: equal, or a near-tie under the oracle's own metric
    bh_g = gpu["bhat"].astype(np.int64)
    bh_o = ref["bhat"]
    tie = np.zeros_like(bh_o, dtype=bool)
    for p in range(2):
        diff = np.nonzero(bh_g[p] != bh_o[p])[0]
        if diff.size and S > 1:
            ok = two_stage_valid(ref["y"][p], diff, bh_g[p][diff], B, W, bps, S)
            assert ok.all(), f"pol {p}: {np.sum(~ok)} two-stage BPS indices are not near-ties"
            tie[p, diff] = True
        elif diff.size:
            D = oracle_bps_metric(ref["y"][p], diff, B, W, bps)
            dmin = D.min(axis=1)
            dg = D[np.arange(diff.size), bh_g[p][diff]]
            ok = dg - dmin <= TIE * dmin
            assert ok.all(), f"pol {p}: {np.sum(~ok)} BPS angles are not near-ties"
            tie[p, diff] = True
    rep["bps_ties"] = int(tie.sum())
    # unwrap counters: m_gpu - m_oracle may change only at a near-tie symbol or
    # the one after it (a tie can move the unwrap branch by a multiple of pi/2;
    # both branches are valid outputs); elsewhere the phases are identical.
    delta = gpu["m"].astype(np.int64) - ref["m"]
    for p in range(2):
        jumps = np.nonzero(np.diff(delta[p]))[0] + 1
        ok = tie[p, jumps] | tie[p, jumps - 1]
        assert ok.all(), f"pol {p}: unwrap branch changes at {jumps[~ok][:5]} without a near-tie"
    phi = O.bps_angles(B)
    ph_g = phi[bh_g] + (gpu["m"] - delta) * (math.pi / 2)
    ph_o = phi[bh_o] + ref["m"] * (math.pi / 2)
    assert np.all(np.abs(ph_g - ph_o)[~tie] < 1e-9), "phases differ where the BPS angles agree"
    rep["branch_shift_syms"] = int(np.count_nonzero(delta))

    if check_bits:
        # bits: symbol-major, pol x then y, I bits then Q bits; the oracle's
        # decisions are moved to the GPU's unwrap branch ((-j)^delta) first
        n_sym = ref["y"].shape[1]
        nl = 2 if bps == 2 else 4
        lb = O.level_bits(bps)
        gb = gpu["bits"][:n_sym * 2 * bps].reshape(n_sym, 2, bps)
        ob = np.zeros_like(gb)
        for p in range(2):
            lI, lQ = ref["levels"][p][0].copy(), ref["levels"][p][1].copy()
            q = np.mod(delta[p], 4)
            for _ in range(3):
                rot = q > 0
                lI[rot], lQ[rot] = lQ[rot], nl - 1 - lI[rot]
                q = np.where(rot, q - 1, q)
            ob[:, p, :] = np.concatenate([lb[lI], lb[lQ]], axis=1)
        mism = np.any(gb != ob, axis=2)  # [n, 2]
        lv = O.levels(bps)
        thr = 0.5 * (lv[1:] + lv[:-1])
        zc = ref["zc"].T  # [n, 2]
        near = np.zeros_like(mism)
        for t in thr:
            near |= (np.abs(zc.real - t) < BOUNDARY) | (np.abs(zc.imag - t) < BOUNDARY)
        explained = near | tie.T
        bad = mism & ~explained
        rep["bit_mismatch_syms"] = int(mism.sum())
        assert not bad.any(), f"{int(bad.sum())} decisions differ without a near-boundary or near-tie reason"
    return rep
