// Host runtime behind the C ABI in include/rx.h: configuration checks,
// FP64 set-up of the CD filter and FFT twiddles, device allocation, the
// push ring, frame scheduling on the library's compute stream, bit pulls
// and statistics.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <string>
#include <thread>
#include <vector>

#include "../../include/rx.h"
#include "rx_handle.h"

using namespace rx;

namespace {

thread_local std::string g_err;

}  // namespace

namespace rxrt {

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return RX_EDEVICE;
}

}  // namespace rxrt

using namespace rxrt;

namespace rxrt {

int log2i(long long v) {
  int r = 0;
  while ((1LL << r) < v) ++r;
  return r;
}

cudaEvent_t get_event(rx_handle* h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// GF(2) 31x31 matrices as 31 column words.
void gf2_mul(const uint32_t* A, const uint32_t* B, uint32_t* C) {  // C = A B
  for (int j = 0; j < 31; ++j) {
    uint32_t col = 0;
    for (int k = 0; k < 31; ++k)
      if ((B[j] >> k) & 1u) col ^= A[k];
    C[j] = col;
  }
}

uint32_t prbs_state(uint64_t seed, int pol) {
  const uint64_t p = (1ULL << 31) - 1;
  const uint64_t off = pol == 0 ? 0 : 0x2545F491ULL;
  const uint64_t v = (seed % p + off) % p;
  return (uint32_t)((v * 1103515245ULL) % p + 1);
}

double rrc_amp(double f, double Rs, double rho) {
  const double a = std::fabs(f) / Rs;
  if (a <= (1 - rho) / 2) return 1.0;
  if (rho <= 0 || a > (1 + rho) / 2) return 0.0;
  return std::sqrt(0.5 * (1.0 + std::cos(M_PI / rho * (a - (1 - rho) / 2))));
}

double erfcinv_host(double y) {  // solve erfc(x) = y, 0 < y < 1, Newton from a rational start
  double x = std::sqrt(-std::log(y / 2.0 + 1e-300));
  for (int i = 0; i < 60; ++i) {
    const double fx = std::erfc(x) - y;
    const double dfx = -2.0 / std::sqrt(M_PI) * std::exp(-x * x);
    const double nx = x - fx / dfx;
    if (std::fabs(nx - x) < 1e-15 * std::max(1.0, std::fabs(x))) { x = nx; break; }
    x = nx;
  }
  return x;
}

template <typename T>
int dalloc(T** p, size_t n, size_t* total) {
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) return fail(RX_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  *total += n * sizeof(T);
  e = cudaMemset(*p, 0, n * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
  return RX_OK;
}

void free_all(rx_handle* h) {
  RxDev& d = h->d;
  void* ptrs[] = {d.ring, d.Hs, d.Hf, d.tw, d.tw2, d.z, d.rot_hi, d.rot_lo, d.acc, d.psd, d.es, d.rec, d.st, d.w_acq,
                  d.chains, d.y, d.bl, d.run_int, d.run_m0, d.run_edge, d.bps_done, d.ber_done, d.dec, d.out, d.prbs_jump, d.ref,
                  d.sync_err, d.win_err, d.hist_y, d.hist_bhat, d.hist_m,
                  nullptr};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (void* p : h->stage)
    if (p) cudaFree(p);
  for (cudaEvent_t e : h->cd_done)
    if (e) cudaEventDestroy(e);
  for (auto& pf : h->pend) {
    cudaEventDestroy(pf.ev_in);
    cudaEventDestroy(pf.ev_start);
    cudaEventDestroy(pf.ev_done);
    for (auto& se : pf.sev) {
      cudaEventDestroy(se.a);
      cudaEventDestroy(se.b);
    }
  }
  for (auto& se : h->ingest_ev) {
    cudaEventDestroy(se.a);
    cudaEventDestroy(se.b);
  }
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  if (h->ev_copy) cudaEventDestroy(h->ev_copy);
  for (int i = 0; i < kStageSlots; ++i) {
    if (h->ev_stage_in[i]) cudaEventDestroy(h->ev_stage_in[i]);
    if (h->ev_stage_free[i]) cudaEventDestroy(h->ev_stage_free[i]);
  }
  if (h->ev_reset) cudaEventDestroy(h->ev_reset);
  if (h->s_copy) cudaStreamDestroy(h->s_copy);
  if (h->s_comp) cudaStreamDestroy(h->s_comp);
  if (h->s_comp2) cudaStreamDestroy(h->s_comp2);
  if (h->s_dem) cudaStreamDestroy(h->s_dem);
  if (h->s_mid) cudaStreamDestroy(h->s_mid);
  for (int i = 0; i < 2; ++i) {
    if (h->ev_mid[i]) cudaEventDestroy(h->ev_mid[i]);
    if (h->ev_bpsd[i]) cudaEventDestroy(h->ev_bpsd[i]);
    if (h->ev_bpsp[i]) cudaEventDestroy(h->ev_bpsp[i]);
  }
  if (h->s_front) cudaStreamDestroy(h->s_front);
  if (h->s_ber) cudaStreamDestroy(h->s_ber);
  for (int i = 0; i < 2; ++i) {
    if (h->ev_dem[i]) cudaEventDestroy(h->ev_dem[i]);
    if (h->ev_berd[i]) cudaEventDestroy(h->ev_berd[i]);
  }
  for (int i = 0; i < kZSlots; ++i) {
    if (h->ev_front[i]) cudaEventDestroy(h->ev_front[i]);
    if (h->ev_mimo[i]) cudaEventDestroy(h->ev_mimo[i]);
  }
}

// Harvest completed frames (in order): latency, device time, bits.
// Elapsed time between two recorded, complete events.  A batched call's
// events are shared by every stream it carried, and the streams are polled
// one after another: the last pair's result is reused.
float elapsed_ms(cudaEvent_t a, cudaEvent_t b, bool* ok) {
  thread_local cudaEvent_t la = nullptr, lb = nullptr;
  thread_local float lms = 0.f;
  thread_local bool lok = false;
  if (a == b) {
    *ok = true;
    return 0.f;
  }
  if (a != la || b != lb) {
    lok = cudaEventElapsedTime(&lms, a, b) == cudaSuccess;
    la = a;
    lb = b;
  }
  *ok = lok;
  return lms;
}

void harvest(rx_handle* h) {
  while (!h->pend.empty()) {
    PendingFrame& pf = h->pend.front();
    if (cudaEventQuery(pf.ev_done) != cudaSuccess) break;
    float a = 0.f, b = 0.f;
    if (pf.gen == h->gen) {
      bool ok = false;
      if (pf.shared) {  // a batched call: events recorded once, shared by its streams
        a = elapsed_ms(pf.ev_in, pf.ev_done, &ok);
        if (ok) h->lat_ms.push_back(a);
        b = elapsed_ms(pf.ev_start, pf.ev_done, &ok);
        if (ok) h->gpu_ms += b;
      } else {
        if (cudaEventElapsedTime(&a, pf.ev_in, pf.ev_done) == cudaSuccess) h->lat_ms.push_back(a);
        if (cudaEventElapsedTime(&b, pf.ev_start, pf.ev_done) == cudaSuccess) h->gpu_ms += b;
      }
      h->bits_done = pf.bits_after;
      h->dec_done = pf.dec_after;
      h->frames_done += pf.nframes;
    }
    for (auto& se : pf.sev) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, se.a, se.b) == cudaSuccess) h->stage_ms[se.stage] += ms;
      h->ev_pool.push_back(se.a);
      h->ev_pool.push_back(se.b);
    }
    if (!pf.shared) {
      h->ev_pool.push_back(pf.ev_in);
      h->ev_pool.push_back(pf.ev_start);
      h->ev_pool.push_back(pf.ev_done);
    }
    h->pend.pop_front();
  }
  while (!h->ingest_ev.empty()) {
    StageEv& se = h->ingest_ev.front();
    if (cudaEventQuery(se.b) != cudaSuccess) break;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, se.a, se.b) == cudaSuccess) h->stage_ms[RX_STAGE_INGEST] += ms;
    h->ev_pool.push_back(se.a);
    h->ev_pool.push_back(se.b);
    h->ingest_ev.pop_front();
  }
  cudaGetLastError();  // clear cudaErrorNotReady
}

// Runs fn (which enqueues work on the compute stream) between two timing
// events when profiling is on.
template <typename Fn>
int staged(rx_handle* h, PendingFrame& pf, int stage, cudaStream_t strm, Fn&& fn) {
  if (!h->cfg.profile) return fn();
  StageEv se{stage, get_event(h), get_event(h)};
  RX_CK(cudaEventRecord(se.a, strm));
  int rc = fn();
  RX_CK(cudaEventRecord(se.b, strm));
  pf.sev.push_back(se);
  return rc;
}

#define RX_STAGE(st, nk, strm, call)                                             \
  do {                                                                           \
    int rc_ = staged(h, pf, st, strm, [&]() -> int {                             \
      cudaError_t e_ = (call);                                                   \
      return e_ == cudaSuccess ? RX_OK : cuda_fail(e_, #call);                   \
    });                                                                          \
    if (rc_ != RX_OK) return rc_;                                                \
    h->stage_n[st] += (nk);                                                      \
  } while (0)

// Waits for everything the library has queued.
cudaError_t sync_all(rx_handle* h) {
  cudaError_t e = h->batch_done ? cudaEventSynchronize(h->batch_done) : cudaSuccess;
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s_copy);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s_front);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s_mid);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s_comp);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s_comp2);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s_dem);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s_ber);
  return e;
}

// Records ev_copy after the ingests queued so far (on the last push stream).
cudaError_t mark_copy(rx_handle* h) {
  if (!h->copy_dirty) return cudaSuccess;
  h->copy_dirty = false;
  return cudaEventRecord(h->ev_copy, h->last_cs);
}

BerPlan plan_ber(rx_handle* h, const FrameArgs& fa, bool final_) {
  const RxDev& d = h->d;
  BerPlan p;
  const long long ks = d.ber_skip;
  const long long need = ks + d.sync_syms;
  if (!h->synced && fa.k_b >= need && need <= fa.k_end && ks > d.sync_dmax) {
    p.sync = true;
    p.sync_sym0 = ks - d.sync_dmax;
    p.sync_nbits = (d.sync_syms + 2 * d.sync_dmax) * d.bps;
    p.launches += 2;
    h->synced = true;
    h->w_next = 0;
  }
  if (h->synced) {
    // count everything decided since the sync window start that is not yet counted
    // the sync window lies in the first frame, so counting starts there
    const long long ka = std::max(fa.k_a, ks);
    const long long hi = std::min(fa.k_b, fa.k_end);
    if (hi > ka) {
      p.ref = true;
      p.ref_sym0 = ka;
      p.ref_nbits = (int)((hi - ka) * d.bps);
      p.launches += 1;
    }
    const long long klim = final_ ? fa.k_end : fa.k_b;
    long long w_to = klim > ks ? (final_ ? (klim - ks + d.slip_win - 1) / d.slip_win : (klim - ks) / d.slip_win) : 0;
    if (w_to < h->w_next) w_to = h->w_next;
    if (hi > ka || w_to > h->w_next) p.launches += 1;  // count (+ slip pass in its last block)
    p.count = true;
    p.ka = ka;
    p.kb = std::max(hi, ka);
    p.w_from = h->w_next;
    p.w_to = w_to;
    p.k_lim = klim;
    h->w_next = w_to;
  }
  return p;
}

// Launch the decision stages (BPS .. BER) for decided range [k_a, k_b):
// BPS on the back stream, then unwrap/demap and the BER work on the BER
// stream, so the next pass's BPS overlaps this pass's demap.  pf.ev_done
// is recorded after the demap (the bits are out).
int launch_decide(rx_handle* h, PendingFrame& pf, const FrameArgs& fa, bool final_, cudaEvent_t after,
                  bool start_here) {
  const long long pass = h->n_decide;
  const int par = (int)(pass & 1);
  const RxDev d = decide_dev(h->d, pass);
  // the BPS of consecutive passes run on two streams (nothing of one is
  // read by the next: the unwrap scan runs with the demap)
  cudaStream_t sp = par ? h->s_comp2 : h->s_comp;
  RX_CK(cudaStreamWaitEvent(sp, after, 0));
  if (start_here) RX_CK(cudaEventRecord(pf.ev_start, sp));
  // this pass's decision buffers were read by the demap of pass n - 2
  if (pass >= 2) RX_CK(cudaStreamWaitEvent(sp, h->ev_dem[par], 0));
  RX_STAGE(RX_STAGE_BPS, 1, sp, launch_bps(d, fa, sp));
  if (fa.f >= 0) RX_CK(cudaEventRecord(h->ev_bpsd[fa.f & 1], sp));
  RX_CK(cudaEventRecord(h->ev_bpsp[par], sp));
  // unwrap scan + demap on their own stream, after the pass's BPS and after
  // the BER work of pass n - 2 has read the decision ring slots they write
  cudaStream_t sd = h->s_dem, sb = h->s_ber;
  RX_CK(cudaStreamWaitEvent(sd, h->ev_bpsp[par], 0));
  if (d.ber_on && pass >= 2) RX_CK(cudaStreamWaitEvent(sd, h->ev_berd[par], 0));
  RX_STAGE(RX_STAGE_DEMAP, 1, sd, launch_unwrap_demap(d, fa, sd));
  RX_CK(cudaEventRecord(h->ev_dem[par], sd));
  // the bits are out; with per-stage timing, the pass ends after its BER
  // work too, so every stage event of the pass is complete at ev_done
  if (!h->cfg.profile) RX_CK(cudaEventRecord(pf.ev_done, sd));
  h->n_decide++;
  if (d.ber_on) {
    RX_CK(cudaStreamWaitEvent(sb, h->ev_dem[par], 0));
    int rcb = staged(h, pf, RX_STAGE_BER, sb, [&]() -> int {
      const BerPlan p = plan_ber(h, fa, final_);
      if (p.sync) {
        RX_CK(launch_ref_gen(d, p.sync_sym0, p.sync_nbits, 0, sb));
        RX_CK(launch_sync(d, sb));
      }
      if (p.ref) RX_CK(launch_ref_gen(d, p.ref_sym0, p.ref_nbits, 1, sb));
      if (p.count) RX_CK(launch_ber(d, p.ka, p.kb, p.w_from, p.w_to, p.k_lim, h->n_win_ring, sb));
      h->stage_n[RX_STAGE_BER] += p.launches;
      return RX_OK;
    });
    if (rcb != RX_OK) return rcb;
    RX_CK(cudaEventRecord(h->ev_berd[par], sb));
  }
  if (h->cfg.profile) {
    RX_CK(cudaStreamWaitEvent(sd, h->ev_berd[par], 0));
    RX_CK(cudaEventRecord(pf.ev_done, sd));
  }
  return RX_OK;
}

FrameArgs frame_args(const rx_handle* h, long long f, bool final_) {
  const RxDev& d = h->d;
  const long long F = d.F;
  const long long n_sym = h->ended ? h->n_total / 2 : LLONG_MAX;
  FrameArgs fa{};
  fa.f = f;
  fa.Ff = (int)std::min(F, (h->ended ? n_sym : LLONG_MAX) - f * F);
  fa.s0 = 2 * f * F - d.c;
  fa.f0 = 2 * f * F;
  fa.f1 = fa.f0 + 2LL * fa.Ff;
  fa.n_valid = h->ended ? h->n_total : h->pushed;
  fa.k_a = std::max(f * F - d.W, 0LL);
  fa.k_b = final_ ? n_sym : (f + 1) * F - d.W;
  fa.k_end = h->ended ? n_sym - h->tail : LLONG_MAX;
  fa.n_sym = n_sym;
  fa.est_only = 0;
  fa.acc_slot = (int)(f & 1);
  return fa;
}

// The timing-acquisition CD pass before the first frame.
FrameArgs est_pass_args(const FrameArgs& fa) {
  FrameArgs fe = fa;
  fe.est_only = 1;
  fe.acc_slot = 2;
  return fe;
}

// Device state with frame f's slot: CD output and rotation tables of
// frames f and f + kZSlots share it.
RxDev slot_dev(const rx_handle* h, long long f) {
  const RxDev& d = h->d;
  const int slot = (int)(f % kZSlots);
  RxDev df = d;
  df.z = d.z + (long long)slot * 2 * d.zlen;
  df.rot_hi = d.rot_hi + (long long)slot * (d.zlen / kRotLo + 2);
  df.rot_lo = d.rot_lo + (long long)slot * kRotLo;
  return df;
}

// Device state of decide pass `pass`: the BPS angles / levels and run sums
// of passes n and n + 1 live in separate buffers, so the demap of pass n
// (on the BER stream) overlaps the BPS of pass n + 1 (on the back stream);
// the BPS of pass n + 2 waits for the demap of pass n.
RxDev decide_dev(const RxDev& base, long long pass) {
  RxDev dd = base;
  if (pass & 1) {
    const long long nruns = base.F / kRun + 4;
    dd.bl += 2LL * (base.F + 2 * base.W);
    dd.run_int += 2 * nruns;
    dd.run_m0 += 2 * nruns;
    dd.run_edge += 4 * nruns;
  }
  return dd;
}

// The decide-only pass at the stream end (the last W symbols, when the
// stream ended exactly at a frame end); k_a = k_b when there is none.
FrameArgs tail_args(const rx_handle* h) {
  const RxDev& d = h->d;
  const long long n_sym = h->n_total / 2;
  FrameArgs fa{};
  fa.f = h->f_next - 1;
  fa.Ff = d.F;
  fa.k_a = h->decided;
  fa.k_b = n_sym;
  fa.k_end = n_sym - h->tail;
  fa.n_sym = n_sym;
  return fa;
}

int launch_frame(rx_handle* h, long long f, bool final_) {
  RxDev& d = h->d;
  const FrameArgs fa = frame_args(h, f, final_);
  h->own_work = true;

  PendingFrame pf;
  pf.f = f;
  pf.gen = h->gen;
  pf.ev_in = get_event(h);
  pf.ev_start = get_event(h);
  pf.ev_done = get_event(h);
  const int slot = (int)(f % kZSlots);
  const RxDev df = slot_dev(h, f);
  cudaStream_t sf = h->s_front;
  RX_CK(mark_copy(h));
  RX_CK(cudaEventRecord(pf.ev_in, h->last_cs));
  // front: CD + estimator, after the input and after the slot's previous user
  RX_CK(cudaStreamWaitEvent(sf, h->ev_copy, 0));
  if (f >= kZSlots) RX_CK(cudaStreamWaitEvent(sf, h->ev_mimo[slot], 0));
  RX_CK(cudaEventRecord(pf.ev_start, sf));
  if (f == 0) {
    const FrameArgs fe = est_pass_args(fa);
    RX_STAGE(RX_STAGE_CD, 1, sf, launch_cd(df, fe, sf));
    RX_STAGE(RX_STAGE_EST, 1, sf, launch_est(df, fe, 0, sf));
  }
  RX_STAGE(RX_STAGE_CD, 1, sf, launch_cd(df, fa, sf));
  RX_CK(cudaEventRecord(h->cd_done[f % h->cd_done.size()], sf));
  RX_STAGE(RX_STAGE_EST, 1, sf, launch_est(df, fa, 1, sf));
  RX_CK(cudaEventRecord(h->ev_front[slot], sf));
  // middle: equaliser, after the frame's front work and after the decisions
  // of frame f - 2 have read the y buffer it reuses
  cudaStream_t sm = h->s_mid;
  RX_CK(cudaStreamWaitEvent(sm, h->ev_front[slot], 0));
  if (f >= 2) RX_CK(cudaStreamWaitEvent(sm, h->ev_bpsd[f & 1], 0));
  if (f == 0) RX_STAGE(RX_STAGE_ACQUIRE, 1, sm, launch_acquire(df, fa, sm));
  RX_STAGE(RX_STAGE_MIMO, 1, sm, launch_mimo(df, fa, sm));
  RX_CK(cudaEventRecord(h->ev_mimo[slot], sm));
  RX_CK(cudaEventRecord(h->ev_mid[f & 1], sm));
  // back: decisions, after the frame's equaliser (the MIMO of frame f + 1
  // runs meanwhile)
  int rc = launch_decide(h, pf, fa, final_, h->ev_mid[f & 1], false);
  if (rc != RX_OK) return rc;
  h->decided = fa.k_b;
  pf.dec_after = fa.k_b;
  pf.bits_after = 2LL * d.bps * fa.k_b;
  h->pend.push_back(pf);
  h->f_next = f + 1;
  return RX_OK;
}

// Decide the last W symbols when the stream ended exactly at a frame end.
int launch_tail(rx_handle* h) {
  RxDev& d = h->d;
  const long long n_sym = h->n_total / 2;
  if (h->f_next == 0 || h->decided >= n_sym) return RX_OK;
  const FrameArgs fa = tail_args(h);
  h->own_work = true;
  PendingFrame pf;
  pf.f = -1;
  pf.nframes = 0;
  pf.gen = h->gen;
  pf.ev_in = get_event(h);
  pf.ev_start = get_event(h);
  pf.ev_done = get_event(h);
  RX_CK(mark_copy(h));
  RX_CK(cudaEventRecord(pf.ev_in, h->last_cs));
  int rc = launch_decide(h, pf, fa, true, h->ev_copy, true);
  if (rc != RX_OK) return rc;
  h->decided = n_sym;
  pf.dec_after = n_sym;
  pf.bits_after = 2LL * d.bps * n_sym;
  h->pend.push_back(pf);
  return RX_OK;
}

int validate(const rx_config* c, std::string& why) {
  if (!(c->baud_hz > 0)) return why = "baud_hz must be > 0", RX_EINVAL;
  if (c->modulation != RX_QPSK && c->modulation != RX_QAM16) return why = "modulation must be RX_QPSK or RX_QAM16", RX_EINVAL;
  if (c->fiber_len_m < 0 || !(c->lambda_m > 0)) return why = "fiber_len_m >= 0 and lambda_m > 0 required", RX_EINVAL;
  if (c->mimo_taps < 3 || c->mimo_taps > kMaxTaps || (c->mimo_taps & 1) == 0) return why = "mimo_taps must be odd in [3, 31]", RX_EINVAL;
  if (c->bps_angles != 32 && c->bps_angles != 64) return why = "bps_angles must be 32 or 64", RX_EINVAL;
  const int W = c->bps_half_window;
  if (W != 8 && W != 12 && W != 16 && W != 24 && W != 32) return why = "bps_half_window must be one of 8, 12, 16, 24, 32", RX_EINVAL;
  if (c->bps_coarse_stride != 1 && c->bps_coarse_stride * (c->modulation == RX_QAM16 ? 8 : 16) != c->bps_angles)
    return why = "bps_coarse_stride must be 1 or bps_angles/16 (QPSK), bps_angles/8 (16QAM)", RX_EINVAL;
  if (c->mimo_block_warps != 0 && c->mimo_block_warps != 1 && c->mimo_block_warps != 2 && c->mimo_block_warps != 4 &&
      c->mimo_block_warps != 8)
    return why = "mimo_block_warps must be 0, 1, 2, 4 or 8", RX_EINVAL;
  if (c->bps_block_runs != 0 && c->bps_block_runs != 4 && c->bps_block_runs != 8)
    return why = "bps_block_runs must be 0, 4 or 8", RX_EINVAL;
  if (c->sub_block_syms != 64) return why = "sub_block_syms must be 64", RX_EINVAL;
  if (c->seg_syms < 64 || c->seg_syms % 64) return why = "seg_syms must be a positive multiple of 64", RX_EINVAL;
  if (c->frame_syms < c->seg_syms || c->frame_syms % c->seg_syms || c->frame_syms % kRun)
    return why = "frame_syms must be a multiple of seg_syms and of 256", RX_EINVAL;
  if (c->frame_syms > (1 << 24)) return why = "frame_syms must be <= 2^24", RX_EINVAL;
  if (c->acq_syms < 64 || c->acq_syms > c->frame_syms || c->cma_syms < 0) return why = "need 64 <= acq_syms <= frame_syms, cma_syms >= 0", RX_EINVAL;
  if (c->storage_dtype != RX_C64 && c->storage_dtype != RX_C16) return why = "storage_dtype must be RX_C64 or RX_C16", RX_EINVAL;
  if (c->max_block_samples < 1) return why = "max_block_samples must be >= 1", RX_EINVAL;
  if (c->prbs_seed) {
    if (c->slip_window < 32 || c->slip_window % 32) return why = "slip_window must be a positive multiple of 32", RX_EINVAL;
    if (c->ber_skip_syms <= c->sync_max_delay || c->sync_max_delay < 0) return why = "ber_skip_syms must exceed sync_max_delay", RX_EINVAL;
    if (c->sync_syms < 64) return why = "sync_syms must be >= 64", RX_EINVAL;
    if ((long long)c->ber_skip_syms + c->sync_syms + c->bps_half_window > c->frame_syms)
      return why = "frame_syms must cover ber_skip_syms + sync_syms + bps_half_window (sync in the first frame)", RX_EINVAL;
  }
  return RX_OK;
}

}  // namespace rxrt

namespace rx {
// Overlap-save halo M - 1 in samples: ceil(1.1 x CD memory) rounded up to
// even (or the configured cd_halo); CD memory = |D| L lambda^2 Rs (1 + rho) / c
// seconds of spread at fs = 2 Rs.
int cd_halo_samples(const rx_config* cfg) {
  const double Rs = cfg->baud_hz, fs = 2.0 * Rs;
  const double rho = std::max(cfg->rrc_rolloff, 0.0);
  const double Dsm = std::fabs(cfg->D_ps_nm_km) * 1e-6;
  const double dlam = cfg->lambda_m * cfg->lambda_m * Rs * (1.0 + rho) / kC;
  const double mem = Dsm * cfg->fiber_len_m * dlam * fs;
  int halo = cfg->cd_halo > 0 ? cfg->cd_halo : (int)std::ceil(1.1 * mem);
  halo += halo & 1;
  return std::max(halo, 2);
}

// Message for rx_last_error() from code outside this file.
void set_last_error(const char* msg) { g_err = msg; }

// Library-internal accessors for the serving layer (not part of the C ABI).
size_t handle_dev_bytes(const rx_handle* h) { return h->dev_bytes; }

// Frames launched and completed so far, and launched work not yet complete
// (frames and end-of-stream passes); completion is polled, nothing waits.
void handle_progress(rx_handle* h, long long* launched, long long* done, long long* pending) {
  harvest(h);
  *launched = h->f_next;
  *done = h->frames_done;
  *pending = (long long)h->pend.size();
}

// Frames launched so far (no polling).
long long handle_launched(const rx_handle* h) { return h->f_next; }

// Decided bits of completed frames not yet pulled, and the output ring's
// capacity in bits (as of the last poll).
void handle_bits(const rx_handle* h, long long* ready, long long* ring_bits) {
  *ready = h->bits_done - h->bits_pulled;
  *ring_bits = 8LL * h->d.out_cap_bytes;
}

// Queues on cs the copy of the bits rx_pull_bits(h, out, cap_bytes, n_bits,
// 0) would return into out (page-locked host memory) without marking them
// pulled: pull_bits_commit(h, *n_bits) does that once the copy is complete.
// Until then the output ring keeps those bits (pushes see them unpulled),
// and no other pull of h may come in between.
int pull_bits_begin(rx_handle* h, uint8_t* out, size_t cap_bytes, size_t* n_bits, cudaStream_t cs) {
  *n_bits = 0;
  harvest(h);
  const bool all_done = h->ended && h->pend.empty() && h->decided >= h->n_total / 2;
  const long long avail = h->bits_done - h->bits_pulled;
  long long nbytes = all_done ? (avail + 7) / 8 : avail / 8;
  nbytes = std::min<long long>(nbytes, (long long)cap_bytes);
  if (nbytes <= 0) return RX_OK;
  const long long cap = h->d.out_cap_bytes;
  const long long o = (h->bits_pulled / 8) % cap;
  const long long first = std::min(nbytes, cap - o);
  RX_CK(cudaMemcpyAsync(out, h->d.out + o, first, cudaMemcpyDeviceToHost, cs));
  if (nbytes > first) RX_CK(cudaMemcpyAsync(out + first, h->d.out, nbytes - first, cudaMemcpyDeviceToHost, cs));
  *n_bits = (size_t)std::min(nbytes * 8, avail);
  return RX_OK;
}

void pull_bits_commit(rx_handle* h, size_t n_bits) { h->bits_pulled += (long long)n_bits; }
}  // namespace rx

extern "C" {

const char* rx_last_error(void) { return g_err.c_str(); }

void rx_config_default(rx_config* c) {
  std::memset(c, 0, sizeof(*c));
  c->baud_hz = 28e9;
  c->modulation = RX_QPSK;
  c->fiber_len_m = 1000e3;
  c->D_ps_nm_km = 17.0;
  c->lambda_m = 1550e-9;
  c->rrc_rolloff = 0.1;
  c->fft_n = 0;
  c->cd_halo = 0;
  c->mimo_taps = 15;
  c->bps_angles = 64;
  c->bps_half_window = 16;
  c->bps_coarse_stride = 1;
  c->sub_block_syms = 64;
  c->seg_syms = 512;
  c->frame_syms = 1 << 16;
  c->cma_syms = 16384;
  c->acq_syms = 20480;
  c->mu_cma = 3e-2f;
  c->mu_dd = 5e-3f;
  c->timing_gain = 0.5f;
  c->storage_dtype = RX_C64;
  c->prbs_seed = 0;
  c->ber_skip_syms = 16384;
  c->sync_syms = 4096;
  c->sync_max_delay = 32;
  c->slip_window = 1024;
  c->max_block_samples = 1 << 17;
  c->history_syms = 0;
  c->profile = 0;
  c->device = 0;
}

int rx_create(const rx_config* cfg, rx_handle** out) {
  if (!cfg || !out) return fail(RX_EINVAL, "null argument");
  *out = nullptr;
  std::string why;
  if (validate(cfg, why) != RX_OK) return fail(RX_EINVAL, why);
  rx_handle* h = new rx_handle();
  h->cfg = *cfg;
  RxDev& d = h->d;
  std::memset(&d, 0, sizeof(d));
  // geometry (FP64)
  const double Rs = cfg->baud_hz, fs = 2.0 * Rs;
  const int halo = rx::cd_halo_samples(cfg);
  int N = cfg->fft_n;
  if (N <= 0) {
    N = 1024;
    while (N < 4 * halo && N < 16384) N *= 2;
    if (2 * halo > N) N *= 2;  // 16384 points would keep less than half of each block: 32768
  }
  if (N < 1024 || N > 32768 || (N & (N - 1))) { delete h; return fail(RX_EINVAL, "fft_n must be a power of two in [1024, 32768]"); }
  if (N - halo < 256) { delete h; return fail(RX_EINVAL, "CD halo too long for the FFT size (need N - halo >= 256)"); }
  {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
      cudaGetLastError();
      delete h;
      return fail(RX_EDEVICE, "no such CUDA device");
    }
    cudaError_t e = cudaSetDevice(cfg->device);
    if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaSetDevice"); }
  }
  d.N = N;
  d.halo = halo;
  d.h = halo / 2;
  d.L = N - halo;
  d.T = cfg->mimo_taps;
  d.c = (d.T - 1) / 2;
  d.K = 64;
  d.S = cfg->seg_syms;
  d.F = cfg->frame_syms;
  d.G = d.F / d.S;
  d.B = cfg->bps_angles;
  d.W = cfg->bps_half_window;
  d.bps_stride = cfg->bps_coarse_stride;
  d.bps_nw = cfg->bps_block_runs ? cfg->bps_block_runs : 8;
  d.mimo_nw = cfg->mimo_block_warps ? cfg->mimo_block_warps : 4;
  d.bps = cfg->modulation;
  d.nl = d.bps == 2 ? 2 : 4;
  d.zlen = 2 * d.F + 2 * d.c;
  d.storage = cfg->storage_dtype;
  d.Rs = Rs;
  d.fs = fs;
  d.mu_cma = cfg->mu_cma;
  d.mu_dd = cfg->mu_dd;
  d.R2 = d.bps == 2 ? 1.0f : 1.32f;
  d.timing_gain = cfg->timing_gain;
  d.cma_syms = cfg->cma_syms;
  d.acq_syms = cfg->acq_syms;
  d.ber_on = cfg->prbs_seed != 0;
  d.ber_skip = cfg->ber_skip_syms;
  d.sync_syms = cfg->sync_syms;
  d.sync_dmax = cfg->sync_max_delay;
  d.slip_win = cfg->slip_window;
  d.hist_syms = cfg->history_syms;

  h->tail = (d.h + 1) / 2 + d.T + d.W;
  // look-ahead: the last overlap-save block of a frame reads up to L + h + c
  // samples beyond the frame end; the BER end rule needs tail + W symbols
  h->la = std::max(d.L + d.h + d.c + 2, 2 * (h->tail + d.W + 2));
  const long long mb = (long long)cfg->max_block_samples;
  d.ring_cap = (2LL * d.F * kRingFrames + 2LL * h->la + d.c + d.h + mb + 1024 + 255) / 256 * 256;  // even: paired ingest
  d.out_cap_bytes = std::max<long long>(1 << 20, 32LL * d.F * 2 * d.bps / 8);
  d.dec_cap = 2LL * d.F + 8192;
  h->n_win_ring = d.F / std::max(d.slip_win, 32) + 8;
  const int nruns = d.F / kRun + 4;
  d.ref_words = (int)(((long long)(d.F + 2 * d.W + 2 * d.sync_dmax + d.sync_syms + d.ber_skip) * d.bps) / 32 + 8);

  int rc = RX_OK;
  const size_t elt = d.storage == RX_C16 ? 4 : 8;
  {
    cudaError_t e = cudaMalloc(&d.ring, 2 * d.ring_cap * elt);
    if (e != cudaSuccess) { free_all(h); delete h; return fail(RX_ENOMEM, "ring allocation failed"); }
    h->dev_bytes += 2 * d.ring_cap * elt;
    cudaMemset(d.ring, 0, 2 * d.ring_cap * elt);
  }
#define RX_AL(p, n) if ((rc = dalloc(&p, n, &h->dev_bytes)) != RX_OK) { free_all(h); delete h; return rc; }
  RX_AL(d.Hs, N);
  RX_AL(d.Hf, N);
  RX_AL(d.tw, N);
  RX_AL(d.tw2, 512 + kTwPass);  // [N table | N/2 table | pass table]: the 32768-point form's halves use the second
  RX_AL(d.z, (long long)kZSlots * 2 * d.zlen);
  RX_AL(d.rot_hi, (long long)kZSlots * (d.zlen / kRotLo + 2));
  RX_AL(d.rot_lo, (long long)kZSlots * kRotLo);
  RX_AL(d.acc, 3);
  RX_AL(d.psd, 3LL * (N / 2));
  RX_AL(d.es, 2);
  RX_AL(d.rec, kMaxTrace);
  RX_AL(d.st, 1);
  RX_AL(d.w_acq, 4 * d.T);
  RX_AL(d.chains, (size_t)d.G * 4 * d.T);
  RX_AL(d.y, 4LL * (kYHist + d.F));
  // decision buffers, two sets by decide-pass parity (decide_dev)
  RX_AL(d.bl, 2 * 2LL * (d.F + 2 * d.W));
  RX_AL(d.run_int, 2 * 2LL * nruns);
  RX_AL(d.run_m0, 2 * 2LL * nruns);
  RX_AL(d.run_edge, 2 * 4LL * nruns);
  RX_AL(d.bps_done, 2);
  RX_AL(d.ber_done, 2);
  RX_AL(d.dec, d.dec_cap);
  RX_AL(d.out, d.out_cap_bytes);
  RX_AL(d.prbs_jump, 64 * 31);
  RX_AL(d.ref, 2LL * d.ref_words + 4);
  RX_AL(d.sync_err, (size_t)(2 * d.sync_dmax + 1) * 2 * 8);
  RX_AL(d.win_err, (size_t)h->n_win_ring * 8);
  if (d.hist_syms > 0) {
    RX_AL(d.hist_y, 2LL * d.hist_syms);
    RX_AL(d.hist_bhat, 2LL * d.hist_syms);
    RX_AL(d.hist_m, 2LL * d.hist_syms);
  }
#undef RX_AL

  // CD x RRC response (FP64 phase reduced mod 2 pi), 1/N folded in; twiddles
  {
    const double L = cfg->fiber_len_m;
    const double Dsi = cfg->D_ps_nm_km * 1e-6;
    const double b2 = -Dsi * cfg->lambda_m * cfg->lambda_m / (2.0 * M_PI * kC);
    std::vector<float2> Hs(N), tw(N);
    for (int k = 0; k < N; ++k) {
      const double fk = (k < N / 2 ? k : k - N) * (fs / N);
      const double w = 2.0 * M_PI * fk;
      const double ph = std::fmod(b2 * L * w * w / 2.0, 2.0 * M_PI);
      double amp = 1.0 / N;
      if (cfg->rrc_rolloff >= 0) amp *= rrc_amp(fk, Rs, cfg->rrc_rolloff);
      Hs[k] = make_float2((float)(amp * std::cos(ph)), (float)(amp * std::sin(ph)));
      const double a = -2.0 * M_PI * (double)k / N;
      tw[k] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    cudaMemcpy(d.Hs, Hs.data(), N * sizeof(float2), cudaMemcpyHostToDevice);
    cudaMemcpy(d.Hf, Hs.data(), N * sizeof(float2), cudaMemcpyHostToDevice);
    cudaMemcpy(d.tw, tw.data(), N * sizeof(float2), cudaMemcpyHostToDevice);
    std::vector<float2> tw2(512 + kTwPass);
    for (int t = 0; t < 2; ++t) {
      const double Nt = (double)N / (1 << t);
      for (int i = 0; i < 128; ++i) {
        const double ah = -2.0 * M_PI * (double)(i * 128) / Nt, al = -2.0 * M_PI * (double)i / Nt;
        tw2[256 * t + i] = make_float2((float)std::cos(ah), (float)std::sin(ah));
        tw2[256 * t + 128 + i] = make_float2((float)std::cos(al), (float)std::sin(al));
      }
    }
    // the radix-16 passes at sub-transform length ns = 16, 256: entry
    // (r - 1) ns + m = exp(-2 pi i r m / (16 ns)), r = 1..15, m < ns
    for (int ns : {16, 256}) {
      float2* t = tw2.data() + 512 + (ns == 16 ? 0 : 15 * 16);
      for (int r = 1; r < 16; ++r)
        for (int m = 0; m < ns; ++m) {
          const double a = -2.0 * M_PI * (double)(r * m) / (16.0 * ns);
          t[(r - 1) * ns + m] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
    }
    cudaMemcpy(d.tw2, tw2.data(), tw2.size() * sizeof(float2), cudaMemcpyHostToDevice);
  }
  // PRBS jump matrices A^(2^i): A shifts the window down one bit and sets
  // bit 30 = bit 3 ^ bit 0.
  {
    std::vector<uint32_t> M(64 * 31);
    uint32_t A[31];
    for (int j = 0; j < 31; ++j) A[j] = (j >= 1 ? 1u << (j - 1) : 0u) | ((j == 0 || j == 3) ? 1u << 30 : 0u);
    std::memcpy(&M[0], A, sizeof(A));
    for (int i = 1; i < 64; ++i) gf2_mul(&M[(i - 1) * 31], &M[(i - 1) * 31], &M[i * 31]);
    cudaMemcpy(d.prbs_jump, M.data(), M.size() * 4, cudaMemcpyHostToDevice);
    d.prbs_state0[0] = prbs_state(cfg->prbs_seed, 0);
    d.prbs_state0[1] = prbs_state(cfg->prbs_seed, 1);
  }
  h->st_init = StreamState{};
  h->st_init.bhat_last[0] = h->st_init.bhat_last[1] = -1;
  cudaMemcpy(d.st, &h->st_init, sizeof(StreamState), cudaMemcpyHostToDevice);
  h->stage_bytes = (size_t)mb * 2 * 16;
  for (int i = 0; i < kStageSlots; ++i) {
    if (cudaMalloc(&h->stage[i], h->stage_bytes) != cudaSuccess) { free_all(h); delete h; return fail(RX_ENOMEM, "staging allocation failed"); }
    h->dev_bytes += h->stage_bytes;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&h->s_copy, cudaStreamNonBlocking);
  for (int i = 0; i < kStageSlots && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&h->ev_stage_in[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_stage_free[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_stage_free[i], h->s_copy);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_comp, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_comp2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_dem, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_mid, cudaStreamNonBlocking);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&h->ev_mid[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_bpsd[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_bpsp[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_front, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_ber, cudaStreamNonBlocking);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&h->ev_dem[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_berd[i], cudaEventDisableTiming);
  }
  for (int i = 0; i < kZSlots && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&h->ev_front[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_mimo[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_copy, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_reset, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_copy, h->s_copy);
  if (e == cudaSuccess) e = cd_set_attributes();
  if (e == cudaSuccess) e = bps_set_attributes();
  if (e == cudaSuccess) e = ber_set_attributes();
  for (int i = 0; i < 512 && e == cudaSuccess; ++i) {
    cudaEvent_t ev = nullptr;
    e = cudaEventCreate(&ev);
    if (e == cudaSuccess) h->ev_pool.push_back(ev);
  }
  h->cd_done.assign(64, nullptr);
  for (auto& ev : h->cd_done)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) { free_all(h); delete h; return cuda_fail(e, "rx_create"); }
  *out = h;
  return RX_OK;
}

int rx_push_block(rx_handle* h, const void* samples, size_t n_per_pol, int dtype, int on_device, void* cuda_stream) {
  if (!h) return fail(RX_EINVAL, "null handle");
  if (h->ended) return fail(RX_ESTATE, "push after end of stream");
  RX_CK(cudaSetDevice(h->cfg.device));
  RxDev& d = h->d;
  const long long F = d.F;
  if (samples == nullptr && n_per_pol == 0) {
    h->ended = true;
    h->n_total = h->pushed;
    const long long n_sym = h->n_total / 2;
    for (long long f = h->f_next; f * F < n_sym; ++f) {
      const bool fin = (f + 1) * F >= n_sym;
      int rc = launch_frame(h, f, fin);
      if (rc != RX_OK) return rc;
      if (fin) h->tail_launched = true;
    }
    if (!h->tail_launched) {
      int rc = launch_tail(h);
      if (rc != RX_OK) return rc;
    }
    return RX_OK;
  }
  if (samples == nullptr) return fail(RX_EINVAL, "samples is NULL");
  if (dtype < RX_C128 || dtype > RX_C16) return fail(RX_EINVAL, "bad dtype");
  if (n_per_pol > h->cfg.max_block_samples) return fail(RX_EINVAL, "n_per_pol exceeds max_block_samples");
  if (on_device < 0 || on_device > 3) return fail(RX_EINVAL, "on_device must be 0, 1, 2 or 3");
  if (n_per_pol == 0) return RX_OK;
  bool async_host = false;
  if (on_device >= 2) {
    // page-locked host memory, without a host wait (the caller keeps the
    // buffer until the stream has passed it): 2 = copied by a copy engine
    // into a staging slot in stream order; 3 = read by the ingest kernel
    // itself through the device mapping (no staging copy)
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, samples) != cudaSuccess || pa.type != cudaMemoryTypeHost ||
        pa.devicePointer == nullptr) {
      cudaGetLastError();
      return fail(RX_EINVAL, "on_device = 2 or 3 needs page-locked host memory mapped for the device");
    }
    if (on_device == 3) {
      samples = pa.devicePointer;
      on_device = 1;
    } else {
      async_host = true;
      on_device = 0;
    }
  }
  const long long n = (long long)n_per_pol;
  // output ring room for the frames this push completes
  {
    long long f = h->f_next, dec = h->decided;
    while (h->pushed + n >= 2 * (f + 1) * F + h->la) {
      dec = (f + 1) * F - d.W;
      ++f;
    }
    harvest(h);
    const long long bits_after = 2LL * d.bps * dec;
    if (bits_after - h->bits_pulled + 64 > 8LL * d.out_cap_bytes)
      return fail(RX_EAGAIN, "output ring full: pull bits first");
  }
  cudaStream_t cs = (cudaStream_t)cuda_stream;
  if (h->copy_dirty && cs != h->last_cs) {  // keep all ingests ordered on one stream's event
    RX_CK(mark_copy(h));
    RX_CK(cudaStreamWaitEvent(cs, h->ev_copy, 0));
  }
  // The copy runs on the caller's stream, so it is ordered after the
  // caller's queued work and the caller's later work is ordered after it.
  // Ring slots being overwritten must no longer be read by launched frames.
  const long long w1 = h->pushed + n;
  while (h->f_waited < h->f_next) {
    const long long ws = 2 * h->f_waited * F - d.c - d.h;
    if (ws >= w1 - d.ring_cap) break;
    RX_CK(cudaStreamWaitEvent(cs, h->cd_done[h->f_waited % h->cd_done.size()], 0));
    h->f_waited++;
  }
  if (h->reset_pending) {
    RX_CK(cudaStreamWaitEvent(cs, h->ev_reset, 0));
    h->reset_pending = false;
  }
  const size_t esz = dtype == RX_C128 ? 16 : (dtype == RX_C64 ? 8 : 4);
  const void* src = samples;
  int sl = -1;
  if (!on_device) {
    // The host->device copy runs on the copy stream into a staging slot, so
    // it does not wait for the ring-slot dependencies of the ingest; the
    // call returns once the copy (not the ingest) is done.
    sl = (int)(h->stage_i++ % kStageSlots);
    RX_CK(cudaStreamWaitEvent(h->s_copy, h->ev_stage_free[sl], 0));
    RX_CK(cudaMemcpyAsync(h->stage[sl], samples, 2 * n * esz, cudaMemcpyHostToDevice, h->s_copy));
    RX_CK(cudaEventRecord(h->ev_stage_in[sl], h->s_copy));
    RX_CK(cudaStreamWaitEvent(cs, h->ev_stage_in[sl], 0));
    src = h->stage[sl];
  }
  if (h->cfg.profile) {
    StageEv se{RX_STAGE_INGEST, get_event(h), get_event(h)};
    RX_CK(cudaEventRecord(se.a, cs));
    RX_CK(launch_ingest(d, src, dtype, n, h->pushed, cs));
    RX_CK(cudaEventRecord(se.b, cs));
    h->ingest_ev.push_back(se);
  } else {
    RX_CK(launch_ingest(d, src, dtype, n, h->pushed, cs));
  }
  h->stage_n[RX_STAGE_INGEST] += 1;
  h->last_cs = cs;
  h->copy_dirty = true;
  if (!on_device) {  // the host buffer is reusable on return
    RX_CK(cudaEventRecord(h->ev_stage_free[sl], cs));
    if (!async_host) RX_CK(cudaEventSynchronize(h->ev_stage_in[sl]));
  }
  h->pushed += n;
  while (h->pushed >= 2 * (h->f_next + 1) * F + h->la) {
    int rc = launch_frame(h, h->f_next, false);
    if (rc != RX_OK) return rc;
  }
  return RX_OK;
}

int rx_pull_bits(rx_handle* h, uint8_t* out, size_t cap_bytes, size_t* n_bits, int timeout_ms) {
  if (!h || (!out && cap_bytes) || !n_bits) return fail(RX_EINVAL, "null argument");
  RX_CK(cudaSetDevice(h->cfg.device));
  *n_bits = 0;
  int rc = RX_OK;
  if (timeout_ms < 0) {
    RX_CK(sync_all(h));
  } else if (timeout_ms > 0) {
    auto t0 = std::chrono::steady_clock::now();
    while (true) {
      harvest(h);
      if (h->pend.empty()) break;
      if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms)) { rc = RX_ETIMEDOUT; break; }
      std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
  }
  harvest(h);
  cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess && le != cudaErrorNotReady) return cuda_fail(le, "device");
  const bool all_done = h->ended && h->pend.empty() && h->decided >= h->n_total / 2;
  long long avail = h->bits_done - h->bits_pulled;
  long long nbytes = all_done ? (avail + 7) / 8 : avail / 8;
  nbytes = std::min<long long>(nbytes, (long long)cap_bytes);
  if (nbytes > 0) {
    const long long b0 = h->bits_pulled / 8;
    const long long cap = h->d.out_cap_bytes;
    const long long o = b0 % cap;
    const long long first = std::min(nbytes, cap - o);
    RX_CK(cudaMemcpy(out, h->d.out + o, first, cudaMemcpyDeviceToHost));
    if (nbytes > first) RX_CK(cudaMemcpy(out + first, h->d.out, nbytes - first, cudaMemcpyDeviceToHost));
    const long long nb = std::min(nbytes * 8, avail);
    h->bits_pulled += nb;
    *n_bits = (size_t)nb;
  }
  if (rc != RX_OK) g_err = "pull wait timed out";
  return rc;
}

int rx_stats(rx_handle* h, rx_stats_t* out) {
  if (!h || !out) return fail(RX_EINVAL, "null argument");
  RX_CK(cudaSetDevice(h->cfg.device));
  RX_CK(sync_all(h));
  harvest(h);
  StreamState st;
  RX_CK(cudaMemcpy(&st, h->d.st, sizeof(st), cudaMemcpyDeviceToHost));
  std::memset(out, 0, sizeof(*out));
  out->samples_in = (uint64_t)h->pushed;
  out->symbols_out = (uint64_t)h->dec_done;
  out->frames = (uint64_t)h->frames_done;
  out->bits = st.bits;
  out->bit_errors = st.errors;
  out->ber = st.bits ? (double)st.errors / (double)st.bits : 0.0;
  out->q_db = 0.0;
  if (out->ber > 0 && out->ber < 0.5) out->q_db = 20.0 * std::log10(std::sqrt(2.0) * erfcinv_host(2.0 * out->ber));
  out->evm = st.evm_den > 0 ? st.evm_num / st.evm_den : 0.0;
  out->cycle_slips = st.slips;
  out->synced = st.synced;
  out->sync_delay = st.sync_delay;
  out->sync_perm = st.sync_perm;
  out->sync_quadrant_x = st.sync_q[0];
  out->sync_quadrant_y = st.sync_q[1];
  out->cma_reinit = st.reinit;
  const long long last = std::min<long long>(h->f_next, kMaxTrace) - 1;
  if (last >= 0) {
    FrameRec r;
    RX_CK(cudaMemcpy(&r, h->d.rec + last, sizeof(r), cudaMemcpyDeviceToHost));
    out->fo_hz = r.dfo;
    out->tau_s = r.tau;
  }
  if (!h->lat_ms.empty()) {
    std::vector<double> v = h->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) { return v[std::min(v.size() - 1, (size_t)std::floor(p * (v.size() - 1) + 0.5))]; };
    out->latency_p50_ms = pct(0.5);
    out->latency_p99_ms = pct(0.99);
  }
  out->gpu_ms_total = h->gpu_ms;
  return RX_OK;
}

int rx_destroy(rx_handle* h) {
  if (!h) return RX_OK;
  cudaSetDevice(h->cfg.device);
  if (h->s_front) cudaStreamSynchronize(h->s_front);
  if (h->s_mid) cudaStreamSynchronize(h->s_mid);
  if (h->s_comp) cudaStreamSynchronize(h->s_comp);
  if (h->s_comp2) cudaStreamSynchronize(h->s_comp2);
  if (h->s_dem) cudaStreamSynchronize(h->s_dem);
  if (h->s_ber) cudaStreamSynchronize(h->s_ber);
  if (h->s_copy) cudaStreamSynchronize(h->s_copy);
  free_all(h);
  delete h;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RX_OK : cuda_fail(e, "rx_destroy");
}

int rx_reset(rx_handle* h) {
  if (!h) return fail(RX_EINVAL, "null handle");
  RX_CK(cudaSetDevice(h->cfg.device));
  harvest(h);
  RxDev& d = h->d;
  cudaStream_t s = h->s_comp;
  // stream-ordered: runs after all queued frames (front and back), before the
  // next stream's work
  RX_CK(mark_copy(h));
  RX_CK(cudaStreamWaitEvent(s, h->ev_copy, 0));
  RX_CK(cudaEventRecord(h->ev_front[0], h->s_front));
  RX_CK(cudaStreamWaitEvent(s, h->ev_front[0], 0));
  RX_CK(cudaEventRecord(h->ev_berd[0], h->s_ber));
  RX_CK(cudaStreamWaitEvent(s, h->ev_berd[0], 0));
  RX_CK(cudaEventRecord(h->ev_mid[0], h->s_mid));
  RX_CK(cudaStreamWaitEvent(s, h->ev_mid[0], 0));
  RX_CK(cudaEventRecord(h->ev_bpsp[1], h->s_comp2));
  RX_CK(cudaStreamWaitEvent(s, h->ev_bpsp[1], 0));
  RX_CK(cudaEventRecord(h->ev_dem[1], h->s_dem));
  RX_CK(cudaStreamWaitEvent(s, h->ev_dem[1], 0));
  RX_CK(cudaMemcpyAsync(d.st, &h->st_init, sizeof(StreamState), cudaMemcpyHostToDevice, s));
  RX_CK(cudaMemcpyAsync(d.Hf, d.Hs, d.N * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  RX_CK(cudaMemsetAsync(d.acc, 0, 3 * sizeof(FrameAcc), s));
  RX_CK(cudaMemsetAsync(d.psd, 0, 3LL * (d.N / 2) * sizeof(double), s));
  RX_CK(cudaMemsetAsync(d.es, 0, 2 * sizeof(EstState), s));
  RX_CK(cudaMemsetAsync(d.win_err, 0, (size_t)h->n_win_ring * 8 * sizeof(unsigned), s));
  RX_CK(cudaMemsetAsync(d.rec, 0, kMaxTrace * sizeof(FrameRec), s));
  if (d.hist_syms > 0) {
    RX_CK(cudaMemsetAsync(d.hist_y, 0, 2 * d.hist_syms * sizeof(float2), s));
    RX_CK(cudaMemsetAsync(d.hist_bhat, 0, 2 * d.hist_syms, s));
    RX_CK(cudaMemsetAsync(d.hist_m, 0, 2 * d.hist_syms * sizeof(int), s));
  }
  RX_CK(cudaEventRecord(h->ev_reset, s));
  RX_CK(cudaStreamWaitEvent(h->s_front, h->ev_reset, 0));
  RX_CK(cudaStreamWaitEvent(h->s_comp2, h->ev_reset, 0));
  RX_CK(cudaStreamWaitEvent(h->s_dem, h->ev_reset, 0));
  RX_CK(cudaStreamWaitEvent(h->s_ber, h->ev_reset, 0));
  RX_CK(cudaStreamWaitEvent(h->s_mid, h->ev_reset, 0));
  h->n_decide = 0;
  h->reset_pending = true;
  h->gen++;
  h->pushed = 0;
  h->n_total = -1;
  h->ended = false;
  h->f_next = h->f_waited = 0;
  h->decided = h->bits_done = h->bits_pulled = h->dec_done = 0;
  h->synced = h->tail_launched = false;
  h->w_next = 0;
  h->lat_ms.clear();
  h->gpu_ms = 0.0;
  h->frames_done = 0;
  return RX_OK;
}

int rx_join(rx_handle* h, void* cuda_stream) {
  if (!h) return fail(RX_EINVAL, "null handle");
  RX_CK(cudaSetDevice(h->cfg.device));
  cudaStream_t ss[6] = {h->s_comp, h->s_comp2, h->s_dem, h->s_front, h->s_ber, h->s_mid};
  for (cudaStream_t x : ss) {
    cudaEvent_t e = get_event(h);
    RX_CK(cudaEventRecord(e, x));
    RX_CK(cudaStreamWaitEvent((cudaStream_t)cuda_stream, e, 0));
    h->ev_pool.push_back(e);
  }
  return RX_OK;
}

int rx_stage_times(rx_handle* h, double* ms, int64_t* launches) {
  if (!h || !ms || !launches) return fail(RX_EINVAL, "null argument");
  RX_CK(cudaSetDevice(h->cfg.device));
  RX_CK(cudaStreamSynchronize(h->s_copy));
  RX_CK(sync_all(h));
  harvest(h);
  for (int i = 0; i < RX_NSTAGES; ++i) {
    ms[i] = h->stage_ms[i];
    launches[i] = h->stage_n[i];
  }
  return RX_OK;
}

int rx_frame_trace(rx_handle* h, double* out, int cap_frames) {
  if (!h || !out) return fail(RX_EINVAL, "null argument");
  RX_CK(cudaSetDevice(h->cfg.device));
  RX_CK(sync_all(h));
  const int n = (int)std::min<long long>(std::min<long long>(h->f_next, kMaxTrace), cap_frames);
  std::vector<FrameRec> r(n);
  if (n > 0) RX_CK(cudaMemcpy(r.data(), h->d.rec, n * sizeof(FrameRec), cudaMemcpyDeviceToHost));
  for (int i = 0; i < n; ++i) {
    out[4 * i + 0] = r[i].tau;
    out[4 * i + 1] = r[i].dfo;
    out[4 * i + 2] = r[i].gain;
    out[4 * i + 3] = r[i].theta;
  }
  return n;
}

int rx_get_taps(rx_handle* h, int which, float* out) {
  if (!h || !out) return fail(RX_EINVAL, "null argument");
  if (which < -1 || which >= h->d.G) return fail(RX_EINVAL, "no such chain");
  RX_CK(cudaSetDevice(h->cfg.device));
  RX_CK(sync_all(h));
  const float2* src = which < 0 ? h->d.w_acq : h->d.chains + (size_t)which * 4 * h->d.T;
  RX_CK(cudaMemcpy(out, src, 4 * h->d.T * sizeof(float2), cudaMemcpyDeviceToHost));
  return RX_OK;
}

int rx_get_equalised(rx_handle* h, int64_t first, int64_t n, float* out) {
  if (!h || !out) return fail(RX_EINVAL, "null argument");
  const long long H = h->d.hist_syms;
  if (first < 0 || n < 0 || first + n > H) return fail(RX_EINVAL, "range outside the inspection history");
  RX_CK(cudaSetDevice(h->cfg.device));
  RX_CK(sync_all(h));
  for (int p = 0; p < 2; ++p)
    RX_CK(cudaMemcpy(out + 2 * p * n, h->d.hist_y + p * H + first, n * sizeof(float2), cudaMemcpyDeviceToHost));
  return RX_OK;
}

int rx_get_phase(rx_handle* h, int64_t first, int64_t n, uint8_t* bhat, int32_t* m) {
  if (!h || !bhat || !m) return fail(RX_EINVAL, "null argument");
  const long long H = h->d.hist_syms;
  if (first < 0 || n < 0 || first + n > H) return fail(RX_EINVAL, "range outside the inspection history");
  RX_CK(cudaSetDevice(h->cfg.device));
  RX_CK(sync_all(h));
  for (int p = 0; p < 2; ++p) {
    RX_CK(cudaMemcpy(bhat + p * n, h->d.hist_bhat + p * H + first, n, cudaMemcpyDeviceToHost));
    RX_CK(cudaMemcpy(m + p * n, h->d.hist_m + p * H + first, n * 4, cudaMemcpyDeviceToHost));
  }
  return RX_OK;
}

}  // extern "C"
