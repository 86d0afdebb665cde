// Host runtime of the KK receiver chain (paper Sec. II): ADC codes ->
// field (the rx_kk front end) -> static equaliser with 4 -> 2 samples per
// symbol -> widely-linear DD-LMS -> decisions -> packed bits.
//
// Each stage keeps its own stream positions:
//   front end   codes pushed / field samples out (rx_kk);
//   equaliser   field samples in (in4) / 2-sps samples out (out2), a whole
//               number of segments of N4/4 until the end; segment b needs
//               field up to b N4/2 + 3N4/4, and a carry holds the field of
//               [2 out2 - N4/4, in4) (fewer than N4 samples);
//   DD-LMS      frames of F symbols; frame f runs once the 2-sps samples
//               reach 2(f+1)F + 1 (its last symbol's taps read x[2k + 2]);
//               the first frame is preceded by the acquisition chain.
// The 2-sps samples wait in one of two buffers from 2fF - 2 on; after the
// frames of a push the rest moves to the other buffer's front.
//
// Streams: the front end runs on the caller's stream, the equaliser, the
// DD-LMS and the decisions on the handle's own (non-blocking) stream, so
// the front end of push k + 1 overlaps the equaliser and DD-LMS of push k.
// The front end writes its field into one of two buffers (push k: buffer
// k mod 2); an event per buffer hands it to the equaliser, another hands it
// back once the equaliser has read it.  rx_kkrx_end joins the handle's
// stream back onto the caller's.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/rx.h"
#include "kkrx_internal.h"

namespace rx {
void set_last_error(const char* msg);
}

struct rx_kkrx {
  rx_kkrx_config cfg;
  rx_kk* fe = nullptr;
  int N4 = 0, L4 = 0, L2 = 0, F = 0, S = 0, bps = 0;
  bool ended = false;
  // equaliser stage
  long long in4 = 0, out2 = 0;
  int cur4 = 0;
  float2* carry4[2] = {nullptr, nullptr};
  float2* field[2] = {nullptr, nullptr};  // the front end's output of push k in field[k & 1]
  size_t field_cap = 0;
  long long npush = 0;       // pushes (and the end) that ran the front end
  cudaStream_t s2 = nullptr; // equaliser + DD-LMS stream
  cudaEvent_t ev_field[2] = {nullptr, nullptr}, ev_read[2] = {nullptr, nullptr}, ev_join = nullptr;
  float2* H2 = nullptr;
  float2* tw4 = nullptr;
  // DD-LMS stage
  float2* x2buf[2] = {nullptr, nullptr};
  int curx = 0;
  long long x2_base = -2, x2_cap = 0;
  long long frames = 0;      // frames done
  float2* taps = nullptr;    // [F/S][8]
  float2* acq_taps = nullptr;
  float2* init_taps = nullptr;
  float2* hist = nullptr;
};

namespace {

int fail(const char* msg, int rc) {
  rx::set_last_error(msg);
  return rc;
}

int cuda_rc(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return RX_OK;
  static thread_local char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  cudaGetLastError();
  return fail(buf, RX_EDEVICE);
}

long long kk_out_after(long long in_pos, int N) {  // the front end's output position
  const long long q = in_pos - N / 4;
  return q >= N / 2 ? q / (N / 2) * (N / 2) : 0;
}

long long eq_out_after(const rx_kkrx* h, long long in4) {
  const long long q = in4 - h->N4 / 4;
  return q >= h->L4 ? q / h->L4 * h->L2 : 0;
}

// The equaliser step over the new field [in4, in4 + n) (in field) that
// produces 2-sps samples up to out2_new, without launching: its arguments,
// segments and carry start.
struct EqPlan {
  rx::KKEqArgs a;
  long long nseg, keep;
  long long n, out2_new;
};

int eq_plan(const rx_kkrx* h, const float2* field, long long n, long long out2_new, EqPlan* p) {
  rx::KKEqArgs& a = p->a;
  a.carry = h->carry4[h->cur4];
  a.carry_start = std::max(0LL, 2 * h->out2 - h->N4 / 4);
  a.in = field;
  a.new_start = h->in4;
  a.in_end = h->in4 + n;
  a.seg0 = h->out2 / h->L2;
  a.out = h->x2buf[h->curx];
  a.out_base = h->x2_base;
  a.out_end = out2_new;
  a.H2 = h->H2;
  a.tw2 = h->tw4;
  if (out2_new - h->x2_base > h->x2_cap) return fail("rx_kkrx: internal 2-sps buffer overflow", RX_EINVAL);
  p->nseg = (out2_new - h->out2 + h->L2 - 1) / h->L2;
  p->keep = std::max(0LL, 2 * out2_new - h->N4 / 4);
  p->n = n;
  p->out2_new = out2_new;
  return RX_OK;
}

void eq_commit(rx_kkrx* h, const EqPlan& p) {
  h->cur4 ^= 1;
  h->in4 += p.n;
  h->out2 = p.out2_new;
}

int run_eq(rx_kkrx* h, const float2* field, long long n, long long out2_new, cudaStream_t s) {
  EqPlan p;
  int rc = eq_plan(h, field, n, out2_new, &p);
  if (rc) return rc;
  rc = cuda_rc(rx::launch_kkeq(p.a, h->N4, p.nseg, s), "rx_kkrx: equaliser kernel");
  if (rc) return rc;
  rc = cuda_rc(rx::launch_kkeq_tail(p.a.carry, p.a.carry_start, p.a.in, p.a.new_start, p.keep, p.a.in_end,
                                    h->carry4[h->cur4 ^ 1], s),
               "rx_kkrx: equaliser carry");
  if (rc) return rc;
  eq_commit(h, p);
  return RX_OK;
}

// Frames that can run with the 2-sps samples up to out2 (end: every frame
// left of the n_sym_end symbols).
long long frames_ready(const rx_kkrx* h, long long out2, bool end, long long n_sym_end) {
  if (end) return (n_sym_end + h->F - 1) / h->F - h->frames;
  long long f = h->frames;
  while (out2 >= 2LL * (f + 1) * h->F + 1) ++f;
  return f - h->frames;
}

// The DD-LMS work of `count` frames (the last may be short when end is
// set), without launching: the acquisition before the first frame, each
// frame's arguments and segment count in order (bits of frame frames + i
// go to bits + i F bps / 8), the move of the remaining 2-sps samples to the
// other buffer, and the state after it.
struct FramePlan {
  bool has_acq = false;
  rx::WLArgs acq;
  std::vector<rx::WLArgs> frames;
  std::vector<long long> segs;
  long long shift_n = 0;  // samples moved (0: none)
  const float2* shift_src = nullptr;
  float2* shift_dst = nullptr;
  long long frames_after = 0, x2_base_after = 0;
  int curx_after = 0;
};

FramePlan plan_frames(const rx_kkrx* h, long long count, bool end, long long n_sym_end, uint8_t* bits) {
  FramePlan p;
  const long long n2 = end ? h->out2 : (1LL << 62);  // before the end every sample read exists
  rx::WLArgs base;
  std::memset(&base, 0, sizeof(base));
  base.x2 = h->x2buf[h->curx];
  base.x2_base = h->x2_base;
  base.n2 = n2;
  base.mu = h->cfg.mu;
  const float2* first_taps = h->acq_taps;
  for (long long i = 0; i < count; ++i) {
    const long long f = h->frames + i;
    const long long k_a = f * (long long)h->F;
    const long long k_end = end ? std::min(k_a + h->F, n_sym_end) : k_a + h->F;
    if (f == 0) {  // acquisition: one sequential chain over the first symbols
      const long long acq = std::min<long long>(h->cfg.acq_syms, end ? n_sym_end : h->cfg.acq_syms);
      if (acq > 0) {
        p.has_acq = true;
        p.acq = base;
        p.acq.k_a = 0;
        p.acq.k_end = acq;
        p.acq.seg = acq;
        p.acq.taps_in = h->init_taps;
        p.acq.taps_out = h->acq_taps;
      } else {
        first_taps = h->init_taps;  // nothing to acquire on: frame 0 starts from the initial taps
      }
    }
    rx::WLArgs w = base;
    w.k_a = k_a;
    w.k_end = k_end;
    w.seg = h->S;
    w.taps_in = f == 0 ? first_taps : h->taps;
    w.taps_in_stride = f == 0 ? 0 : 8;
    w.taps_out = h->taps;
    w.bits = bits + i * ((long long)h->F * h->bps / 8);
    w.k_bits = k_a;
    w.hist = h->hist;
    w.hist_syms = h->cfg.history_syms;
    p.frames.push_back(w);
    p.segs.push_back((k_end - k_a + h->S - 1) / h->S);
  }
  p.frames_after = h->frames + count;
  p.curx_after = h->curx;
  p.x2_base_after = h->x2_base;
  if (count > 0 && !end) {  // keep the 2-sps samples from 2 frames F - 2 on
    const long long nb = 2 * p.frames_after * (long long)h->F - 2;
    const long long keep = h->out2 - nb;
    if (keep > 0) {
      p.shift_n = keep;
      p.shift_src = h->x2buf[h->curx] + (nb - h->x2_base);
      p.shift_dst = h->x2buf[h->curx ^ 1];
    }
    p.curx_after = h->curx ^ 1;
    p.x2_base_after = nb;
  }
  return p;
}

void commit_frames(rx_kkrx* h, const FramePlan& p) {
  h->frames = p.frames_after;
  h->curx = p.curx_after;
  h->x2_base = p.x2_base_after;
}

int run_frames(rx_kkrx* h, long long count, bool end, long long n_sym_end, uint8_t* bits, cudaStream_t s) {
  const bool q16 = h->cfg.modulation == RX_QAM16;
  const FramePlan p = plan_frames(h, count, end, n_sym_end, bits);
  int rc = RX_OK;
  if (p.has_acq) rc = cuda_rc(rx::launch_wl(p.acq, q16, 1, s), "rx_kkrx: acquisition");
  for (size_t i = 0; i < p.frames.size() && !rc; ++i)
    rc = cuda_rc(rx::launch_wl(p.frames[i], q16, p.segs[i], s), "rx_kkrx: DD-LMS");
  if (!rc && p.shift_n > 0)
    rc = cuda_rc(cudaMemcpyAsync(p.shift_dst, p.shift_src, p.shift_n * sizeof(float2), cudaMemcpyDeviceToDevice, s),
                 "rx_kkrx: 2-sps carry");
  if (rc) return rc;
  commit_frames(h, p);
  return RX_OK;
}

}  // namespace

extern "C" void rx_kkrx_config_default(rx_kkrx_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  rx_kk_config_default(&c->fe);
  c->baud_hz = 1e9;
  c->modulation = RX_QPSK;
  c->fiber_len_m = 0.0;
  c->D_ps_nm_km = 17.0;
  c->lambda_m = 1550e-9;
  c->rrc_rolloff = 0.01;
  c->eq_fft_n = 1024;
  c->mu = 5e-3f;
  c->seg_syms = 512;
  c->frame_syms = 1 << 20;
  c->acq_syms = 8192;
  c->history_syms = 0;
}

extern "C" int rx_kkrx_create(const rx_kkrx_config* cfg, rx_kkrx** out) {
  if (!cfg || !out) return fail("rx_kkrx_create: null argument", RX_EINVAL);
  *out = nullptr;
  const rx_kkrx_config& c = *cfg;
  if (!(c.baud_hz > 0.0) || std::fabs(c.fe.fs_hz - 4.0 * c.baud_hz) > 1e-6 * c.fe.fs_hz)
    return fail("rx_kkrx_create: fe.fs_hz must be 4 x baud_hz (4 samples per symbol)", RX_EINVAL);
  if (c.modulation != RX_QPSK && c.modulation != RX_QAM16)
    return fail("rx_kkrx_create: modulation must be RX_QPSK or RX_QAM16", RX_EINVAL);
  if (c.eq_fft_n != 1024 && c.eq_fft_n != 2048) return fail("rx_kkrx_create: eq_fft_n must be 1024 or 2048", RX_EINVAL);
  if (!(c.rrc_rolloff > 0.0 && c.rrc_rolloff <= 1.0)) return fail("rx_kkrx_create: rrc_rolloff must be in (0, 1]", RX_EINVAL);
  if (!(c.mu > 0.f && c.mu < 1.f)) return fail("rx_kkrx_create: mu must be in (0, 1)", RX_EINVAL);
  if (c.seg_syms < 64 || c.seg_syms % 64) return fail("rx_kkrx_create: seg_syms must be a multiple of 64", RX_EINVAL);
  if (c.frame_syms < c.seg_syms || c.frame_syms % c.seg_syms || c.frame_syms > (1 << 24))
    return fail("rx_kkrx_create: frame_syms must be a multiple of seg_syms, at most 2^24", RX_EINVAL);
  if (c.acq_syms < 0 || c.acq_syms % 64 || c.acq_syms > c.frame_syms)
    return fail("rx_kkrx_create: acq_syms must be a multiple of 64 and at most frame_syms", RX_EINVAL);
  if (c.history_syms < 0) return fail("rx_kkrx_create: history_syms must be >= 0", RX_EINVAL);
  rx_kkrx* h = new rx_kkrx;
  h->cfg = c;
  int rc = rx_kk_create(&c.fe, &h->fe);
  if (rc) {
    delete h;
    return rc;
  }
  h->N4 = c.eq_fft_n;
  h->L4 = h->N4 / 2;
  h->L2 = h->N4 / 4;
  h->F = c.frame_syms;
  h->S = c.seg_syms;
  h->bps = c.modulation;
  h->field_cap = c.fe.max_block_samples + c.fe.fft_n;
  // 2-sps samples waiting: two frames' worth plus one push's output
  h->x2_cap = 2LL * h->F + 16 + (long long)(c.fe.max_block_samples + c.fe.fft_n + h->N4) / 2 + h->L2;
  bool ok = cudaMalloc(&h->field[0], h->field_cap * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&h->field[1], h->field_cap * sizeof(float2)) == cudaSuccess &&
            cudaStreamCreateWithFlags(&h->s2, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&h->ev_field[0], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&h->ev_field[1], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&h->ev_read[0], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&h->ev_read[1], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) == cudaSuccess &&
            cudaMalloc(&h->carry4[0], h->N4 * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&h->carry4[1], h->N4 * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&h->H2, (h->N4 / 2) * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&h->tw4, 256 * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&h->x2buf[0], h->x2_cap * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&h->x2buf[1], h->x2_cap * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&h->taps, (size_t)(h->F / h->S) * 8 * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&h->acq_taps, 8 * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&h->init_taps, 8 * sizeof(float2)) == cudaSuccess &&
            (c.history_syms == 0 || cudaMalloc(&h->hist, c.history_syms * sizeof(float2)) == cudaSuccess);
  if (ok) {
    // static equaliser: exp(+j beta2 L w^2 / 2) at w = 2 pi (f + f_shift) x RRC(f), FP64, phase
    // reduced mod 2 pi; bins 0 .. N4/4 - 1 then -N4/4 .. -1 (f = k fs / N4); 1/N4 folded in
    const double fs = c.fe.fs_hz, Rs = c.baud_hz, rho = c.rrc_rolloff;
    const double b2 = -(c.D_ps_nm_km * 1e-6) * c.lambda_m * c.lambda_m / (2.0 * M_PI * 299792458.0);
    std::vector<float2> H(h->N4 / 2), tw(256), init(8, make_float2(0.f, 0.f));
    for (int i = 0; i < h->N4 / 2; ++i) {
      const int k = i < h->N4 / 4 ? i : i - h->N4 / 2;
      const double f = k * fs / h->N4;
      const double w = 2.0 * M_PI * (f + c.fe.f_shift_hz);
      const double ph = std::fmod(b2 * c.fiber_len_m * w * w / 2.0, 2.0 * M_PI);
      const double a = std::fabs(f) / Rs;
      double amp = 0.0;
      if (a <= (1 - rho) / 2) amp = 1.0;
      else if (a <= (1 + rho) / 2) amp = std::sqrt(0.5 * (1.0 + std::cos(M_PI / rho * (a - (1 - rho) / 2))));
      amp /= h->N4;
      H[i] = make_float2((float)(amp * std::cos(ph)), (float)(amp * std::sin(ph)));
    }
    for (int i = 0; i < 128; ++i) {
      const double ah = -2.0 * M_PI * (double)(i * 128) / h->N4, al = -2.0 * M_PI * (double)i / h->N4;
      tw[i] = make_float2((float)std::cos(ah), (float)std::sin(ah));
      tw[128 + i] = make_float2((float)std::cos(al), (float)std::sin(al));
    }
    init[1] = make_float2(1.f, 0.f);  // h1 = unit tap at offset 0, h2 = 0
    ok = cudaMemcpy(h->H2, H.data(), H.size() * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(h->tw4, tw.data(), 256 * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(h->init_taps, init.data(), 8 * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    rx_kkrx_destroy(h);
    return fail("rx_kkrx_create: device allocation failed", RX_ENOMEM);
  }
  *out = h;
  return RX_OK;
}

// What a push of n codes will complete: the front end's new field
// samples, the equaliser's output position, the frames and their bytes.
struct PushForecast {
  long long c1, out2_new, nf;
  size_t need;
};

PushForecast forecast(const rx_kkrx* h, size_t n) {
  int64_t fin = 0, fout = 0;
  rx_kk_position(h->fe, &fin, &fout);
  PushForecast f;
  f.c1 = kk_out_after(fin + (long long)n, h->cfg.fe.fft_n) - fout;
  f.out2_new = eq_out_after(h, h->in4 + f.c1);
  f.nf = frames_ready(h, f.out2_new, false, 0);
  f.need = (size_t)f.nf * ((size_t)h->F * h->bps / 8);
  return f;
}

extern "C" int rx_kkrx_push(rx_kkrx* h, const int16_t* codes, size_t n, int on_device, uint8_t* bits,
                            size_t bits_cap_bytes, size_t* n_bits, void* cuda_stream) {
  if (!h || !n_bits || (n > 0 && !codes)) return fail("rx_kkrx_push: null argument", RX_EINVAL);
  *n_bits = 0;
  if (h->ended) return fail("rx_kkrx_push: stream already ended", RX_ESTATE);
  if (n > h->cfg.fe.max_block_samples) return fail("rx_kkrx_push: n exceeds fe.max_block_samples", RX_EINVAL);
  if (n == 0) return RX_OK;
  const PushForecast fc = forecast(h, n);
  const long long c1 = fc.c1, out2_new = fc.out2_new, nf = fc.nf;
  const size_t need = fc.need;
  if (need > 0 && (!bits || bits_cap_bytes < need))
    return fail("rx_kkrx_push: bits is null or bits_cap_bytes is smaller than the frames this push completes",
                RX_EINVAL);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int fb = (int)(h->npush & 1);
  int rc = RX_OK;
  if (h->npush >= 2) rc = cuda_rc(cudaStreamWaitEvent(s, h->ev_read[fb], 0), "rx_kkrx_push: field buffer");
  if (rc) return rc;
  size_t got = 0;
  rc = rx_kk_push(h->fe, codes, n, on_device, reinterpret_cast<float*>(h->field[fb]), h->field_cap, &got, s);
  if (rc) return rc;
  if ((long long)got != c1) return fail("rx_kkrx_push: front-end output count mismatch", RX_EINVAL);
  h->npush++;
  rc = cuda_rc(cudaEventRecord(h->ev_field[fb], s), "rx_kkrx_push: event");
  if (!rc) rc = cuda_rc(cudaStreamWaitEvent(h->s2, h->ev_field[fb], 0), "rx_kkrx_push: event");
  if (!rc && got > 0) rc = run_eq(h, h->field[fb], (long long)got, out2_new, h->s2);
  if (!rc) rc = cuda_rc(cudaEventRecord(h->ev_read[fb], h->s2), "rx_kkrx_push: event");
  if (!rc) rc = run_frames(h, nf, false, 0, bits, h->s2);
  if (rc) return rc;
  *n_bits = need * 8;
  return RX_OK;
}

extern "C" int rx_kkrx_end(rx_kkrx* h, uint8_t* bits, size_t bits_cap_bytes, size_t* n_bits, void* cuda_stream) {
  if (!h || !n_bits) return fail("rx_kkrx_end: null argument", RX_EINVAL);
  *n_bits = 0;
  if (h->ended) return fail("rx_kkrx_end: stream already ended", RX_ESTATE);
  int64_t fin = 0, fout = 0;
  rx_kk_position(h->fe, &fin, &fout);
  const long long n4 = fin;            // every code becomes a field sample
  const long long n2 = n4 / 2;
  const long long n_sym = n2 / 2;
  const long long nf = frames_ready(h, n2, true, n_sym);
  const long long last = n_sym - (h->frames + std::max(nf, 1LL) - 1) * (long long)h->F;
  const size_t need = nf > 0 ? (size_t)(nf - 1) * ((size_t)h->F * h->bps / 8) + (size_t)(last * h->bps + 7) / 8 : 0;
  if (need > 0 && (!bits || bits_cap_bytes < need))
    return fail("rx_kkrx_end: bits is null or bits_cap_bytes is smaller than the remaining frames' bits", RX_EINVAL);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int fb = (int)(h->npush & 1);
  int rc = RX_OK;
  if (h->npush >= 2) rc = cuda_rc(cudaStreamWaitEvent(s, h->ev_read[fb], 0), "rx_kkrx_end: field buffer");
  if (rc) return rc;
  size_t got = 0;
  rc = rx_kk_end(h->fe, reinterpret_cast<float*>(h->field[fb]), h->field_cap, &got, s);
  if (rc) return rc;
  h->npush++;
  rc = cuda_rc(cudaEventRecord(h->ev_field[fb], s), "rx_kkrx_end: event");
  if (!rc) rc = cuda_rc(cudaStreamWaitEvent(h->s2, h->ev_field[fb], 0), "rx_kkrx_end: event");
  if (!rc && n2 > h->out2) rc = run_eq(h, h->field[fb], (long long)got, n2, h->s2);
  if (!rc) rc = cuda_rc(cudaEventRecord(h->ev_read[fb], h->s2), "rx_kkrx_end: event");
  if (!rc) rc = run_frames(h, nf, true, n_sym, bits, h->s2);
  // the bits and the handle's state are complete in the caller's stream order from here
  if (!rc) rc = cuda_rc(cudaEventRecord(h->ev_join, h->s2), "rx_kkrx_end: join");
  if (!rc) rc = cuda_rc(cudaStreamWaitEvent(s, h->ev_join, 0), "rx_kkrx_end: join");
  if (rc) return rc;
  h->ended = true;
  *n_bits = nf > 0 ? (size_t)((nf - 1) * (long long)h->F + last) * h->bps : 0;
  return RX_OK;
}

extern "C" int rx_kkrx_equalised(rx_kkrx* h, int64_t first, int64_t n, float* out) {
  if (!h || (n > 0 && !out)) return fail("rx_kkrx_equalised: null argument", RX_EINVAL);
  if (first < 0 || n < 0 || first + n > h->cfg.history_syms)
    return fail("rx_kkrx_equalised: range outside history_syms", RX_EINVAL);
  if (n == 0) return RX_OK;
  cudaSetDevice(h->cfg.fe.device);
  if (cudaDeviceSynchronize() != cudaSuccess) return cuda_rc(cudaGetLastError(), "rx_kkrx_equalised");
  return cuda_rc(cudaMemcpy(out, h->hist + first, n * sizeof(float2), cudaMemcpyDeviceToHost), "rx_kkrx_equalised");
}

extern "C" int rx_kkrx_reset(rx_kkrx* h) {
  if (!h) return fail("rx_kkrx_reset: null handle", RX_EINVAL);
  const int rc = cuda_rc(cudaStreamSynchronize(h->s2), "rx_kkrx_reset");  // no work of the old stream in flight
  if (rc) return rc;
  h->npush = 0;
  rx_kk_reset(h->fe);
  h->ended = false;
  h->in4 = h->out2 = 0;
  h->cur4 = h->curx = 0;
  h->x2_base = -2;
  h->frames = 0;
  return RX_OK;
}

extern "C" void rx_kkrx_destroy(rx_kkrx* h) {
  if (!h) return;
  cudaSetDevice(h->cfg.fe.device);
  rx_kk_destroy(h->fe);
  if (h->s2) cudaStreamSynchronize(h->s2);
  cudaFree(h->field[0]);
  cudaFree(h->field[1]);
  for (int i = 0; i < 2; ++i) {
    if (h->ev_field[i]) cudaEventDestroy(h->ev_field[i]);
    if (h->ev_read[i]) cudaEventDestroy(h->ev_read[i]);
  }
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->s2) cudaStreamDestroy(h->s2);
  cudaFree(h->carry4[0]);
  cudaFree(h->carry4[1]);
  cudaFree(h->H2);
  cudaFree(h->tw4);
  cudaFree(h->x2buf[0]);
  cudaFree(h->x2buf[1]);
  cudaFree(h->taps);
  cudaFree(h->acq_taps);
  cudaFree(h->init_taps);
  cudaFree(h->hist);
  delete h;
}

// ---- many receivers in one launch per stage -------------------------------
//
// A batch push runs every channel's front end through one rx_kk_batch graph
// replay, then one replay of a graph of the equaliser (a block per output
// segment of any channel, found from the prefix sums of the channels'
// uneven segment counts) and its carries, then the DD-LMS of the frames
// that completed: one launch for every channel's acquisition, one for the
// first frame each channel completed, one for the second, ... (a channel's
// frames stay in order), and one for the moves of the 2-sps samples.  All
// on the caller's stream.  Two table slots (with a graph each) alternate,
// as in rx_kk_batch.

struct rx_kkrx_batch {
  std::vector<rx_kkrx*> ch;
  rx_kk_batch* fe = nullptr;
  int N4 = 0, device = 0, slot = 0;
  rx::KKEqBatchTable* host_tab[2] = {nullptr, nullptr};
  rx::KKEqBatchTable* dev_tab[2] = {nullptr, nullptr};
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaGraphNode_t eq_node[2] = {nullptr, nullptr};
  cudaKernelNodeParams eq_params[2];
  cudaEvent_t done[2] = {nullptr, nullptr};
  bool used[2] = {false, false};
  rx::WLBatchTable* host_wl[2] = {nullptr, nullptr};
  rx::WLBatchTable* dev_wl[2] = {nullptr, nullptr};
};

extern "C" int rx_kkrx_batch_create(rx_kkrx* const* channels, int n_channels, rx_kkrx_batch** out) {
  if (!channels || !out || n_channels < 1) return fail("rx_kkrx_batch_create: null argument or no channels", RX_EINVAL);
  *out = nullptr;
  if (n_channels > rx::kKKEqBatchMax) return fail("rx_kkrx_batch_create: at most 256 channels", RX_EINVAL);
  for (int c = 0; c < n_channels; ++c) {
    const rx_kkrx* h = channels[c];
    if (!h) return fail("rx_kkrx_batch_create: null channel", RX_EINVAL);
    const rx_kkrx* h0 = channels[0];
    if (h->N4 != h0->N4 || h->F != h0->F || h->S != h0->S || h->bps != h0->bps ||
        h->cfg.acq_syms != h0->cfg.acq_syms || h->cfg.fe.fft_n != h0->cfg.fe.fft_n ||
        h->cfg.fe.device != h0->cfg.fe.device)
      return fail("rx_kkrx_batch_create: channels must share fft_n, eq_fft_n, frame, segment and acquisition "
                  "lengths, modulation and device", RX_EINVAL);
    for (int d = 0; d < c; ++d)
      if (channels[d] == channels[c]) return fail("rx_kkrx_batch_create: a channel appears twice", RX_EINVAL);
  }
  rx_kkrx_batch* b = new rx_kkrx_batch;
  b->ch.assign(channels, channels + n_channels);
  b->N4 = channels[0]->N4;
  b->device = channels[0]->cfg.fe.device;
  int rc = cuda_rc(cudaSetDevice(b->device), "rx_kkrx_batch_create");
  for (int c = 0; c < n_channels && !rc; ++c)  // no single-push work of a channel still in flight
    rc = cuda_rc(cudaStreamSynchronize(channels[c]->s2), "rx_kkrx_batch_create");
  std::vector<rx_kk*> fes(n_channels);
  for (int c = 0; c < n_channels; ++c) fes[c] = channels[c]->fe;
  if (!rc) rc = rx_kk_batch_create(fes.data(), n_channels, &b->fe);
  for (int k = 0; k < 2 && !rc; ++k) {
    rc = cuda_rc(cudaHostAlloc(&b->host_tab[k], sizeof(rx::KKEqBatchTable), cudaHostAllocDefault), "table");
    if (!rc) rc = cuda_rc(cudaMalloc(&b->dev_tab[k], sizeof(rx::KKEqBatchTable)), "table");
    if (!rc) rc = cuda_rc(cudaEventCreateWithFlags(&b->done[k], cudaEventDisableTiming), "event");
    if (!rc) rc = cuda_rc(cudaHostAlloc(&b->host_wl[k], sizeof(rx::WLBatchTable), cudaHostAllocDefault), "table");
    if (!rc) rc = cuda_rc(cudaMalloc(&b->dev_wl[k], sizeof(rx::WLBatchTable)), "table");
    if (rc) break;
    std::memset(b->host_tab[k], 0, sizeof(rx::KKEqBatchTable));
    cudaKernelNodeParams eq, tail;
    rc = cuda_rc(rx::kkeq_batch_nodes(b->N4, &eq, &tail), "rx_kkrx_batch_create: kernels");
    if (!rc) rc = cuda_rc(cudaGraphCreate(&b->graph[k], 0), "graph");
    cudaGraphNode_t copy = nullptr, tnode = nullptr;
    if (!rc)
      rc = cuda_rc(cudaGraphAddMemcpyNode1D(&copy, b->graph[k], nullptr, 0, b->dev_tab[k], b->host_tab[k],
                                            sizeof(rx::KKEqBatchTable), cudaMemcpyHostToDevice),
                   "graph copy node");
    void* arg[1] = {&b->dev_tab[k]};
    eq.gridDim = dim3(1);
    eq.kernelParams = arg;
    tail.gridDim = dim3((unsigned)n_channels);
    tail.kernelParams = arg;
    if (!rc) rc = cuda_rc(cudaGraphAddKernelNode(&b->eq_node[k], b->graph[k], &copy, 1, &eq), "equaliser node");
    if (!rc) rc = cuda_rc(cudaGraphAddKernelNode(&tnode, b->graph[k], &b->eq_node[k], 1, &tail), "carry node");
    if (!rc) rc = cuda_rc(cudaGraphInstantiate(&b->exec[k], b->graph[k], 0), "graph instantiate");
    b->eq_params[k] = eq;
  }
  if (rc) {
    rx_kkrx_batch_destroy(b);
    return rc;
  }
  *out = b;
  return RX_OK;
}

extern "C" int rx_kkrx_batch_push(rx_kkrx_batch* b, const int16_t* const* codes, const size_t* n,
                                  uint8_t* const* bits, const size_t* bits_cap_bytes, size_t* n_bits,
                                  void* cuda_stream) {
  if (!b || !codes || !n || !bits || !bits_cap_bytes || !n_bits)
    return fail("rx_kkrx_batch_push: null argument", RX_EINVAL);
  const int nch = (int)b->ch.size();
  std::vector<PushForecast> fc(nch);
  for (int c = 0; c < nch; ++c) {  // all or nothing: check every channel first
    rx_kkrx* h = b->ch[c];
    n_bits[c] = 0;
    if (h->ended) return fail("rx_kkrx_batch_push: a channel's stream already ended", RX_ESTATE);
    if (n[c] > h->cfg.fe.max_block_samples) return fail("rx_kkrx_batch_push: n exceeds fe.max_block_samples", RX_EINVAL);
    if (n[c] > 0 && !codes[c]) return fail("rx_kkrx_batch_push: null codes", RX_EINVAL);
    fc[c] = forecast(h, n[c]);
    if (fc[c].need > 0 && (!bits[c] || bits_cap_bytes[c] < fc[c].need))
      return fail("rx_kkrx_batch_push: a channel's bits capacity is smaller than the frames the push completes",
                  RX_EINVAL);
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int rc = cuda_rc(cudaSetDevice(b->device), "rx_kkrx_batch_push");
  if (rc) return rc;
  // front ends: one graph replay
  std::vector<float*> fout(nch);
  std::vector<size_t> fcap(nch), got(nch);
  for (int c = 0; c < nch; ++c) {
    fout[c] = reinterpret_cast<float*>(b->ch[c]->field[b->ch[c]->npush & 1]);
    fcap[c] = b->ch[c]->field_cap;
  }
  rc = rx_kk_batch_push(b->fe, codes, n, fout.data(), fcap.data(), got.data(), cuda_stream);
  if (rc) return rc;
  // equalisers: one graph replay over every channel's new segments
  const int k = b->slot;
  if (b->used[k]) {
    rc = cuda_rc(cudaEventSynchronize(b->done[k]), "rx_kkrx_batch_push: table slot");
    if (rc) return rc;
  }
  rx::KKEqBatchTable* t = b->host_tab[k];
  std::vector<EqPlan> plans(nch);
  t->nch = nch;
  t->offs[0] = 0;
  for (int c = 0; c < nch; ++c) {
    rx_kkrx* h = b->ch[c];
    if ((long long)got[c] != fc[c].c1) return fail("rx_kkrx_batch_push: front-end output count mismatch", RX_EINVAL);
    if (got[c] > 0) {
      rc = eq_plan(h, h->field[h->npush & 1], (long long)got[c], fc[c].out2_new, &plans[c]);
      if (rc) return rc;
    } else {  // no new field: no segments and an empty carry copy
      plans[c].a.in_end = h->in4;
      plans[c].nseg = 0;
      plans[c].keep = h->in4;
    }
    t->args[c] = plans[c].a;
    t->offs[c + 1] = t->offs[c] + plans[c].nseg;
    t->carry_dst[c] = h->carry4[h->cur4 ^ 1];
    t->keep_from[c] = plans[c].keep;
  }
  if (t->offs[nch] > 0x7fffffffLL) return fail("rx_kkrx_batch_push: too many segments in one batch", RX_EINVAL);
  cudaKernelNodeParams ep = b->eq_params[k];
  void* arg[1] = {&b->dev_tab[k]};
  ep.kernelParams = arg;
  ep.gridDim = dim3((unsigned)std::max(1LL, t->offs[nch]));
  rc = cuda_rc(cudaGraphExecKernelNodeSetParams(b->exec[k], b->eq_node[k], &ep), "rx_kkrx_batch_push: grid");
  if (!rc) rc = cuda_rc(cudaGraphLaunch(b->exec[k], s), "rx_kkrx_batch_push: graph");
  if (rc) return rc;
  for (int c = 0; c < nch; ++c) {
    rx_kkrx* h = b->ch[c];
    if (n[c] > 0) h->npush++;
    if (got[c] > 0) eq_commit(h, plans[c]);
  }
  // DD-LMS of the frames that completed: one launch for every acquisition,
  // one per frame ordinal, one for the moves of the 2-sps samples (a channel
  // with more frames than ordinals runs them on its own, in order)
  const bool q16 = b->ch[0]->cfg.modulation == RX_QAM16;
  rx::WLBatchTable* w = b->host_wl[k];
  for (int node = 0; node < rx::kWLNodes; ++node) {
    w->n[node] = 0;
    w->offs[node][0] = 0;
  }
  w->nshift = 0;
  for (int c = 0; c < nch; ++c) {
    rx_kkrx* h = b->ch[c];
    n_bits[c] = fc[c].need * 8;
    if (fc[c].nf == 0) continue;
    if (fc[c].nf > rx::kWLNodes - 1) {
      rc = run_frames(h, fc[c].nf, false, 0, bits[c], s);
      if (rc) return rc;
      continue;
    }
    const FramePlan fp = plan_frames(h, fc[c].nf, false, 0, bits[c]);
    auto add = [&](int node, const rx::WLArgs& a, long long segs) {
      const int e = w->n[node]++;
      w->args[node][e] = a;
      w->offs[node][e + 1] = w->offs[node][e] + segs;
    };
    if (fp.has_acq) add(0, fp.acq, 1);
    for (size_t i = 0; i < fp.frames.size(); ++i) add(1 + (int)i, fp.frames[i], fp.segs[i]);
    if (fp.shift_n > 0) {
      w->shift_src[w->nshift] = fp.shift_src;
      w->shift_dst[w->nshift] = fp.shift_dst;
      w->shift_n[w->nshift] = fp.shift_n;
      w->nshift++;
    }
    commit_frames(h, fp);
  }
  bool any = w->nshift > 0;
  for (int node = 0; node < rx::kWLNodes; ++node) any = any || w->n[node] > 0;
  if (any) {
    rc = cuda_rc(cudaMemcpyAsync(b->dev_wl[k], w, sizeof(rx::WLBatchTable), cudaMemcpyHostToDevice, s),
                 "rx_kkrx_batch_push: DD-LMS table");
    for (int node = 0; node < rx::kWLNodes && !rc; ++node)
      rc = cuda_rc(rx::launch_wl_batch(b->dev_wl[k], node, q16, w->offs[node][w->n[node]], s),
                   "rx_kkrx_batch_push: DD-LMS");
    if (!rc) rc = cuda_rc(rx::launch_x2_shift_batch(b->dev_wl[k], w->nshift, s), "rx_kkrx_batch_push: 2-sps carry");
    if (rc) return rc;
  }
  rc = cuda_rc(cudaEventRecord(b->done[k], s), "rx_kkrx_batch_push: event");
  if (rc) return rc;
  b->used[k] = true;
  b->slot ^= 1;
  return RX_OK;
}

extern "C" void rx_kkrx_batch_destroy(rx_kkrx_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  for (int k = 0; k < 2; ++k) {
    if (b->done[k]) cudaEventSynchronize(b->done[k]);
    if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
    if (b->graph[k]) cudaGraphDestroy(b->graph[k]);
    if (b->done[k]) cudaEventDestroy(b->done[k]);
    cudaFreeHost(b->host_tab[k]);
    cudaFree(b->dev_tab[k]);
    cudaFreeHost(b->host_wl[k]);
    cudaFree(b->dev_wl[k]);
  }
  rx_kk_batch_destroy(b->fe);
  delete b;
}
