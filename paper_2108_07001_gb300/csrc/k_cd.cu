// a1 chromatic-dispersion compensation by overlap-save, with the frame's
// timing (a3) and frequency-offset (a2) statistics accumulated on the fly,
// and the per-frame estimator kernel.
//
// Overlap-save (paper Sec. II: 100 % overlap-save frequency-domain
// processing; the overlap with the previous buffer is carried so the
// stream is contiguous, and CD is compensated in the frequency domain):
// block j of a frame keeps output samples [s0 + jL, s0 + (j+1)L) from the
// circular filtering of input samples [s0 + jL - h, +N) (zero outside the
// stream), H = exp(+j beta2 L w^2 / 2) * RRC * exp(+j w tau) / N.
//
// One thread block per (OLS block, polarisation): the window is read from
// the device ring straight into shared memory (the halo is just the
// neighbouring ring samples, no copy), transformed, filtered, inverse
// transformed and the kept samples are written once.  While the spectrum is
// in shared memory the block adds its Godard band-edge correlation
// sum_{k<N/2} Y[k] conj(Y[k+N/2]) (times (-1)^window_start) to the frame
// accumulator; after the inverse transform it adds the in-frame power and
// the periodogram |FFT_{N/2}(z^4)|^2 of its symbol-spaced in-frame samples
// (Welch average over blocks and polarisations, FP64 sums of the FP32 block
// terms, so the result does not depend on the order of the blocks).  The first
// forward pass reads the window from the ring into registers, the filter
// and the Godard sum ride on the last forward pass, and the last inverse
// pass writes z and the periodogram input directly, so each transform
// makes one shared-memory round trip fewer per end.
#include <cooperative_groups.h>

#include "fft_smem.cuh"

namespace rx {

template <int NT>
__device__ __forceinline__ float block_sum(float v, float* scratch) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  float r = 0.f;
  if (w == 0) {
    r = (l < NT / 32) ? scratch[l] : 0.f;
    r = warp_sum(r);
  }
  return r;  // valid in warp 0
}

template <int N, int NT, int STOR>
__device__ __forceinline__ void cd_ols_body(const RxDev& d, const FrameArgs& fa, VBlock vb) {
  extern __shared__ float2 buf[];
  __shared__ float scratch[NT / 32];
  __shared__ float2 tw_s[2 * kTwSplit];  // [hi | lo] two-level twiddle table
  constexpr bool TP = N >= 8192;          // the direct pass table repays its copy from 8192 points on
  __shared__ float2 tp_s[TP ? kTwPass : 1];
  for (int i = threadIdx.x; i < 2 * kTwSplit; i += NT) tw_s[i] = d.tw2[i];
  if (TP)
    for (int i = threadIdx.x; i < kTwPass; i += NT) tp_s[i] = d.tw2[4 * kTwSplit + i];
  const int pol = vb.y;
  const long long a = fa.s0 + (long long)vb.x * d.L;
  const long long zlen_f = 2LL * fa.Ff + 2 * d.c;
  const int keep = (int)min((long long)d.L, fa.s0 + zlen_f - a);
  const long long lo = a - d.h;
  const long long rbase = (long long)pol * d.ring_cap;
  // ring slot of window sample 0 (the window is shorter than the ring, so
  // it wraps at most once)
  long long r0 = lo % d.ring_cap;
  if (r0 < 0) r0 += d.ring_cap;

  // first forward pass (radix 16, no twiddles) straight from the ring:
  // butterfly j takes window samples j + r N/16
  const bool interior = lo >= 0 && lo + N <= fa.n_valid && r0 + N <= d.ring_cap;
  {
    constexpr int NB = N / 16;
    constexpr int PER = (NB + NT - 1) / NT;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int j = threadIdx.x + u * NT;
      if ((NB % NT) == 0 || j < NB) {
        float2 v[16];
        if (interior) {  // the window lies inside the stream and does not wrap the ring
          const long long b0 = rbase + r0 + j;
#pragma unroll
          for (int r = 0; r < 16; ++r) v[r] = load_sample(d.ring, STOR, b0 + r * NB);
        } else {
#pragma unroll
          for (int r = 0; r < 16; ++r) {
            const int i = j + r * NB;
            const long long n = lo + i;
            long long slot = r0 + i;
            if (slot >= d.ring_cap) slot -= d.ring_cap;
            v[r] = (n >= 0 && n < fa.n_valid) ? load_sample(d.ring, STOR, rbase + slot) : make_float2(0.f, 0.f);
          }
        }
        dft<16, false>(v);
#pragma unroll
        for (int r = 0; r < 16; ++r) buf[swz(16 * j + r)] = v[r];
      }
    }
  }
  __syncthreads();
  constexpr int NSL = last_ns<N>();  // sub-transform length of the last pass
  constexpr int RL = N / NSL;        // its radix; its butterfly j (< NSL) outputs bins j + r NSL
  constexpr int PERL = (NSL + NT - 1) / NT;
  fft_passes<N, NT, 16, NSL, false, TP>(buf, tw_s, 1, tp_s);

  // last forward pass, filter and Godard sum over bin pairs (k, k + N/2) =
  // outputs (r, r + RL/2) of one butterfly
  float gr = 0.f, gi = 0.f;
  {
    float2 v[PERL][RL];
#pragma unroll
    for (int u = 0; u < PERL; ++u) {
      const int j = threadIdx.x + u * NT;
      if ((NSL % NT) == 0 || j < NSL) {
#pragma unroll
        for (int r = 0; r < RL; ++r) v[u][r] = buf[swz(j + r * NSL)];
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PERL; ++u) {
      const int j = threadIdx.x + u * NT;
      if ((NSL % NT) == 0 || j < NSL) {
        pass_butterfly<N, RL, NSL, false, TP>(v[u], j, tw_s, 1, tp_s);
#pragma unroll
        for (int r = 0; r < RL; ++r) v[u][r] = cmul(v[u][r], __ldg(&d.Hf[j + r * NSL]));
#pragma unroll
        for (int r = 0; r < RL / 2; ++r) {
          const float2 p = cmulc(v[u][r], v[u][r + RL / 2]);
          gr += p.x;
          gi += p.y;
        }
        if (!fa.est_only) {
#pragma unroll
          for (int r = 0; r < RL; ++r) buf[swz(j + r * NSL)] = v[u][r];
        }
      }
    }
  }
  gr = block_sum<NT>(gr, scratch);
  gi = block_sum<NT>(gi, scratch);
  if (threadIdx.x == 0) {
    const float sg = (lo & 1) ? -1.f : 1.f;
    FrameAcc* acc = d.acc + fa.acc_slot;
    atomicAdd(&acc->C[0], (double)(sg * gr));
    atomicAdd(&acc->C[1], (double)(sg * gi));
  }
  if (fa.est_only) return;
  fft_passes<N, NT, 1, NSL, true, TP>(buf, tw_s, 1, tp_s);  // block_sum ended with a barrier

  // last inverse pass: output o = j + r NSL is window sample o; the kept
  // ones (h <= o < h + keep) go to z, their in-frame power is summed, and
  // the 4th powers of the even in-frame samples are placed as the input of
  // the N/2-point periodogram transform (slot (n - e0)/2)
  float2* zp = d.z + (long long)pol * d.zlen + (a - fa.s0);
  const long long lo_n = max(a, fa.f0), hi_n = min(a + keep, fa.f1);
  const long long e0 = lo_n + (lo_n & 1);
  const int cnt = hi_n > e0 ? (int)((hi_n - e0 + 1) / 2) : 0;
  const int off = d.h + (int)(e0 - a);  // window index of sample e0
  const bool inframe = a >= fa.f0 && a + keep <= fa.f1;  // every kept sample is in the frame
  float pw = 0.f;
  {
    float2 v[PERL][RL];
#pragma unroll
    for (int u = 0; u < PERL; ++u) {
      const int j = threadIdx.x + u * NT;
      if ((NSL % NT) == 0 || j < NSL) {
#pragma unroll
        for (int r = 0; r < RL; ++r) v[u][r] = buf[swz(j + r * NSL)];
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PERL; ++u) {
      const int j = threadIdx.x + u * NT;
      if ((NSL % NT) == 0 || j < NSL) {
        pass_butterfly<N, RL, NSL, true, TP>(v[u], j, tw_s, 1, tp_s);
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int o = j + r * NSL;
          const float2 x = v[u][r];
          if (o >= d.h && o < d.h + keep) {
            zp[o - d.h] = x;
            const float p2 = fmaf(x.x, x.x, x.y * x.y);  // the same rounding on both paths
            if (inframe) {
              pw += p2;
            } else {
              const long long n = a + (o - d.h);
              if (n >= fa.f0 && n < fa.f1) pw += p2;
            }
            const int q = o - off;
            if (q >= 0 && (q & 1) == 0 && (q >> 1) < cnt) {
              const float2 x2 = make_float2(x.x * x.x - x.y * x.y, 2.f * x.x * x.y);
              buf[swz(q >> 1)] = make_float2(x2.x * x2.x - x2.y * x2.y, 2.f * x2.x * x2.y);
            }
          }
        }
      }
    }
  }
  // zero padding of the periodogram input (slots no output was placed in)
  for (int i = cnt + threadIdx.x; i < N / 2; i += NT) buf[swz(i)] = make_float2(0.f, 0.f);
  pw = block_sum<NT>(pw, scratch);  // ends with a barrier
  if (threadIdx.x == 0) atomicAdd(&d.acc[fa.acc_slot].P, (double)pw);
  if (cnt == 0) return;

  // N/2-point transform of the 4th powers; |.|^2 of its last pass is added
  // to the frame's periodogram (Welch sum over blocks and polarisations)
  constexpr int N2 = N / 2;
  constexpr int NSL2 = last_ns<N2>();
  constexpr int RL2 = N2 / NSL2;
  constexpr int PERL2 = (NSL2 + NT - 1) / NT;
  fft_passes<N2, NT, 1, NSL2, false, TP>(buf, tw_s, 2, tp_s);
  double* psd = d.psd + (long long)fa.acc_slot * N2;
  {
    float2 v[PERL2][RL2];
#pragma unroll
    for (int u = 0; u < PERL2; ++u) {
      const int j = threadIdx.x + u * NT;
      if ((NSL2 % NT) == 0 || j < NSL2) {
#pragma unroll
        for (int r = 0; r < RL2; ++r) v[u][r] = buf[swz(j + r * NSL2)];
      }
    }
#pragma unroll
    for (int u = 0; u < PERL2; ++u) {
      const int j = threadIdx.x + u * NT;
      if ((NSL2 % NT) == 0 || j < NSL2) {
        pass_butterfly<N2, RL2, NSL2, false, TP>(v[u], j, tw_s, 2, tp_s);
#pragma unroll
        for (int r = 0; r < RL2; ++r)
          atomicAdd(&psd[j + r * NSL2], (double)(v[u][r].x * v[u][r].x + v[u][r].y * v[u][r].y));
      }
    }
  }
}

template <int N, int NT, int STOR>
__global__ void __launch_bounds__(NT) cd_ols_kernel(RxDev d, FrameArgs fa) {
  cd_ols_body<N, NT, STOR>(d, fa, own_block());
}

// Batched: pass 0 runs the timing-acquisition pass (fe), pass 1 the frame.
template <int N, int NT, int STOR>
__global__ void __launch_bounds__(NT) cd_ols_batch_kernel(BView v, int pass) {
  int fi;
  VBlock vb;
  if (!batch_block(v, fi, vb)) return;
  const BFrame& f = v.frames[fi];
  cd_ols_body<N, NT, STOR>(f.d, pass ? f.fa : f.fe, vb);
}

// ---- 32768-point overlap-save on a cluster of two CTAs -------------------
//
// The 32768-point complex array (256 KB) is larger than one CTA's shared
// memory, so each OLS block is a cluster of two CTAs holding half of the
// transform each, joined by distributed shared memory.  Radix-2 splits at
// both ends make the halves independent 16384-point transforms:
//   forward (decimation in frequency): CTA 0 transforms u[i] = x[i] +
//   x[i + N/2], giving the even bins X[2k]; CTA 1 transforms
//   v[i] = (x[i] - x[i + N/2]) W_N^i, giving the odd bins X[2k + 1] (each
//   CTA reads both halves of the window from the ring);
//   filter, Godard sum: bin pairs (k, k + N/2) have equal parity, so each
//   CTA sums over its own bins;
//   inverse: CTA 0 holds E = IDFT_{N/2}(even bins), CTA 1 O = IDFT_{N/2}(odd
//   bins), and z[n] = E[n mod N/2] +- W_N^{-n mod N/2} O[n mod N/2] (+ for
//   n < N/2): each CTA forms the kept samples of its half, reading the
//   other half-transform from its peer's shared memory;
//   periodogram (N/2 = 16384 points): both CTAs place the 4th powers in
//   both CTAs' buffers, then split once more (CTA 0 even bins, CTA 1 odd
//   bins of two 8192-point transforms).
// Every cluster barrier is reached by both CTAs on every path (their
// branch conditions depend only on the block and the frame).
constexpr int kCdN2 = 16384;  // half-transform per CTA
constexpr int kCdNT2 = 1024;

template <int STOR>
__device__ __forceinline__ void cd_ols2_body(const RxDev& d, const FrameArgs& fa, VBlock vb) {
  namespace cg = cooperative_groups;
  constexpr int N2 = kCdN2, NT = kCdNT2;
  extern __shared__ float2 buf[];
  __shared__ float scratch[NT / 32];
  __shared__ float2 tw_s[2 * kTwSplit];  // twiddles of the 16384-point half-transforms
  __shared__ float2 tn_s[2 * kTwSplit];  // W_32768^m, m < 16384
  __shared__ float2 tp_s[kTwPass];       // direct pass table
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  float2* peer = cl.map_shared_rank(buf, rank ^ 1);
  for (int i = threadIdx.x; i < 2 * kTwSplit; i += NT) {
    tn_s[i] = d.tw2[i];
    tw_s[i] = d.tw2[2 * kTwSplit + i];
  }
  for (int i = threadIdx.x; i < kTwPass; i += NT) tp_s[i] = d.tw2[4 * kTwSplit + i];
  __syncthreads();
  const int pol = vb.y;
  const long long a = fa.s0 + (long long)(vb.x >> 1) * d.L;
  const long long zlen_f = 2LL * fa.Ff + 2 * d.c;
  const int keep = (int)min((long long)d.L, fa.s0 + zlen_f - a);
  const long long lo = a - d.h;
  const long long rbase = (long long)pol * d.ring_cap;
  long long r0 = lo % d.ring_cap;
  if (r0 < 0) r0 += d.ring_cap;
  // the window lies inside the stream and does not wrap the ring: plain loads
  const bool interior = lo >= 0 && lo + 2 * N2 <= fa.n_valid && r0 + 2 * N2 <= d.ring_cap;
  auto sample = [&](int i) -> float2 {  // window sample i (zero outside the stream)
    if (interior) return load_sample(d.ring, STOR, rbase + r0 + i);
    const long long n = lo + i;
    long long slot = r0 + i;
    if (slot >= d.ring_cap) slot -= d.ring_cap;
    return (n >= 0 && n < fa.n_valid) ? load_sample(d.ring, STOR, rbase + slot) : make_float2(0.f, 0.f);
  };

  // first forward pass (radix 16) of the half-transform, fused with the
  // split: butterfly j takes local samples j + r N2/16
  {
    const int j = threadIdx.x;
    float2 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int i = j + r * (N2 / 16);
      const float2 x0 = sample(i), x1 = sample(i + N2);
      v[r] = rank == 0 ? cadd(x0, x1) : cmul(csub(x0, x1), twiddle(tn_s, i));
    }
    dft<16, false>(v);
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[swz(16 * j + r)] = v[r];
  }
  __syncthreads();
  constexpr int NSL = last_ns<N2>();
  constexpr int RL = N2 / NSL;
  constexpr int PERL = (NSL + NT - 1) / NT;
  fft_passes<N2, NT, 16, NSL, false, true>(buf, tw_s, 1, tp_s);

  // last forward pass, filter (global bin 2k + rank) and Godard sum over
  // the local pairs (k, k + N2/2) = global (k, k + N/2)
  float gr = 0.f, gi = 0.f;
  {
    float2 v[PERL][RL];
#pragma unroll
    for (int u = 0; u < PERL; ++u) {
      const int j = threadIdx.x + u * NT;
      if ((NSL % NT) == 0 || j < NSL) {
#pragma unroll
        for (int r = 0; r < RL; ++r) v[u][r] = buf[swz(j + r * NSL)];
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PERL; ++u) {
      const int j = threadIdx.x + u * NT;
      if ((NSL % NT) == 0 || j < NSL) {
        pass_butterfly<N2, RL, NSL, false, true>(v[u], j, tw_s, 1, tp_s);
#pragma unroll
        for (int r = 0; r < RL; ++r) v[u][r] = cmul(v[u][r], __ldg(&d.Hf[2 * (j + r * NSL) + rank]));
#pragma unroll
        for (int r = 0; r < RL / 2; ++r) {
          const float2 p = cmulc(v[u][r], v[u][r + RL / 2]);
          gr += p.x;
          gi += p.y;
        }
        if (!fa.est_only) {
#pragma unroll
          for (int r = 0; r < RL; ++r) buf[swz(j + r * NSL)] = v[u][r];
        }
      }
    }
  }
  gr = block_sum<NT>(gr, scratch);
  gi = block_sum<NT>(gi, scratch);
  if (threadIdx.x == 0) {
    const float sg = (lo & 1) ? -1.f : 1.f;
    FrameAcc* acc = d.acc + fa.acc_slot;
    atomicAdd(&acc->C[0], (double)(sg * gr));
    atomicAdd(&acc->C[1], (double)(sg * gi));
  }
  if (fa.est_only) return;  // both CTAs: no shared memory of the peer was touched
  fft_passes<N2, NT, 1, NSL, true, true>(buf, tw_s, 1, tp_s);
  {  // last inverse pass: the half-transform E (rank 0) or O (rank 1) stays in place
    float2 v[PERL][RL];
#pragma unroll
    for (int u = 0; u < PERL; ++u) {
      const int j = threadIdx.x + u * NT;
      if ((NSL % NT) == 0 || j < NSL) {
#pragma unroll
        for (int r = 0; r < RL; ++r) v[u][r] = buf[swz(j + r * NSL)];
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PERL; ++u) {
      const int j = threadIdx.x + u * NT;
      if ((NSL % NT) == 0 || j < NSL) {
        pass_butterfly<N2, RL, NSL, true, true>(v[u], j, tw_s, 1, tp_s);
#pragma unroll
        for (int r = 0; r < RL; ++r) buf[swz(j + r * NSL)] = v[u][r];
      }
    }
  }
  cl.sync();  // both half-transforms complete

  // kept samples of this CTA's half: window index n = rank N2 + m
  float2* zp = d.z + (long long)pol * d.zlen + (a - fa.s0);
  const long long lo_n = max(a, fa.f0), hi_n = min(a + keep, fa.f1);
  const long long e0 = lo_n + (lo_n & 1);
  const int cnt = hi_n > e0 ? (int)((hi_n - e0 + 1) / 2) : 0;
  const int off = d.h + (int)(e0 - a);  // window index of sample e0
  constexpr int PM = N2 / NT;
  float pw = 0.f;
#pragma unroll 4
  for (int k = 0; k < PM; ++k) {
    const int m = threadIdx.x + k * NT;
    const int o = rank * N2 + m;
    if (o >= d.h && o < d.h + keep) {
      const float2 own = buf[swz(m)], oth = peer[swz(m)];
      const float2 E = rank ? oth : own, O = rank ? own : oth;
      float2 w = twiddle(tn_s, m);
      w.y = -w.y;  // W_N^{-m}
      const float2 t = cmul(w, O);
      const float2 x = rank ? csub(E, t) : cadd(E, t);
      zp[o - d.h] = x;
      const long long n = a + (o - d.h);
      if (n >= fa.f0 && n < fa.f1) pw += x.x * x.x + x.y * x.y;
    }
  }
  pw = block_sum<NT>(pw, scratch);
  if (threadIdx.x == 0) atomicAdd(&d.acc[fa.acc_slot].P, (double)pw);
  cl.sync();  // the peer has read this CTA's half-transform
  if (cnt == 0) return;  // both CTAs

  // periodogram input in both CTAs' buffers: slots [0, cnt) are written
  // (each by the CTA that owns the sample, into both buffers), the rest are
  // zero; the two sets are disjoint, so the zeroing needs no barrier
  for (int i = cnt + threadIdx.x; i < N2; i += NT) buf[swz(i)] = make_float2(0.f, 0.f);
  // the 4th powers of the even in-frame samples this thread wrote to z
  // (read back from its own stores) go to slot (n - e0) / 2
#pragma unroll 4
  for (int k = 0; k < PM; ++k) {
    const int o = rank * N2 + threadIdx.x + k * NT;
    const int q = o - off;
    if (o >= d.h && o < d.h + keep && q >= 0 && (q & 1) == 0 && (q >> 1) < cnt) {
      const float2 x = zp[o - d.h];
      const float2 x2 = make_float2(x.x * x.x - x.y * x.y, 2.f * x.x * x.y);
      const float2 x4 = make_float2(x2.x * x2.x - x2.y * x2.y, 2.f * x2.x * x2.y);
      buf[swz(q >> 1)] = x4;
      peer[swz(q >> 1)] = x4;
    }
  }
  cl.sync();  // every slot written; no access to the peer's memory after this
  // split of the 16384-point periodogram transform: rank 0 even bins, rank 1 odd
  constexpr int NP = N2 / 2;
#pragma unroll
  for (int k = 0; k < NP / NT; ++k) {
    const int s = threadIdx.x + k * NT;
    const float2 x0 = buf[swz(s)], x1 = buf[swz(s + NP)];
    buf[swz(s)] = rank == 0 ? cadd(x0, x1) : cmul(csub(x0, x1), twiddle(tw_s, s));
  }
  __syncthreads();
  constexpr int NSP = last_ns<NP>();
  constexpr int RP = NP / NSP;
  constexpr int PERP = (NSP + NT - 1) / NT;
  fft_passes<NP, NT, 1, NSP, false, true>(buf, tw_s, 2, tp_s);
  double* psd = d.psd + (long long)fa.acc_slot * (d.N / 2);
  {
    float2 v[PERP][RP];
#pragma unroll
    for (int u = 0; u < PERP; ++u) {
      const int j = threadIdx.x + u * NT;
      if ((NSP % NT) == 0 || j < NSP) {
#pragma unroll
        for (int r = 0; r < RP; ++r) v[u][r] = buf[swz(j + r * NSP)];
      }
    }
#pragma unroll
    for (int u = 0; u < PERP; ++u) {
      const int j = threadIdx.x + u * NT;
      if ((NSP % NT) == 0 || j < NSP) {
        pass_butterfly<NP, RP, NSP, false, true>(v[u], j, tw_s, 2, tp_s);
#pragma unroll
        for (int r = 0; r < RP; ++r)
          atomicAdd(&psd[2 * (j + r * NSP) + rank], (double)(v[u][r].x * v[u][r].x + v[u][r].y * v[u][r].y));
      }
    }
  }
}

// Grid x = 2 x OLS blocks (a cluster per block), y = polarisation.
template <int STOR>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kCdNT2) cd_ols2_kernel(RxDev d, FrameArgs fa) {
  cd_ols2_body<STOR>(d, fa, own_block());
}

// Batched: the launch list gives every frame an even number of blocks, so
// the two CTAs of a cluster always fall on the same frame.
template <int STOR>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kCdNT2) cd_ols2_batch_kernel(BView v, int pass) {
  int fi;
  VBlock vb;
  if (!batch_block(v, fi, vb)) return;  // both CTAs of a cluster (even offsets)
  const BFrame& f = v.frames[fi];
  cd_ols2_body<STOR>(f.d, pass ? f.fa : f.fe, vb);
}

// x reduced to [-pi, pi] in FP64 (x - 2 pi rint(x / 2 pi)).
__device__ __forceinline__ double wrap_pi(double x) {
  constexpr double kTwoPi = 6.283185307179586477, kInvTwoPi = 0.15915494309189533577;
  return fma(-kTwoPi, rint(x * kInvTwoPi), x);
}

// Per-frame estimator, nb blocks of 1024 threads.  Every block recomputes
// the frame's scalars from the FP64 sums (same values in every block) and
// fills its slice of the next H and of the rotation tables; block 0 writes
// the estimator state of the next frame and the trace record.
// mode 0 (timing acquisition of the first frame): tau = -arg(C)/(2 pi Rs).
// mode 1 (after the frame's CD pass): FO from the periodogram (argmax, lowest
//   index on ties; parabola through the logs of the peak and its cyclic
//   neighbours; frames shorter than kFoeMinSyms keep the previous estimate),
//   AGC gain 1/sqrt(mean |z|^2), the frame's rotation tables,
//   tau <- tau + gain_t * residual, theta <- theta + w * 2 F_f.
// Accumulators and estimator state are double-buffered by frame parity:
// frame f reads acc/psd slot fa.acc_slot and state es[f & 1], clears the
// other accumulator slot and writes es[(f + 1) & 1].
__device__ __forceinline__ void est_body(const RxDev& d, const FrameArgs& fa, int mode, VBlock vb) {
  __shared__ long long sv[32];
  __shared__ int si[32];
  __shared__ double sh[4];
  const int tid = threadIdx.x;
  const FrameAcc* acc = d.acc + fa.acc_slot;
  const double* psd = d.psd + (long long)fa.acc_slot * (d.N / 2);
  // FP64 transcendentals run on one thread only (the FP64 pipe is narrow)
  if (tid == 0) {
    const double C_re = acc->C[0], C_im = acc->C[1];
    sh[3] = (C_re == 0.0 && C_im == 0.0) ? 0.0 : -atan2(C_im, C_re) / (2.0 * M_PI * d.Rs);
  }
  __syncthreads();
  const double resid = sh[3];
  double tau_next;
  if (mode == 1) {
    const EstState es = d.es[fa.f & 1];
    const int n2 = d.N / 2;
    // argmax (lowest index on ties) on the bit patterns: the sums are >= 0,
    // and non-negative doubles order like their bits as integers
    long long best = -1;
    int bi = 0;
    for (int k = tid; k < n2; k += 1024) {
      const long long v = __double_as_longlong(psd[k]);
      if (v > best) { best = v; bi = k; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if ((tid & 31) == 0) { sv[tid >> 5] = best; si[tid >> 5] = bi; }
    __syncthreads();
    if (tid < 32) {
      best = sv[tid];
      bi = si[tid];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const long long ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
    }
    if (tid == 0) {
      const double pm = psd[(bi - 1 + n2) % n2], p0 = psd[bi], pp = psd[(bi + 1) % n2];
      double dl = 0.0;
      if (pm > 0.0 && pp > 0.0 && p0 > 0.0) {
        const double lm = log(pm), l0 = log(p0), lp = log(pp);
        const double den = lm - 2.0 * l0 + lp;
        if (den < 0.0) dl = 0.5 * (lm - lp) / den;
      }
      const int ks = bi < n2 / 2 ? bi : bi - n2;
      double dfo = (ks + dl) * (d.Rs / n2) / 4.0;
      // a frame shorter than kFoeMinSyms keeps the previous frame's estimate
      if (fa.f > 0 && fa.Ff < kFoeMinSyms) dfo = es.dfo_prev;
      const double P = acc->P / (2.0 * (double)(fa.f1 - fa.f0));
      const double gain = P > 0.0 ? 1.0 / sqrt(P) : 1.0;
      const double om = 2.0 * M_PI * dfo / d.fs;
      sh[0] = om;
      sh[1] = gain;
      sh[2] = es.tau + (double)d.timing_gain * resid;
      if (vb.x == 0) {
        if (fa.f < kMaxTrace) {
          FrameRec r;
          r.tau = es.tau;
          r.dfo = dfo;
          r.gain = gain;
          r.theta = es.theta;
          d.rec[fa.f] = r;
        }
        EstState nx;
        nx.tau = sh[2];
        nx.theta = wrap_pi(es.theta + om * (double)(fa.f1 - fa.f0));
        nx.dfo_prev = dfo;
        nx.pad = 0.0;
        d.es[(fa.f + 1) & 1] = nx;
      }
    }
    __syncthreads();
    const double om = sh[0], gain = sh[1], theta = es.theta;
    tau_next = sh[2];
    const float omf = (float)om;  // |w l| < 1024 |w|: FP32 phase is exact to ~1e-6 rad
    for (int l = vb.x * 1024 + tid; l < kRotLo; l += vb.nx * 1024) {
      float s, c;
      sincosf(omf * (float)l, &s, &c);
      d.rot_lo[l] = make_float2(c, -s);
    }
    const int nhi = (d.zlen + kRotLo - 1) / kRotLo;
    for (int hh = vb.x * 1024 + tid; hh < nhi; hh += vb.nx * 1024) {
      const double ph = wrap_pi(theta + om * (double)(hh * kRotLo - d.c));
      float s, c;
      sincosf((float)ph, &s, &c);
      d.rot_hi[hh] = make_float2((float)gain * c, -(float)gain * s);
    }
    // clear the other accumulator slot for the next frame's CD pass
    double* psd_n = d.psd + (long long)((fa.f + 1) & 1) * (d.N / 2);
    for (int k = vb.x * 1024 + tid; k < n2; k += vb.nx * 1024) psd_n[k] = 0.0;
    if (vb.x == 0 && tid == 0) {
      FrameAcc* an = d.acc + ((fa.f + 1) & 1);
      an->C[0] = an->C[1] = an->P = 0.0;
    }
  } else {
    tau_next = resid;
    if (vb.x == 0 && tid == 0) {
      EstState nx;
      nx.tau = resid;
      nx.theta = 0.0;
      nx.dfo_prev = 0.0;
      nx.pad = 0.0;
      d.es[0] = nx;
    }
  }
  // exp(+j 2 pi f_k tau) = sincospi(2 (k'/N) fs tau), k' = k or k - N: the
  // scalar fs tau is formed in FP64, the per-bin product (k'/N exact) in FP32
  const float u2 = (float)(2.0 * d.fs * tau_next) / (float)d.N;
  for (int k = vb.x * 1024 + tid; k < d.N; k += vb.nx * 1024) {
    const int kk = k < d.N / 2 ? k : k - d.N;
    float s, c;
    sincospif((float)kk * u2, &s, &c);
    d.Hf[k] = cmul(d.Hs[k], make_float2(c, s));
  }
}

__global__ void __launch_bounds__(1024) est_kernel(RxDev d, FrameArgs fa, int mode) {
  est_body(d, fa, mode, own_block());
}

// Batched: mode 0 on the timing-acquisition pass (fe), mode 1 on the frame.
__global__ void __launch_bounds__(1024) est_batch_kernel(BView v, int mode) {
  int fi;
  VBlock vb;
  if (!batch_block(v, fi, vb)) return;
  const BFrame& f = v.frames[fi];
  est_body(f.d, mode ? f.fa : f.fe, mode, vb);
}

// ---- host-side launchers -------------------------------------------------

template <int N, int NT>
static cudaError_t launch_cd_n(const RxDev& d, const FrameArgs& fa, cudaStream_t s) {
  const long long zlen_f = 2LL * fa.Ff + 2 * d.c;
  const int nblk = (int)((zlen_f + d.L - 1) / d.L);
  const size_t smem = sizeof(float2) * N;
  dim3 grid(nblk, 2);
  if (d.storage == 2) {
    cd_ols_kernel<N, NT, 2><<<grid, NT, smem, s>>>(d, fa);
  } else {
    cd_ols_kernel<N, NT, 1><<<grid, NT, smem, s>>>(d, fa);
  }
  return cudaGetLastError();
}

template <int N, int NT>
static cudaError_t cd_attr_n() {
  const int smem = (int)(sizeof(float2) * N);
  cudaError_t e = cudaFuncSetAttribute(cd_ols_kernel<N, NT, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(cd_ols_kernel<N, NT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(cd_ols_batch_kernel<N, NT, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(cd_ols_batch_kernel<N, NT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

static cudaError_t launch_cd2(const RxDev& d, const FrameArgs& fa, cudaStream_t s) {
  const long long zlen_f = 2LL * fa.Ff + 2 * d.c;
  const int nblk = (int)((zlen_f + d.L - 1) / d.L);
  const size_t smem = sizeof(float2) * kCdN2;
  dim3 grid(2 * nblk, 2);
  if (d.storage == 2) cd_ols2_kernel<2><<<grid, kCdNT2, smem, s>>>(d, fa);
  else cd_ols2_kernel<1><<<grid, kCdNT2, smem, s>>>(d, fa);
  return cudaGetLastError();
}

static cudaError_t cd2_attr() {
  const int smem = (int)(sizeof(float2) * kCdN2);
  cudaError_t e = cudaFuncSetAttribute(cd_ols2_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(cd_ols2_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(cd_ols2_batch_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(cd_ols2_batch_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

// Opt-in to the dynamic shared memory of every FFT size (once per process).
cudaError_t cd_set_attributes() {
  cudaError_t e = cd_attr_n<1024, 256>();
  if (e == cudaSuccess) e = cd_attr_n<2048, 256>();
  if (e == cudaSuccess) e = cd_attr_n<4096, 256>();
  if (e == cudaSuccess) e = cd_attr_n<8192, 512>();
  if (e == cudaSuccess) e = cd_attr_n<16384, 1024>();
  if (e == cudaSuccess) e = cd2_attr();
  return e;
}

cudaError_t launch_cd(const RxDev& d, const FrameArgs& fa, cudaStream_t s) {
  switch (d.N) {
    case 1024: return launch_cd_n<1024, 256>(d, fa, s);
    case 2048: return launch_cd_n<2048, 256>(d, fa, s);
    case 4096: return launch_cd_n<4096, 256>(d, fa, s);
    case 8192: return launch_cd_n<8192, 512>(d, fa, s);
    case 16384: return launch_cd_n<16384, 1024>(d, fa, s);
    case 32768: return launch_cd2(d, fa, s);
    default: return cudaErrorInvalidValue;
  }
}

int est_grid_x(const RxDev& d) { return max(1, min(16, (d.N + 1023) / 1024)); }

cudaError_t launch_est(const RxDev& d, const FrameArgs& fa, int mode, cudaStream_t s) {
  est_kernel<<<est_grid_x(d), 1024, 0, s>>>(d, fa, mode);
  return cudaGetLastError();
}

// ---- batched launchers (grids as above, one row per polarisation) ---------

int cd_grid_x(const RxDev& d, const FrameArgs& fa) {
  const long long zlen_f = 2LL * fa.Ff + 2 * d.c;
  const int nblk = (int)((zlen_f + d.L - 1) / d.L);
  return d.N == 32768 ? 2 * nblk : nblk;  // a cluster of two CTAs per block at N = 32768
}

template <int N, int NT>
static cudaError_t launch_cd_batch_n(const RxDev& d, const BView& v, int blocks, int pass, cudaStream_t s) {
  const size_t smem = sizeof(float2) * N;
  if (d.storage == 2) return launch_k(cd_ols_batch_kernel<N, NT, 2>, blocks, NT, smem, s, v, pass);
  return launch_k(cd_ols_batch_kernel<N, NT, 1>, blocks, NT, smem, s, v, pass);
}

// Every frame of v has d's FFT size and storage type.
cudaError_t launch_cd_batch(const RxDev& d, const BView& v, int blocks, int pass, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  switch (d.N) {
    case 1024: return launch_cd_batch_n<1024, 256>(d, v, blocks, pass, s);
    case 2048: return launch_cd_batch_n<2048, 256>(d, v, blocks, pass, s);
    case 4096: return launch_cd_batch_n<4096, 256>(d, v, blocks, pass, s);
    case 8192: return launch_cd_batch_n<8192, 512>(d, v, blocks, pass, s);
    case 16384: return launch_cd_batch_n<16384, 1024>(d, v, blocks, pass, s);
    case 32768: {
      const size_t smem = sizeof(float2) * kCdN2;
      if (d.storage == 2) return launch_k(cd_ols2_batch_kernel<2>, blocks, kCdNT2, smem, s, v, pass);
      return launch_k(cd_ols2_batch_kernel<1>, blocks, kCdNT2, smem, s, v, pass);
    }
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_est_batch(const BView& v, int blocks, int mode, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  return launch_k(est_batch_kernel, blocks, 1024, 0, s, v, mode);
}

}  // namespace rx
