// Parts shared by the blind-phase-search kernels (full search in k_bps.cu,
// two-stage search in k_bps2.cu): the unwrap increment, the per-run
// decisions / unwrap sums / EVM sums, the block epilogue, and the unwrap
// scan that turns the runs' unwrap sums into run start counters (paper
// Sec. II: the carrier phase is followed across the whole stream, so the
// pi/2 branch of every symbol depends on all before it).
#pragma once

#include "rx_internal.cuh"

namespace rx {

__device__ __forceinline__ int unwrap_inc(int a, int b, int B) {  // floor((2(a-b)+B)/(2B))
  const int x = 2 * (a - b) + B;
  return (x >= 2 * B) - (x < 0);
}

// One run of ract symbols starting at symbol kr, all 32 lanes of a warp:
// the decision of every symbol at its angle bh[ko] (cs_s: cos/sin of the B
// angles), its packed label in d.bl, the unwrap increments inside the run
// and the EVM sums over the counted symbols.  yat(ko) returns symbol
// kr + ko.  Lane 0 writes the run's unwrap sum and edge angles; evn / evd
// receive the warp's EVM sums (every lane).
template <class YAt>
__device__ __forceinline__ void bps_finish_run(const RxDev& d, const FrameArgs& fa, int pol, int run, int nruns,
                                               long long kr, int ract, const uint8_t* bh, const float2* cs_s,
                                               YAt yat, float& evn, float& evd) {
  const int lane = threadIdx.x & 31;
  float en = 0.f, ed = 0.f;
  int inc_sum = 0;
  uint16_t* blp = d.bl + (long long)pol * (d.F + 2 * d.W);
  for (int ko = lane; ko < ract; ko += 32) {
    const int b = bh[ko];
    if (ko > 0) inc_sum += unwrap_inc(bh[ko - 1], b, d.B);
    const float2 yv = yat(ko);
    const float2 csb = cs_s[b];
    const float zx = fmaf(yv.x, csb.x, yv.y * csb.y), zy = fmaf(yv.y, csb.x, -yv.x * csb.y);
    const int lI = level_of(zx, d.nl), lQ = level_of(zy, d.nl);
    const long long k = kr + ko;
    blp[k - fa.k_a] = (uint16_t)(b | (lI << 8) | (lQ << 12));
    if (k >= d.ber_skip && k < fa.k_end) {
      const float dx = level_val(lI, d.nl), dy = level_val(lQ, d.nl);
      en += (zx - dx) * (zx - dx) + (zy - dy) * (zy - dy);
      ed += dx * dx + dy * dy;
    }
  }
  const float incf = warp_sum((float)inc_sum);
  evn = warp_sum(en);
  evd = warp_sum(ed);
  const int stride = d.F / kRun + 4;
  if (lane == 0 && run < nruns) {
    d.run_int[pol * stride + run] = (int)lrintf(incf);
    d.run_edge[(pol * stride + run) * 2 + 0] = bh[0];
    d.run_edge[(pol * stride + run) * 2 + 1] = bh[ract - 1];
  }
}

// Block epilogue (every thread of the block, at most NT threads, calls it
// after its warps' bps_finish_run calls): the block's EVM sums go to the
// statistics.  evn / evd: the calling warp's sums (read on lane 0).
template <int NT>
__device__ __forceinline__ void bps_finish_block(const RxDev& d, float evn, float evd) {
  __shared__ float red_s[NT / 32][2];
  const int NW = (int)(blockDim.x >> 5);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red_s[warp][0] = evn;
    red_s[warp][1] = evd;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f, c = 0.f;
    for (int w = 0; w < NW; ++w) {
      a += red_s[w][0];
      c += red_s[w][1];
    }
    if (c > 0.f) {
      atomicAdd(&d.st->evm_num, (double)a);
      atomicAdd(&d.st->evm_den, (double)c);
    }
  }
}

// Unwrap scan of one polarisation's frame (one NT-thread block, after the
// BPS of the frame and after the previous frame's scan, in stream order):
// the runs' unwrap sums become each run's starting counter, and the last
// angle and counter carry to the next frame.  Kept out of the BPS kernel,
// so the BPS of consecutive frames depend on nothing of each other.
template <int NT>
__device__ __forceinline__ void unwrap_scan_body(const RxDev& d, const FrameArgs& fa, int pol) {
  __shared__ int part[NT];
  const long long n_dec = fa.k_b - fa.k_a;
  const int nruns = (int)((n_dec + kRun - 1) / kRun);
  if (nruns <= 0) return;
  const int stride = d.F / kRun + 4;
  const int per = (nruns + NT - 1) / NT;
  const int r0 = threadIdx.x * per, r1 = min(r0 + per, nruns);
  const int b_last_prev = d.st->bhat_last[pol];
  int loc = 0;
  for (int r = r0; r < r1; ++r) {
    const int bf = d.run_edge[(pol * stride + r) * 2 + 0];
    const int bp = r == 0 ? b_last_prev : d.run_edge[(pol * stride + r - 1) * 2 + 1];
    loc += (bp >= 0 ? unwrap_inc(bp, bf, d.B) : 0) + d.run_int[pol * stride + r];
  }
  part[threadIdx.x] = loc;
  __syncthreads();
  for (int o = 1; o < NT; o <<= 1) {
    const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  const int m_last = d.st->m_last[pol];
  int acc = m_last + (threadIdx.x > 0 ? part[threadIdx.x - 1] : 0);
  for (int r = r0; r < r1; ++r) {
    const int bf = d.run_edge[(pol * stride + r) * 2 + 0];
    const int bp = r == 0 ? b_last_prev : d.run_edge[(pol * stride + r - 1) * 2 + 1];
    const int binc = bp >= 0 ? unwrap_inc(bp, bf, d.B) : 0;
    d.run_m0[pol * stride + r] = acc + binc;
    acc += binc + d.run_int[pol * stride + r];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    d.st->m_last[pol] = m_last + part[NT - 1];
    d.st->bhat_last[pol] = d.run_edge[(pol * stride + nruns - 1) * 2 + 1];
  }
}

}  // namespace rx
