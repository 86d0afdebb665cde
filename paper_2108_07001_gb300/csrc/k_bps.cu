// a6 blind phase search, a7 decisions and Gray demapping (paper Sec. II:
// the equaliser's decisions are demapped and transferred to memory).
//
// BPS: phi_b = (b/B - 1/2) pi/2; D_{k,b} = sum_{|i|<=W} d(y_{k+i} e^{-j phi_b})
// with d the squared distance to the nearest constellation point (symbols
// outside the stream contribute nothing); b_k = argmin_b D_{k,b}.
// Unwrap: m_k = m_{k-1} + round((phi_{k-1} - phi_k)/(pi/2)), computed in
// integers as floor((2 (b_{k-1} - b_k) + B) / 2B); the decision is
// dec(y_k e^{-j(phi_b + m pi/2)}) = dec(y_k e^{-j phi_b}) (-j)^m.
//
// Kernel layout: lane = test angle, a group of B/32 warps slides a
// (2W+1)-symbol window along a run of kRun symbols of one polarisation,
// keeping the last 2W+1 metrics in registers (the loop is unrolled by 2W+1
// so the ring index is static).  After every 2W+1 steps the group has
// written the window sums of those steps to shared memory as
// order-preserving keys (float bits with the low 6 bits replaced by the
// angle) and reduces each symbol's B keys with an integer min.  Runs that
// touch no stream edge take an unpredicated path.  The last block of each
// polarisation (found with an atomic counter after a fence; nothing waits)
// turns the runs' unwrap sums into each run's starting counter.  The metric is the squared
// distance in scaled units where the levels are odd integers: QPSK
// (x sqrt2, levels +-1): per dimension |u| - 1; 16QAM (x sqrt10, levels
// +-1, +-3): ||u| - 2| - 1.  Keeping the (small) distance itself, rather
// than an equivalent large correlation, keeps the key's 17-bit resolution
// relative to the quantity being minimised.
#include "rx_internal.cuh"

namespace rx {

template <int B>
__device__ __forceinline__ void group_sync(int g) {
  if constexpr (B == 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(B) : "memory");
  }
}

__device__ __forceinline__ int unwrap_inc(int a, int b, int B) {  // floor((2(a-b)+B)/(2B))
  const int x = 2 * (a - b) + B;
  return (x >= 2 * B) - (x < 0);
}

template <int B, int W, bool QAM16, bool EDGE>
__device__ __forceinline__ void bps_window_step(const float2* __restrict__ yb, int u, int s, int sv_lo, int sv_hi,
                                                float c_s, float s_s, float& D, float& ring_u) {
  float m = 0.f;
  if (!EDGE || (s >= sv_lo && s < sv_hi)) {
    const float2 yv = yb[u];
    const float zx = fmaf(yv.x, c_s, yv.y * s_s);
    const float zy = fmaf(yv.y, c_s, -yv.x * s_s);
    float ex, ey;
    if (QAM16) {
      ex = fabsf(fabsf(zx) - 2.f) - 1.f;
      ey = fabsf(fabsf(zy) - 2.f) - 1.f;
    } else {
      ex = fabsf(zx) - 1.f;
      ey = fabsf(zy) - 1.f;
    }
    m = fmaf(ex, ex, ey * ey);
  }
  D += m;
  D -= ring_u;
  ring_u = m;
}

// One block = 8 warps = 256/B runs of kRun symbols of one polarisation.
template <int B, int W, bool QAM16>
__global__ void __launch_bounds__(256) bps_kernel(RxDev d, FrameArgs fa) {
  constexpr int HALVES = B / 32;         // warps per group
  constexpr int GROUPS = 8 / HALVES;     // runs per block
  constexpr int WIN = 2 * W + 1;
  constexpr int ROW = B + 4;             // padded key row (words)
  extern __shared__ __align__(16) uint32_t keys_smem[];  // [GROUPS][WIN][ROW]
  __shared__ int bh_s[GROUPS][WIN];
  __shared__ float2 cs_s[B];
  __shared__ float red_s[8][3];
  __shared__ int part[256];
  __shared__ int am_last;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = warp / HALVES, wg = warp % HALVES;
  const int tg = wg * 32 + lane;  // thread index within the group
  const int pol = blockIdx.y;
  const long long n_dec = fa.k_b - fa.k_a;
  const int nruns = (int)((n_dec + kRun - 1) / kRun);
  const int run = blockIdx.x * GROUPS + g;
  const long long kr = fa.k_a + (long long)run * kRun;
  const int ract = run < nruns ? (int)min((long long)kRun, fa.k_b - kr) : 0;

  if (threadIdx.x < B) {
    float sb, cb;
    sincospif(((float)threadIdx.x / (float)B - 0.5f) * 0.5f, &sb, &cb);
    cs_s[threadIdx.x] = make_float2(cb, sb);
  }
  const int b = tg;  // this lane's test angle
  float cs, sn;
  sincospif(((float)b / (float)B - 0.5f) * 0.5f, &sn, &cs);
  const float sc = QAM16 ? 3.16227766016837933f : 1.41421356237309505f;
  const float c_s = cs * sc, s_s = sn * sc;

  // y of the frame with its history: symbol i is yf[i - fbase] for i >= fbase - kYHist
  const long long fbase = fa.f * (long long)d.F;
  const float2* yf = d.y + ((long long)(fa.f & 1) * 2 + pol) * (kYHist + d.F) + kYHist;
  const long long ylim = min(fa.n_sym, fbase + fa.Ff);  // symbols beyond do not exist (yet)
  // window step s reads symbol kr - W + s; valid steps [sv_lo, sv_hi)
  const int total = ract + 2 * W;
  const float2* yrun = yf + (kr - W - fbase);
  const int sv_lo = (int)max(0LL, (long long)W - kr);
  const int sv_hi = (int)min((long long)total, ylim - (kr - W));
  const bool edge = sv_lo > 0 || sv_hi < total;
  __syncthreads();  // cs_s

  float ring[WIN];
#pragma unroll
  for (int u = 0; u < WIN; ++u) ring[u] = 0.f;
  float D = 0.f;
  float evn = 0.f, evd = 0.f;
  int inc_sum = 0;
  int bh_prev = -1, bh_first = -1;
  uint16_t* blp = d.bl + (long long)pol * (d.F + 2 * d.W);
  uint32_t* krow = keys_smem + (g * WIN) * ROW + b;
  for (int base = 0; base < total; base += WIN) {
    const float2* yb = yrun + base;
    if (!edge && base + WIN <= total) {
#pragma unroll
      for (int u = 0; u < WIN; ++u) {
        bps_window_step<B, W, QAM16, false>(yb, u, base + u, sv_lo, sv_hi, c_s, s_s, D, ring[u]);
        krow[u * ROW] = (__float_as_uint(fmaxf(D, 0.f)) & ~63u) | (uint32_t)b;
      }
    } else {
#pragma unroll
      for (int u = 0; u < WIN; ++u) {
        if (base + u < total) {
          bps_window_step<B, W, QAM16, true>(yb, u, base + u, sv_lo, sv_hi, c_s, s_s, D, ring[u]);
          krow[u * ROW] = (__float_as_uint(fmaxf(D, 0.f)) & ~63u) | (uint32_t)b;
        }
      }
    }
    // outputs of this super-step: steps s in [max(base, 2W), min(base + WIN, total))
    const int s_lo = max(base, 2 * W), s_hi = min(base + WIN, total);
    if (s_hi > s_lo) {
      group_sync<B>(g);
      const int half = tg % HALVES;
      for (int s = s_lo + tg / HALVES; s < s_lo + 32 * ((s_hi - s_lo + 31) / 32); s += 32) {
        const int u = s - base;
        const bool act = s < s_hi;
        uint32_t best = 0xffffffffu;
        if (act) {
          const uint4* row = reinterpret_cast<const uint4*>(keys_smem + (g * WIN + u) * ROW + half * 32);
#pragma unroll
          for (int c4 = 0; c4 < 8; ++c4) {
            const uint4 v = row[c4];
            best = min(best, min(min(v.x, v.y), min(v.z, v.w)));
          }
        }
        if (HALVES == 2) best = min(best, __shfl_xor_sync(0xffffffffu, best, 1));
        if (act && half == 0) bh_s[g][u] = (int)(best & 63u);
      }
      group_sync<B>(g);
      // decisions, unwrap increments and EVM of the super-step's outputs
      for (int s = s_lo + tg; s < s_hi; s += B) {
        const int u = s - base;
        const int ko = s - 2 * W;  // output index in the run
        const long long k = kr + ko;
        const int bh = bh_s[g][u];
        const int bprev = (s == s_lo) ? (s == 2 * W ? -1 : bh_prev) : bh_s[g][u - 1];
        if (bprev >= 0) inc_sum += unwrap_inc(bprev, bh, B);
        const float2 yv = yrun[W + ko];
        const float2 csb = cs_s[bh];
        const float zx = fmaf(yv.x, csb.x, yv.y * csb.y), zy = fmaf(yv.y, csb.x, -yv.x * csb.y);
        const int lI = level_of(zx, d.nl), lQ = level_of(zy, d.nl);
        blp[k - fa.k_a] = (uint16_t)(bh | (lI << 8) | (lQ << 12));
        if (k >= d.ber_skip && k < fa.k_end) {
          const float dx = level_val(lI, d.nl), dy = level_val(lQ, d.nl);
          evn += (zx - dx) * (zx - dx) + (zy - dy) * (zy - dy);
          evd += dx * dx + dy * dy;
        }
      }
      if (s_lo == 2 * W) bh_first = bh_s[g][s_lo - base];
      bh_prev = bh_s[g][s_hi - 1 - base];
    }
  }
  // run results: internal unwrap sum, first and last angle
  const float incf = warp_sum((float)inc_sum);
  evn = warp_sum(evn);
  evd = warp_sum(evd);
  if (lane == 0) {
    red_s[warp][0] = incf;
    red_s[warp][1] = evn;
    red_s[warp][2] = evd;
  }
  __syncthreads();
  const int stride = d.F / kRun + 4;
  if (threadIdx.x < GROUPS) {
    const int gg = threadIdx.x;
    const int rr = blockIdx.x * GROUPS + gg;
    if (rr < nruns) {
      float si = 0.f;
      for (int w = 0; w < HALVES; ++w) si += red_s[gg * HALVES + w][0];
      d.run_int[pol * stride + rr] = (int)lrintf(si);
    }
  }
  if (tg == 0 && run < nruns) {
    d.run_edge[(pol * stride + run) * 2 + 0] = bh_first;
    d.run_edge[(pol * stride + run) * 2 + 1] = bh_prev;
  }
  if (threadIdx.x == 0) {
    float a = 0.f, c = 0.f;
    for (int w = 0; w < 8; ++w) { a += red_s[w][1]; c += red_s[w][2]; }
    if (c > 0.f) {
      atomicAdd(&d.st->evm_num, (double)a);
      atomicAdd(&d.st->evm_den, (double)c);
    }
  }
  // the last block of this polarisation turns run sums into run start counters
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = atomicAdd(&d.bps_done[pol], 1u) == gridDim.x - 1;
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  const int per = (nruns + 255) / 256;
  const int r0 = threadIdx.x * per, r1 = min(r0 + per, nruns);
  const int b_last_prev = d.st->bhat_last[pol];
  int loc = 0;
  for (int r = r0; r < r1; ++r) {
    const int bf = __ldcg(&d.run_edge[(pol * stride + r) * 2 + 0]);
    const int bp = r == 0 ? b_last_prev : __ldcg(&d.run_edge[(pol * stride + r - 1) * 2 + 1]);
    loc += (bp >= 0 ? unwrap_inc(bp, bf, B) : 0) + __ldcg(&d.run_int[pol * stride + r]);
  }
  part[threadIdx.x] = loc;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  const int m_last = d.st->m_last[pol];
  int acc = m_last + (threadIdx.x > 0 ? part[threadIdx.x - 1] : 0);
  for (int r = r0; r < r1; ++r) {
    const int bf = __ldcg(&d.run_edge[(pol * stride + r) * 2 + 0]);
    const int bp = r == 0 ? b_last_prev : __ldcg(&d.run_edge[(pol * stride + r - 1) * 2 + 1]);
    const int binc = bp >= 0 ? unwrap_inc(bp, bf, B) : 0;
    d.run_m0[pol * stride + r] = acc + binc;
    acc += binc + __ldcg(&d.run_int[pol * stride + r]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    d.st->m_last[pol] = m_last + part[255];
    d.st->bhat_last[pol] = __ldcg(&d.run_edge[(pol * stride + nruns - 1) * 2 + 1]);
    d.bps_done[pol] = 0;
  }
}

// Quadrant rotation by -m (multiply by (-j)^m): (lI, lQ) -> (lQ, nl-1-lI).
__device__ __forceinline__ void rot_minus(int& lI, int& lQ, int m, int nl) {
  const int q = ((m % 4) + 4) % 4;
  for (int i = 0; i < q; ++i) {
    const int t = lI;
    lI = lQ;
    lQ = nl - 1 - t;
  }
}

__device__ __forceinline__ uint32_t gray_bits(int l, int nl) {  // MSB first
  return nl == 2 ? (uint32_t)(1 - l) : (uint32_t)(l ^ (l >> 1));
}

// Demap: one block per run, thread t handles symbols k_r + 2t, k_r + 2t + 1
// of both polarisations.  Writes the output bits, the decision ring and
// the inspection history.
__global__ void __launch_bounds__(128) demap_kernel(RxDev d, FrameArgs fa) {
  __shared__ int sc[2][128];
  const int r = blockIdx.x;
  const long long kr = fa.k_a + (long long)r * kRun;
  const int t = threadIdx.x;
  const int stride = d.F / kRun + 4;
  const int B = d.B;
  const long long n_dec = fa.k_b - fa.k_a;
  int lev[2][2], mm[2][2], bh[2][2];
  bool val[2];
  for (int j = 0; j < 2; ++j) val[j] = (kr + 2 * t + j) < fa.k_b;
  for (int pol = 0; pol < 2; ++pol) {
    const uint16_t* blp = d.bl + (long long)pol * (d.F + 2 * d.W);
    const long long i0 = kr - fa.k_a + 2 * t;
    int c0 = 0, c1 = 0;
    int v0 = val[0] ? blp[i0] : 0, v1 = val[1] ? blp[i0 + 1] : 0;
    bh[pol][0] = v0 & 63;
    bh[pol][1] = v1 & 63;
    lev[pol][0] = v0 >> 8;
    lev[pol][1] = v1 >> 8;
    if (val[0] && t > 0) c0 = unwrap_inc(blp[i0 - 1] & 63, bh[pol][0], B);
    if (val[1]) c1 = unwrap_inc(bh[pol][0], bh[pol][1], B);
    sc[pol][t] = c0 + c1;
    mm[pol][0] = c0;
    mm[pol][1] = c0 + c1;
  }
  __syncthreads();
  for (int o = 1; o < 128; o <<= 1) {
    int a0 = t >= o ? sc[0][t - o] : 0, a1 = t >= o ? sc[1][t - o] : 0;
    __syncthreads();
    sc[0][t] += a0;
    sc[1][t] += a1;
    __syncthreads();
  }
  const int nl = d.nl, hb = d.bps / 2;
  uint32_t bits = 0;
  int nbits = 0;
  uint8_t decb[2] = {0, 0};
  for (int j = 0; j < 2; ++j) {
    const long long k = kr + 2 * t + j;
    for (int pol = 0; pol < 2; ++pol) {
      const int excl = t > 0 ? sc[pol][t - 1] : 0;
      const int m = d.run_m0[pol * stride + r] + excl + mm[pol][j];
      int lI = lev[pol][j] & 15, lQ = lev[pol][j] >> 4;
      rot_minus(lI, lQ, m, nl);
      bits = (bits << hb) | gray_bits(lI, nl);
      bits = (bits << hb) | gray_bits(lQ, nl);
      nbits += 2 * hb;
      decb[j] |= (uint8_t)((lI | (lQ << 2)) << (4 * pol));
      if (val[j] && d.hist_syms > 0 && k < d.hist_syms) {
        d.hist_bhat[(long long)pol * d.hist_syms + k] = (uint8_t)bh[pol][j];
        d.hist_m[(long long)pol * d.hist_syms + k] = m;
      }
    }
  }
  // output bits: 2*bps bits per symbol, symbol k starts at bit 2*bps*k
  const int sb = 2 * d.bps;  // bits per symbol
  for (int j = 0; j < 2; ++j) {
    const long long k = kr + 2 * t + j;
    if (!val[j]) continue;
    d.dec[k % d.dec_cap] = decb[j];
    const uint32_t symbits = (bits >> ((1 - j) * sb)) & ((1u << sb) - 1u);
    const long long bitpos = k * sb;
    if (sb == 8) {
      d.out[(bitpos >> 3) % d.out_cap_bytes] = (uint8_t)symbits;
    } else {  // 4 bits: high nibble for even symbols
      const long long byte = (bitpos >> 3) % d.out_cap_bytes;
      if ((k & 1) == 0) {
        uint8_t v = (uint8_t)(symbits << 4);
        if (val[1] && j == 0) v |= (uint8_t)((bits) & 15u);
        d.out[byte] = v;
      }
    }
  }
  (void)n_dec;
}

// ---- launchers ------------------------------------------------------------

template <int B, int W, bool Q>
static void launch_bps_t(const RxDev& d, const FrameArgs& fa, cudaStream_t s) {
  constexpr int GROUPS = 8 / (B / 32);
  const long long n_dec = fa.k_b - fa.k_a;
  const int nruns = (int)((n_dec + kRun - 1) / kRun);
  dim3 grid((nruns + GROUPS - 1) / GROUPS, 2);
  const size_t smem = sizeof(uint32_t) * GROUPS * (2 * W + 1) * (B + 4);
  bps_kernel<B, W, Q><<<grid, 256, smem, s>>>(d, fa);
}

template <int B, int W>
static cudaError_t bps_attr_t() {
  constexpr int GROUPS = 8 / (B / 32);
  const int smem = (int)(sizeof(uint32_t) * GROUPS * (2 * W + 1) * (B + 4));
  cudaError_t e = cudaFuncSetAttribute(bps_kernel<B, W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(bps_kernel<B, W, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

// Opt-in to the dynamic shared memory of every instantiation (once per process).
cudaError_t bps_set_attributes() {
  cudaError_t e = cudaSuccess;
#define RX_BA(b, w) if (e == cudaSuccess) e = bps_attr_t<b, w>();
  RX_BA(64, 16) RX_BA(32, 16) RX_BA(64, 32) RX_BA(32, 32) RX_BA(64, 8) RX_BA(32, 8)
  RX_BA(64, 12) RX_BA(32, 12) RX_BA(64, 24) RX_BA(32, 24)
#undef RX_BA
  return e;
}

cudaError_t launch_bps(const RxDev& d, const FrameArgs& fa, cudaStream_t s) {
  if (fa.k_b <= fa.k_a) return cudaSuccess;
  const bool q16 = d.bps == 4;
#define RX_BW(b, w)                                   \
  if (d.B == b && d.W == w) {                         \
    if (q16) launch_bps_t<b, w, true>(d, fa, s);      \
    else launch_bps_t<b, w, false>(d, fa, s);         \
    return cudaGetLastError();                        \
  }
  RX_BW(64, 16) RX_BW(32, 16) RX_BW(64, 32) RX_BW(32, 32) RX_BW(64, 8) RX_BW(32, 8)
  RX_BW(64, 12) RX_BW(32, 12) RX_BW(64, 24) RX_BW(32, 24)
#undef RX_BW
  return cudaErrorInvalidValue;
}

cudaError_t launch_unwrap_demap(const RxDev& d, const FrameArgs& fa, cudaStream_t s) {
  if (fa.k_b <= fa.k_a) return cudaSuccess;
  const long long n_dec = fa.k_b - fa.k_a;
  const int nruns = (int)((n_dec + kRun - 1) / kRun);
  demap_kernel<<<nruns, 128, 0, s>>>(d, fa);
  return cudaGetLastError();
}

}  // namespace rx
