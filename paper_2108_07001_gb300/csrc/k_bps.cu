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
// so the ring index is static).  Every 32 outputs the group writes its
// window sums to shared memory as order-preserving keys
// (float bits with the low 6 bits replaced by the angle code) and reduces
// each symbol's B keys with integer min/max.  For QPSK the metric is the
// equivalent |Re z| + |Im z| (maximised): |z - dec z|^2 = |z|^2 + 1 -
// sqrt2 (|Re z| + |Im z|) and |z|^2 does not depend on b.  For 16QAM,
// in sqrt10-scaled units, the per-dimension distance to the nearest of
// {-3,-1,1,3} is ||u| - 2| - 1.
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

template <int B, int W, bool QAM16>
__global__ void __launch_bounds__(256) bps_kernel(RxDev d, FrameArgs fa) {
  constexpr int HALVES = B / 32;         // warps per group
  constexpr int GROUPS = 8 / HALVES;     // runs per block
  constexpr int NCH = B / 4;             // 16-byte chunks per key row
  constexpr int WIN = 2 * W + 1;
  __shared__ __align__(16) uint32_t keys[GROUPS][32][B];
  __shared__ int bh_s[GROUPS][33];
  __shared__ float red_s[8][3];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = warp / HALVES, wg = warp % HALVES;
  const int pol = blockIdx.y;
  const long long n_dec = fa.k_b - fa.k_a;
  const int run = blockIdx.x * GROUPS + g;
  const long long kr = fa.k_a + (long long)run * kRun;
  const bool active = kr < fa.k_b;
  const int ract = active ? (int)min((long long)kRun, fa.k_b - kr) : 0;

  const int b = wg * 32 + lane;
  float cs, sn;
  sincospif(((float)b / (float)B - 0.5f) * 0.5f, &sn, &cs);
  const float sc = QAM16 ? 3.16227766016837933f : 1.0f;
  const float c_s = cs * sc, s_s = sn * sc;

  const float2* ycur = d.y + (long long)(fa.f & 1) * 2 * d.F + (long long)pol * d.F;
  const float2* yprev = d.y + (long long)((fa.f + 1) & 1) * 2 * d.F + (long long)pol * d.F;
  const long long fbase = fa.f * (long long)d.F;
  const long long ylim = min(fa.n_sym, fbase + fa.Ff);  // symbols beyond do not exist (yet)

  float ring[WIN];
#pragma unroll
  for (int u = 0; u < WIN; ++u) ring[u] = 0.f;
  float D = 0.f;
  float evn = 0.f, evd = 0.f;
  int inc_sum = 0;
  int bh_prev = -1;
  const int total = ract + 2 * W;
  uint16_t* blp = d.bl + (long long)pol * (d.F + 2 * d.W);
  for (int base = 0; base < total; base += WIN) {
#pragma unroll
    for (int u = 0; u < WIN; ++u) {
      const int s = base + u;
      if (s < total) {
        const long long i = kr - W + s;  // symbol entering the window
        float m = 0.f;
        if (i >= 0 && i < ylim) {
          const float2 yv = (i >= fbase) ? ycur[i - fbase] : yprev[i - fbase + d.F];
          const float zx = fmaf(yv.x, c_s, yv.y * s_s);
          const float zy = fmaf(yv.y, c_s, -yv.x * s_s);
          if (QAM16) {
            const float ex = fabsf(fabsf(zx) - 2.f) - 1.f, ey = fabsf(fabsf(zy) - 2.f) - 1.f;
            m = fmaf(ex, ex, ey * ey);
          } else {
            m = fabsf(zx) + fabsf(zy);
          }
        }
        D += m - ring[u];
        ring[u] = m;
        const int o = s - 2 * W;
        if (o >= 0) {
          const int ol = o & 31;
          const uint32_t code = QAM16 ? (uint32_t)b : (uint32_t)(63 - b);
          const uint32_t key = (__float_as_uint(fmaxf(D, 0.f)) & ~63u) | code;
          const int ch = (b >> 2) ^ (ol & (NCH - 1));
          keys[g][ol][ch * 4 + (b & 3)] = key;
          if (ol == 31 || o == ract - 1) {
            group_sync<B>(g);
            // reduce the chunk's outputs: thread t of the group -> output t / HALVES
            const int tg = wg * 32 + lane;
            const int oc = tg / HALVES, half = tg % HALVES;
            const int nout = ol + 1;
            uint32_t best = QAM16 ? 0xffffffffu : 0u;
            if (oc < nout) {
#pragma unroll
              for (int c4 = 0; c4 < 8; ++c4) {
                const int chk = (half * 8 + c4) ^ (oc & (NCH - 1));
                const uint4 v = *reinterpret_cast<const uint4*>(&keys[g][oc][chk * 4]);
                if (QAM16) {
                  best = min(best, min(min(v.x, v.y), min(v.z, v.w)));
                } else {
                  best = max(best, max(max(v.x, v.y), max(v.z, v.w)));
                }
              }
            }
            if (HALVES == 2) {
              const uint32_t ob = __shfl_xor_sync(0xffffffffu, best, 1);
              best = QAM16 ? min(best, ob) : max(best, ob);
            }
            const int bh = QAM16 ? (int)(best & 63u) : 63 - (int)(best & 63u);
            if (half == 0 && oc < nout) bh_s[g][oc + 1] = bh;
            if (tg == 0) bh_s[g][0] = bh_prev;
            group_sync<B>(g);
            if (half == 0 && oc < nout) {
              const long long k = kr + (o - ol) + oc;
              const int bprev = bh_s[g][oc];
              if (bprev >= 0 && k > kr) inc_sum += unwrap_inc(bprev, bh, B);
              // decision at the chosen angle
              const float2 yv = (k >= fbase) ? ycur[k - fbase] : yprev[k - fbase + d.F];
              float sb, cb;
              sincospif(((float)bh / (float)B - 0.5f) * 0.5f, &sb, &cb);
              const float zx = fmaf(yv.x, cb, yv.y * sb), zy = fmaf(yv.y, cb, -yv.x * sb);
              const int lI = level_of(zx, d.nl), lQ = level_of(zy, d.nl);
              blp[k - fa.k_a] = (uint16_t)(bh | (lI << 8) | (lQ << 12));
              if (k >= d.ber_skip && k < fa.k_end) {
                const float dx = level_val(lI, d.nl), dy = level_val(lQ, d.nl);
                evn += (zx - dx) * (zx - dx) + (zy - dy) * (zy - dy);
                evd += dx * dx + dy * dy;
              }
            }
            // carry for the next chunk (read before the next chunk's first
            // barrier, after which bh_s is rewritten)
            bh_prev = bh_s[g][nout];
          }
        }
      }
    }
  }
  // block reduction of the run's unwrap increments and EVM sums
  float incf = (float)inc_sum;
  incf = warp_sum(incf);
  evn = warp_sum(evn);
  evd = warp_sum(evd);
  if (lane == 0) {
    red_s[warp][0] = incf;
    red_s[warp][1] = evn;
    red_s[warp][2] = evd;
  }
  __syncthreads();
  if (threadIdx.x < GROUPS) {
    const int gg = threadIdx.x;
    float si = 0.f;
    for (int w = 0; w < HALVES; ++w) si += red_s[gg * HALVES + w][0];
    const int rr = blockIdx.x * GROUPS + gg;
    const long long krr = fa.k_a + (long long)rr * kRun;
    const int nruns = (int)((n_dec + kRun - 1) / kRun);
    if (krr < fa.k_b && rr < nruns) d.run_int[pol * (d.F / kRun + 4) + rr] = (int)lrintf(si);
  }
  if (threadIdx.x == 0) {
    float a = 0.f, c = 0.f;
    for (int w = 0; w < 8; ++w) { a += red_s[w][1]; c += red_s[w][2]; }
    if (c > 0.f) {
      atomicAdd(&d.st->evm_num, (double)a);
      atomicAdd(&d.st->evm_den, (double)c);
    }
  }
}

// Unwrap counter at the first symbol of every run (one block, per pol):
// m(k_r) = m_last + sum over earlier runs of (boundary inc + internal incs)
// + the run's own boundary increment.
__global__ void __launch_bounds__(1024) unwrap_scan_kernel(RxDev d, FrameArgs fa) {
  __shared__ int part[1024];
  const long long n_dec = fa.k_b - fa.k_a;
  const int nruns = (int)((n_dec + kRun - 1) / kRun);
  const int stride = d.F / kRun + 4;
  const int B = d.B;
  for (int pol = 0; pol < 2; ++pol) {
    const uint16_t* blp = d.bl + (long long)pol * (d.F + 2 * d.W);
    const int per = (nruns + 1023) / 1024;
    const int r0 = threadIdx.x * per;
    int loc = 0;
    for (int r = r0; r < min(r0 + per, nruns); ++r) {
      const int bfirst = blp[(long long)r * kRun] & 63;
      const int bprev = r == 0 ? d.st->bhat_last[pol] : (blp[(long long)r * kRun - 1] & 63);
      const int binc = bprev >= 0 ? unwrap_inc(bprev, bfirst, B) : 0;
      loc += binc + d.run_int[pol * stride + r];
    }
    part[threadIdx.x] = loc;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
      __syncthreads();
      part[threadIdx.x] += v;
      __syncthreads();
    }
    int acc = d.st->m_last[pol] + (threadIdx.x > 0 ? part[threadIdx.x - 1] : 0);
    for (int r = r0; r < min(r0 + per, nruns); ++r) {
      const int bfirst = blp[(long long)r * kRun] & 63;
      const int bprev = r == 0 ? d.st->bhat_last[pol] : (blp[(long long)r * kRun - 1] & 63);
      const int binc = bprev >= 0 ? unwrap_inc(bprev, bfirst, B) : 0;
      d.run_m0[pol * stride + r] = acc + binc;
      acc += binc + d.run_int[pol * stride + r];
    }
    __syncthreads();
    if (threadIdx.x == 1023) {
      d.st->m_last[pol] = d.st->m_last[pol] + part[1023];
      d.st->bhat_last[pol] = blp[n_dec - 1] & 63;
    }
    __syncthreads();
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
  bps_kernel<B, W, Q><<<grid, 256, 0, s>>>(d, fa);
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
  unwrap_scan_kernel<<<1, 1024, 0, s>>>(d, fa);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long n_dec = fa.k_b - fa.k_a;
  const int nruns = (int)((n_dec + kRun - 1) / kRun);
  demap_kernel<<<nruns, 128, 0, s>>>(d, fa);
  return cudaGetLastError();
}

}  // namespace rx
