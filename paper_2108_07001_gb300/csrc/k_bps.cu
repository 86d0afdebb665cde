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
// Kernel layout: one warp per run of kRun symbols of one polarisation;
// lane l holds the test angles l + 32a (B/32 per lane) and slides a
// (2W+1)-symbol window with the last 2W+1 metrics in registers (the loop is
// unrolled by 2W+1 so the ring index is static).  Each step the lane writes
// the smaller of its angles' order-preserving keys (float bits with the
// low 6 bits replaced by the angle) to a shared-memory row; the rows are
// reduced with an integer min once per super-step of 2W+1 steps (QPSK with
// 64 angles derives a lane's second angle from the rotation of its first,
// see bps_kernel).  Runs that touch no
// stream edge take no per-step predicate.  A separate one-block-per-
// polarisation kernel, queued before the demap, turns the runs' unwrap
// sums into each run's starting counter (so the BPS of the next frame
// need not wait for this one).
#include "bps_common.cuh"

namespace rx {

// Metric of one symbol at one test angle (scaled squared distance).
template <bool QAM16>
__device__ __forceinline__ float bps_metric(float2 yv, float c_s, float s_s) {
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
  return fmaf(ex, ex, ey * ey);
}

// Dynamic shared memory of one block: per warp, WIN - 1 + NSUP key rows of
// ROW words, then the staged symbols (float4 {x, y, h, 0} in the paired
// QPSK form, float2 otherwise).
template <int B, int W, bool QAM16>
struct BpsSmem {
  static constexpr bool PAIR = !QAM16 && B == 64;
  static constexpr int WIN = 2 * W + 1;
  static constexpr int ROW = 36;                         // padded key row (words)
  static constexpr int YS = kRun + 2 * W;                // staged symbols per run
  static constexpr int NSUP = (YS + WIN - 1) / WIN;      // super-steps per run
  static constexpr int ROWS = WIN - 1 + NSUP;            // key rows per warp
  static constexpr int YSP = (NSUP * WIN + 7) / 8 * 8;     // staged entries (whole super-steps)
  static constexpr size_t KEY_WARP = sizeof(uint32_t) * ROWS * ROW;  // key rows of one warp
  static constexpr size_t Y_WARP = (size_t)YSP * (PAIR ? 24 : 8);    // staged symbols of one warp
  // a block of nw warps (runs): every warp's key rows, then every warp's symbols
  static constexpr size_t bytes(int nw) { return (size_t)nw * (KEY_WARP + Y_WARP); }
  static constexpr size_t BYTES = bytes(8);  // the largest block (8 runs)
};

// One warp = one run of kRun symbols of one polarisation; lane l holds the
// test angles l + 32 a (a < B/32), each with its own register ring of the
// last 2W+1 metrics.  Per window step the lane packs its angles' window
// sums into keys and keeps the smaller, so a row of 32 keys per output is
// reduced afterwards: rows 0..2W-1 of a super-step of 2W+1 steps are
// reduced at its end (one pass of 32 lanes for W = 16), the last row of
// every super-step goes to a row of its own, reduced once per run.
//
// QPSK with B = 64 (the paired form): angle l + 32 is angle l + pi/4, and
// with z = sc y e^{-j phi_l} (sc = sqrt 2, points at +-1 +-j) the metric
// halves are d_l / 2 = h - (|z_x| + |z_y|) and
// d_{l+32} / 2 = h - sqrt2 max(|z_x|, |z_y|), h = |y|^2 + 1 (|z|^2 = 2|y|^2
// and rotating z by -pi/4 maps |z_x| + |z_y| to sqrt2 max(|z_x|, |z_y|)).
// One rotation then serves both angles of a lane.  h carries a relative
// bias of 2^-17 (common to all angles of a symbol, so the argmin is that of
// d) that keeps every metric positive under rounding; symbols outside the
// stream are staged as y = 0, h = 0 and contribute exactly 0.
template <int B, int W, bool QAM16>
__device__ __forceinline__ void bps_body(const RxDev& d, const FrameArgs& fa, VBlock vb) {
  using SM = BpsSmem<B, W, QAM16>;
  constexpr bool PAIR = SM::PAIR;
  constexpr int APL = B / 32;            // angles per lane
  constexpr int WIN = SM::WIN;
  constexpr int ROW = SM::ROW;
  extern __shared__ __align__(16) uint32_t keys_smem[];
  __shared__ uint8_t bh_s[8][kRun];
  __shared__ float2 cs_s[B];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pol = vb.y;
  const long long n_dec = fa.k_b - fa.k_a;
  const int nruns = (int)((n_dec + kRun - 1) / kRun);
  const int nw = (int)(blockDim.x >> 5);  // runs per block (d.bps_nw)
  const int run = vb.x * nw + warp;
  const long long kr = fa.k_a + (long long)run * kRun;
  const int ract = run < nruns ? (int)min((long long)kRun, fa.k_b - kr) : 0;

  if (threadIdx.x < B) {
    float sb, cb;
    sincospif(((float)threadIdx.x / (float)B - 0.5f) * 0.5f, &sb, &cb);
    cs_s[threadIdx.x] = make_float2(cb, sb);
  }
  const float sc = QAM16 ? 3.16227766016837933f : 1.41421356237309505f;
  float c_s[APL], s_s[APL];
#pragma unroll
  for (int a = 0; a < APL; ++a) {
    float cs, sn;
    sincospif(((float)(lane + 32 * a) / (float)B - 0.5f) * 0.5f, &sn, &cs);
    c_s[a] = cs * sc;
    s_s[a] = sn * sc;
  }

  // stage the run's symbols kr - W .. kr + ract + W (zero outside the stream)
  const long long fbase = fa.f * (long long)d.F;
  const float2* yf = d.y + ((long long)(fa.f & 1) * 2 + pol) * (kYHist + d.F) + kYHist;
  const long long ylim = min(fa.n_sym, fbase + fa.Ff);  // symbols beyond do not exist (yet)
  const int total = ract + 2 * W;
  const int sv_lo = (int)max(0LL, (long long)W - kr);
  const int sv_hi = (int)min((long long)total, ylim - (kr - W));
  uint32_t* kw = keys_smem + warp * SM::ROWS * ROW;
  unsigned char* ybase = reinterpret_cast<unsigned char*>(keys_smem) + nw * SM::KEY_WARP;
  float4* ys4 = reinterpret_cast<float4*>(ybase) + warp * SM::YSP;            // paired: {x, y, y, x}
  float2* hs2 = reinterpret_cast<float2*>(ybase + (size_t)nw * SM::YSP * 16) + warp * SM::YSP;  // paired: {h, h}
  float2* ys2 = reinterpret_cast<float2*>(ybase) + warp * SM::YSP;
  // the paired form stages whole super-steps (zeros past the run) and so
  // runs every super-step, the partial last one included, without predicates
  if constexpr (PAIR) {
    // a fixed count per lane: every lane's loads are in flight before the
    // first store
    constexpr int PER = (SM::NSUP * WIN + 31) / 32;
    float2 v[PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int i = lane + 32 * r;
      v[r] = (i < SM::NSUP * WIN && i >= sv_lo && i < sv_hi) ? yf[kr - W - fbase + i] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int i = lane + 32 * r;
      if (i < SM::NSUP * WIN) {
        const bool in = i >= sv_lo && i < sv_hi;
        const float h = in ? fmaf(v[r].x, v[r].x, fmaf(v[r].y, v[r].y, 1.f)) * (1.f + 0x1p-17f) : 0.f;
        ys4[i] = make_float4(v[r].x, v[r].y, v[r].y, v[r].x);
        hs2[i] = make_float2(h, h);
      }
    }
  } else {
    for (int i = lane; i < total; i += 32) {
      const bool in = i >= sv_lo && i < sv_hi;
      ys2[i] = in ? yf[kr - W - fbase + i] : make_float2(0.f, 0.f);
    }
  }
  const bool edge = sv_lo > 0 || sv_hi < total;
  __syncthreads();  // cs_s, staged symbols

  float ring[APL][WIN];
#pragma unroll
  for (int a = 0; a < APL; ++a)
#pragma unroll
    for (int u = 0; u < WIN; ++u) ring[a][u] = 0.f;
  float D[APL];
#pragma unroll
  for (int a = 0; a < APL; ++a) D[a] = 0.f;

  // metrics of the lane's angles for staged symbol i (in == false: zero)
  auto metrics_v = [&](const float4 v, float (&m)[APL]) {
    const float zx = fmaf(v.x, c_s[0], v.y * s_s[0]);
    const float zy = fmaf(v.y, c_s[0], -v.x * s_s[0]);
    const float ax = fabsf(zx), ay = fabsf(zy);
    m[0] = (v.z - ax) - ay;
    m[1] = fmaf(-1.41421356237309505f, fmaxf(ax, ay), v.z);
  };
  auto metrics = [&](int i, bool in, float (&m)[APL]) {
    if constexpr (PAIR) {
      const float4 v = ys4[i];
      const float zx = fmaf(v.x, c_s[0], v.y * s_s[0]);
      const float zy = fmaf(v.y, c_s[0], -v.x * s_s[0]);
      const float ax = fabsf(zx), ay = fabsf(zy);
      m[0] = (v.z - ax) - ay;
      m[1] = fmaf(-1.41421356237309505f, fmaxf(ax, ay), v.z);
    } else {
      const float2 yv = ys2[i];
#pragma unroll
      for (int a = 0; a < APL; ++a) m[a] = in ? bps_metric<QAM16>(yv, c_s[a], s_s[a]) : 0.f;
    }
  };

  // paired form: packed window sums and ring (angle l low, l + 32 high)
  unsigned long long ring2[PAIR ? WIN : 1];
  unsigned long long D2 = 0ull;
#pragma unroll
  for (int u = 0; u < (PAIR ? WIN : 1); ++u) ring2[u] = 0ull;
  const unsigned long long CC2 = f2pk(c_s[0], c_s[0]), SS2 = f2pk(s_s[0], -s_s[0]);
  const unsigned long long NG2 = f2pk(-1.f, -1.41421356237309505f);
  int sup = 0;
  for (int base = 0; base < total; base += WIN, ++sup) {
    if (PAIR || (!edge && base + WIN <= total)) {
      // interior: every step is a real symbol (paired form: or a staged zero);
      // the paired form loads the staged symbols two steps ahead
      if constexpr (PAIR) {
        // packed pairs: (zx, zy) = (x, y) c + (y, x) (s, -s); (g0, g1) =
        // (h, h) + (|zx| + |zy|, max(|zx|, |zy|)) (-1, -sqrt2); D += g - ring
        const ulonglong2* pq_s = reinterpret_cast<const ulonglong2*>(ys4);
        const unsigned long long* hh_s = reinterpret_cast<const unsigned long long*>(hs2);
        ulonglong2 q0 = pq_s[base], q1 = pq_s[base + 1];
        unsigned long long h0 = hh_s[base], h1 = hh_s[base + 1];
#pragma unroll
        for (int u = 0; u < WIN; ++u) {
          const ulonglong2 pq = q0;
          const unsigned long long hh = h0;
          q0 = q1;
          h0 = h1;
          if (u + 2 < WIN) {
            q1 = pq_s[base + u + 2];
            h1 = hh_s[base + u + 2];
          }
          const unsigned long long zz = f2fma(pq.y, SS2, f2mul(pq.x, CC2));
          float zx, zy;
          f2up(zz, zx, zy);
          const float ax = fabsf(zx), ay = fabsf(zy);
          const unsigned long long g = f2fma(f2pk(ax + ay, fmaxf(ax, ay)), NG2, hh);
          D2 = f2add(D2, f2sub(g, ring2[u]));
          ring2[u] = g;
          float d0, d1;
          f2up(D2, d0, d1);
          const uint32_t key = min((__float_as_uint(d0) & ~63u) | (uint32_t)lane,
                                   (__float_as_uint(d1) & ~63u) | (uint32_t)(lane + 32));
          kw[(u < WIN - 1 ? u : WIN - 1 + sup) * ROW + lane] = key;
        }
      } else {
#pragma unroll
        for (int u = 0; u < WIN; ++u) {
          float m[APL];
          metrics(base + u, true, m);
          uint32_t key = 0xffffffffu;
#pragma unroll
          for (int a = 0; a < APL; ++a) {
            D[a] += m[a] - ring[a][u];
            ring[a][u] = m[a];
            key = min(key, (__float_as_uint(D[a]) & ~63u) | (uint32_t)(lane + 32 * a));
          }
          kw[(u < WIN - 1 ? u : WIN - 1 + sup) * ROW + lane] = key;
        }
      }
    } else {
#pragma unroll
      for (int u = 0; u < WIN; ++u) {
        const int s = base + u;
        if (s < total) {
          float m[APL];
          metrics(s, s >= sv_lo && s < sv_hi, m);
          uint32_t key = 0xffffffffu;
#pragma unroll
          for (int a = 0; a < APL; ++a) {
            D[a] += m[a];
            D[a] -= ring[a][u];
            ring[a][u] = m[a];
            key = min(key, (__float_as_uint(fmaxf(D[a], 0.f)) & ~63u) | (uint32_t)(lane + 32 * a));
          }
          kw[(u < WIN - 1 ? u : WIN - 1 + sup) * ROW + lane] = key;
        }
      }
    }
    // reduce rows 0..WIN-2 of the super-step: steps [max(base, 2W), min(base + WIN - 1, total))
    const int s_lo = max(base, 2 * W), s_hi = min(base + WIN - 1, total);
    __syncwarp();
    for (int s = s_lo + lane; s < s_hi; s += 32) {
      const uint4* row = reinterpret_cast<const uint4*>(kw + (s - base) * ROW);
      uint32_t best = 0xffffffffu;
#pragma unroll
      for (int c4 = 0; c4 < 8; ++c4) {
        const uint4 v = row[c4];
        best = min(best, min(min(v.x, v.y), min(v.z, v.w)));
      }
      bh_s[warp][s - 2 * W] = (uint8_t)(best & 63u);
    }
    __syncwarp();
  }
  // the last row of every super-step: step base_t + WIN - 1 of super-step t
  for (int t = lane; t < sup; t += 32) {
    const int s = t * WIN + WIN - 1;
    if (s >= 2 * W && s < total) {
      const uint4* row = reinterpret_cast<const uint4*>(kw + (WIN - 1 + t) * ROW);
      uint32_t best = 0xffffffffu;
#pragma unroll
      for (int c4 = 0; c4 < 8; ++c4) {
        const uint4 v = row[c4];
        best = min(best, min(min(v.x, v.y), min(v.z, v.w)));
      }
      bh_s[warp][s - 2 * W] = (uint8_t)(best & 63u);
    }
  }
  __syncwarp();
  // decisions, unwrap increments and EVM of the run; then the block epilogue
  float evn, evd;
  bps_finish_run(d, fa, pol, run, nruns, kr, ract, bh_s[warp], cs_s,
                 [&](int ko) { return PAIR ? make_float2(ys4[W + ko].x, ys4[W + ko].y) : ys2[W + ko]; }, evn, evd);
  bps_finish_block<256>(d, evn, evd);
}

template <int B, int W, bool QAM16>
__global__ void __launch_bounds__(256, 2) bps_kernel(RxDev d, FrameArgs fa) {
  bps_body<B, W, QAM16>(d, fa, own_block());
}

template <int B, int W, bool QAM16>
__global__ void __launch_bounds__(256, 2) bps_batch_kernel(BView v) {
  int fi;
  VBlock vb;
  if (!batch_block(v, fi, vb)) return;
  const BFrame& f = v.frames[fi];
  bps_body<B, W, QAM16>(f.d, f.fa, vb);
}

// Quadrant rotation by -m (multiply by (-j)^m); one quarter turn maps
// (lI, lQ) -> (lQ, nl-1-lI), so q = m mod 4 turns give the cases below.
__device__ __forceinline__ void rot_minus(int& lI, int& lQ, int m, int nl) {
  const int q = m & 3;  // m mod 4 in [0, 4) for negative m too
  const int a = lI, b = lQ, ra = nl - 1 - lI, rb = nl - 1 - lQ;
  lI = q == 0 ? a : q == 1 ? b : q == 2 ? ra : rb;
  lQ = q == 0 ? b : q == 1 ? ra : q == 2 ? rb : a;
}

__device__ __forceinline__ uint32_t gray_bits(int l, int nl) {  // MSB first
  return nl == 2 ? (uint32_t)(1 - l) : (uint32_t)(l ^ (l >> 1));
}

// Demap: one block per run, thread t handles symbols k_r + 2t, k_r + 2t + 1
// of both polarisations.  Writes the output bits, the decision ring and
// the inspection history.
__device__ __forceinline__ void demap_body(const RxDev& d, const FrameArgs& fa, VBlock vb) {
  __shared__ int wt[2][4];
  const int r = vb.x;
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
    mm[pol][0] = c0;
    mm[pol][1] = c0 + c1;
  }
  // exclusive prefix over the block's threads of c0 + c1 (both polarisations):
  // warp scans, then the warps' totals
  const int lane = t & 31, w = t >> 5;
  int incl[2] = {mm[0][1], mm[1][1]};
#pragma unroll
  for (int pol = 0; pol < 2; ++pol)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int a = __shfl_up_sync(0xffffffffu, incl[pol], o);
      if (lane >= o) incl[pol] += a;
    }
  if (lane == 31) {
    wt[0][w] = incl[0];
    wt[1][w] = incl[1];
  }
  __syncthreads();
  int excl[2];
#pragma unroll
  for (int pol = 0; pol < 2; ++pol) {
    int base = 0;
    for (int ww = 0; ww < w; ++ww) base += wt[pol][ww];
    excl[pol] = base + incl[pol] - mm[pol][1];
  }
  const int nl = d.nl, hb = d.bps / 2;
  uint32_t bits = 0;
  int nbits = 0;
  uint8_t decb[2] = {0, 0};
  for (int j = 0; j < 2; ++j) {
    const long long k = kr + 2 * t + j;
    for (int pol = 0; pol < 2; ++pol) {
      const int m = d.run_m0[pol * stride + r] + excl[pol] + mm[pol][j];
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

__global__ void __launch_bounds__(256) unwrap_scan_kernel(RxDev d, FrameArgs fa) {
  unwrap_scan_body<256>(d, fa, blockIdx.x);
}

// Batched: virtual block x = polarisation of the frame.
__global__ void __launch_bounds__(256) unwrap_scan_batch_kernel(BView v) {
  int fi;
  VBlock vb;
  if (!batch_block(v, fi, vb)) return;
  const BFrame& f = v.frames[fi];
  unwrap_scan_body<256>(f.d, f.fa, vb.x);
}

__global__ void __launch_bounds__(128) demap_kernel(RxDev d, FrameArgs fa) {
  demap_body(d, fa, own_block());
}

__global__ void __launch_bounds__(128) demap_batch_kernel(BView v) {
  int fi;
  VBlock vb;
  if (!batch_block(v, fi, vb)) return;
  const BFrame& f = v.frames[fi];
  demap_body(f.d, f.fa, vb);
}

// ---- launchers ------------------------------------------------------------

cudaError_t bps2_set_attributes();  // k_bps2.cu
cudaError_t launch_bps2(const RxDev& d, const FrameArgs& fa, cudaStream_t s);

template <int B, int W, bool Q>
static void launch_bps_t(const RxDev& d, const FrameArgs& fa, cudaStream_t s) {
  const long long n_dec = fa.k_b - fa.k_a;
  const int nruns = (int)((n_dec + kRun - 1) / kRun);
  const int nw = d.bps_nw;
  dim3 grid((nruns + nw - 1) / nw, 2);
  bps_kernel<B, W, Q><<<grid, 32 * nw, BpsSmem<B, W, Q>::bytes(nw), s>>>(d, fa);
}

template <int B, int W>
static cudaError_t bps_attr_t() {
  cudaError_t e = cudaFuncSetAttribute(bps_kernel<B, W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)BpsSmem<B, W, true>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(bps_kernel<B, W, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)BpsSmem<B, W, false>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(bps_batch_kernel<B, W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)BpsSmem<B, W, true>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(bps_batch_kernel<B, W, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)BpsSmem<B, W, false>::BYTES);
  return e;
}

// Opt-in to the dynamic shared memory of every instantiation (once per process).
cudaError_t bps_set_attributes() {
  cudaError_t e = cudaSuccess;
#define RX_BA(b, w) if (e == cudaSuccess) e = bps_attr_t<b, w>();
  RX_BA(64, 16) RX_BA(32, 16) RX_BA(64, 32) RX_BA(32, 32) RX_BA(64, 8) RX_BA(32, 8)
  RX_BA(64, 12) RX_BA(32, 12) RX_BA(64, 24) RX_BA(32, 24)
#undef RX_BA
  if (e == cudaSuccess) e = bps2_set_attributes();
  return e;
}

cudaError_t launch_bps(const RxDev& d, const FrameArgs& fa, cudaStream_t s) {
  if (fa.k_b <= fa.k_a) return cudaSuccess;
  if (d.bps_stride > 1) return launch_bps2(d, fa, s);
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

// ---- batched launchers (every frame of v has d's B, W, modulation and stride)

int launch_bps2_batch(const RxDev& d, const BView& v, int blocks, cudaStream_t s);  // k_bps2.cu

int bps_grid_x(const RxDev& d, const FrameArgs& fa) {
  const long long n_dec = fa.k_b - fa.k_a;
  const int nruns = (int)((n_dec + kRun - 1) / kRun);
  return d.bps_stride > 1 ? (nruns + 15) / 16 : (nruns + d.bps_nw - 1) / d.bps_nw;
}

int demap_grid_x(const FrameArgs& fa) { return (int)((fa.k_b - fa.k_a + kRun - 1) / kRun); }

cudaError_t launch_bps_batch(const RxDev& d, const BView& v, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  if (d.bps_stride > 1) return (cudaError_t)launch_bps2_batch(d, v, blocks, s);
  const bool q16 = d.bps == 4;
#define RX_BW(b, w)                                                                                 \
  if (d.B == b && d.W == w) {                                                                       \
    if (q16)                                                                                        \
      return launch_k(bps_batch_kernel<b, w, true>, blocks, 32 * d.bps_nw, BpsSmem<b, w, true>::bytes(d.bps_nw), s, v); \
    return launch_k(bps_batch_kernel<b, w, false>, blocks, 32 * d.bps_nw, BpsSmem<b, w, false>::bytes(d.bps_nw), s, v); \
  }
  RX_BW(64, 16) RX_BW(32, 16) RX_BW(64, 32) RX_BW(32, 32) RX_BW(64, 8) RX_BW(32, 8)
  RX_BW(64, 12) RX_BW(32, 12) RX_BW(64, 24) RX_BW(32, 24)
#undef RX_BW
  return cudaErrorInvalidValue;
}

cudaError_t launch_demap_batch(const BView& v, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  return launch_k(demap_batch_kernel, blocks, 128, 0, s, v);
}

cudaError_t launch_scan_batch(const BView& v, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  return launch_k(unwrap_scan_batch_kernel, blocks, 256, 0, s, v);
}

// The unwrap scan (one block per polarisation), then the demap.
cudaError_t launch_unwrap_demap(const RxDev& d, const FrameArgs& fa, cudaStream_t s) {
  if (fa.k_b <= fa.k_a) return cudaSuccess;
  const long long n_dec = fa.k_b - fa.k_a;
  const int nruns = (int)((n_dec + kRun - 1) / kRun);
  unwrap_scan_kernel<<<2, 256, 0, s>>>(d, fa);
  demap_kernel<<<nruns, 128, 0, s>>>(d, fa);
  return cudaGetLastError();
}

}  // namespace rx
