// a6, reduced-cost form: two-stage blind phase search.
//
// Stage 1 is the blind phase search of k_bps.cu restricted to the C = B/S
// coarse angles b = S j (C = 16 for QPSK, 8 for 16QAM): the same window
// costs D_{k,j} = sum_{|i|<=W} d(y_{k+i} e^{-j phi_{Sj}}), j* = argmin.
// Stage 2 places the fine index on the B-angle grid at the vertex of the
// parabola through the costs of j* and its two neighbours (cyclic in j:
// the cost is pi/2-periodic in the angle): c = D- - 2 D0 + D+,
// delta = (D- - D+) / (2c) in [-1/2, 1/2] (0 if c <= 0),
// b = (S j* + floor(S delta + 1/2)) mod B.  The unwrap, decisions and
// demapping that follow are those of the full search.
//
// Kernel layout: a warp holds four consecutive runs of kRun symbols, one
// per group of 8 lanes; lane q of a group holds coarse angles q and q + 8
// (QPSK) or q (16QAM) with its own register ring of the last 2W+1 metrics,
// exactly as one lane of the full search holds its fine angles.  With a
// quarter of the angles a group covers a run with 8 lanes instead of 32.
// Each run's window is staged on its own, at a stride that puts the four
// runs' loads of a step in different shared-memory banks.
// QPSK uses the gain form: d = |y|^2 + 2 - 2 (|z_x| + |z_y|), so the argmin
// of D is the argmax of G = sum (|z_x| + |z_y|) (the |y|^2 + 2 part is the
// same for every angle), and angle j + 8 is angle j + pi/4, whose gain is
// sqrt2 max(|z_x|, |z_y|): one rotation per lane and step serves both.
// Symbols outside the stream are staged as zeros and add nothing to G; in
// 16QAM they carry a zero weight.  Each step the lanes store their angles'
// keys (float bits with the low 4 bits replaced by the angle) in a row;
// every R steps (R divides 2W+1) one lane per (row, run) finds the best key,
// reads the two neighbours and writes the refined index.
#include <climits>

#include "bps_common.cuh"

namespace rx {

// Rows between two reductions: a divisor of the window length 2W+1 (so a
// row's place in the unrolled super-step is static), at most 25.
constexpr int bps2_period(int win) {
  return win % 11 == 0 ? 11 : win % 13 == 0 ? 13 : win % 7 == 0 ? 7 : win;
}

// Staging stride between the runs of a warp (entries of EB bytes): at least
// `steps`, and 8 words apart modulo the 32 banks so that the four runs'
// loads of one step fall in different banks.
constexpr int bps2_stride(int steps, int eb) {
  int gs = steps;
  while ((gs * eb / 4) % 32 != 8) ++gs;
  return gs;
}

// Dynamic shared memory of one 4-warp block, per warp: R key rows of ROWW
// words, the staged symbols of its four runs (each run's window on its
// own, GS entries apart: float2 {x, y} for QPSK, float4 {x, y, weight, 0}
// for 16QAM) and the runs' angle indices.
template <int W, bool QAM16>
struct Bps2Smem {
  static constexpr int C = QAM16 ? 8 : 16;              // coarse angles
  static constexpr int G = 4;                           // runs per warp
  static constexpr int WIN = 2 * W + 1;
  static constexpr int R = bps2_period(WIN);
  static constexpr int ROWW = G * C + 4;                // padded key row (words)
  static constexpr int YS = kRun + 2 * W;               // steps per run
  static constexpr int NSUP = (YS + WIN - 1) / WIN;
  static constexpr int STEPS = NSUP * WIN;              // steps run (zeros past the run)
  static constexpr int EB = QAM16 ? 16 : 8;              // bytes per staged symbol
  static constexpr int GS = bps2_stride(STEPS, EB);
  static constexpr size_t KEY_BYTES = sizeof(uint32_t) * R * ROWW;
  static constexpr size_t Y_BYTES = (size_t)EB * G * GS;
  static constexpr size_t BH_BYTES = G * kRun;
  static constexpr size_t WARP_BYTES = KEY_BYTES + Y_BYTES + BH_BYTES;
  static constexpr size_t BYTES = 4 * WARP_BYTES;
  static_assert(KEY_BYTES % 16 == 0 && Y_BYTES % 16 == 0, "16-byte aligned parts");
  static constexpr int MIN_BLOCKS = W <= 16 ? 4 : 2;    // register budget of the window ring
};

// Word of coarse angle j in a QPSK run's 16 keys (a lane's two angles
// q and q + 8 are adjacent so that one 64-bit store writes both).
__device__ __forceinline__ int qpsk_word(int j) { return 2 * (j & 7) + (j >> 3); }

template <int W, bool QAM16>
__device__ __forceinline__ void bps2_body(const RxDev& d, const FrameArgs& fa, VBlock vb) {
  using SM = Bps2Smem<W, QAM16>;
  constexpr int C = SM::C, G = SM::G, WIN = SM::WIN, R = SM::R, ROWW = SM::ROWW;
  extern __shared__ __align__(16) unsigned char bps2_smem[];
  __shared__ float2 cs_s[64];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane >> 3, q = lane & 7;
  const int pol = vb.y;
  const int B = d.B, S = d.bps_stride;
  const long long n_dec = fa.k_b - fa.k_a;
  const int nruns = (int)((n_dec + kRun - 1) / kRun);
  const int run0 = (vb.x * 4 + warp) * G;
  const long long kw0 = fa.k_a + (long long)run0 * kRun;
  // symbols left from the warp's first run on (runs are consecutive; only
  // the last run of the frame can be short)
  const int rem = (int)max(0LL, min(fa.k_b - kw0, (long long)G * kRun));
  auto run_len = [&](int g) -> int { return min(max(rem - g * kRun, 0), kRun); };

  if (threadIdx.x < B) {
    float sb, cb;
    sincospif(((float)threadIdx.x / (float)B - 0.5f) * 0.5f, &sb, &cb);
    cs_s[threadIdx.x] = make_float2(cb, sb);
  }
  // the lane's first coarse angle, fine index S q
  const float sc = QAM16 ? 3.16227766016837933f : 1.f;
  float c0, s0;
  sincospif(((float)(S * q) / (float)B - 0.5f) * 0.5f, &s0, &c0);
  c0 *= sc;
  s0 *= sc;

  unsigned char* wbase = bps2_smem + warp * SM::WARP_BYTES;
  uint32_t* kw = reinterpret_cast<uint32_t*>(wbase);
  float4* ys4 = reinterpret_cast<float4*>(wbase + SM::KEY_BYTES);  // 16QAM
  float2* ys2 = reinterpret_cast<float2*>(wbase + SM::KEY_BYTES);  // QPSK
  uint8_t* bh_w = wbase + SM::KEY_BYTES + SM::Y_BYTES;

  // stage run g's window, symbols kw0 + g kRun - W + i for i < STEPS, at
  // entry g GS + i (zero outside the stream)
  const long long fbase = fa.f * (long long)d.F;
  const float2* yf = d.y + ((long long)(fa.f & 1) * 2 + pol) * (kYHist + d.F) + kYHist;
  const long long ylim = min(fa.n_sym, fbase + fa.Ff);  // symbols beyond do not exist (yet)
  // eight loads per lane in flight before their stores
  for (int e0 = 0; e0 < G * SM::STEPS; e0 += 8 * 32) {
    float2 v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int e = e0 + lane + 32 * r;
      const int g = e / SM::STEPS, i = e - g * SM::STEPS;
      const long long k = kw0 + (long long)g * kRun - W + i;
      v[r] = (e < G * SM::STEPS && k >= 0 && k < ylim) ? yf[k - fbase] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int e = e0 + lane + 32 * r;
      if (e < G * SM::STEPS) {
        const int g = e / SM::STEPS, i = e - g * SM::STEPS;
        const long long k = kw0 + (long long)g * kRun - W + i;
        if (QAM16) ys4[g * SM::GS + i] = make_float4(v[r].x, v[r].y, (k >= 0 && k < ylim) ? 1.f : 0.f, 0.f);
        else ys2[g * SM::GS + i] = v[r];
      }
    }
  }
  __syncthreads();  // cs_s, staged symbols

  // Reduction of the R rows of steps s_first .. s_first + R - 1: one lane
  // per (row, run); the refined index of the run's symbol s - 2W.
  auto reduce_rows = [&](int s_first) {
    for (int it = lane; it < R * G; it += 32) {
      const int g = it / R, t = it - g * R;
      const int s = s_first + t;
      const int ko = s - 2 * W;
      if (ko < 0 || ko >= run_len(g)) continue;
      const uint32_t* row = kw + t * ROWW + g * C;
      const uint4* row4 = reinterpret_cast<const uint4*>(row);
      int j;
      float f0, fm, fp, num, den;
      if constexpr (QAM16) {  // metric keys, smallest wins, angle in the low bits
        uint32_t best = 0xffffffffu;
#pragma unroll
        for (int c4 = 0; c4 < C / 4; ++c4) {
          const uint4 v = row4[c4];
          best = min(best, min(min(v.x, v.y), min(v.z, v.w)));
        }
        j = (int)(best & 15u);
        f0 = __uint_as_float(best & ~15u);
        fm = __uint_as_float(row[(j - 1) & (C - 1)] & ~15u);
        fp = __uint_as_float(row[(j + 1) & (C - 1)] & ~15u);
        num = fm - fp;
        den = fm - 2.f * f0 + fp;
      } else {  // gain keys, largest wins (signed: a rounding residue below 0 loses)
        int best = INT_MIN;
#pragma unroll
        for (int c4 = 0; c4 < C / 4; ++c4) {
          const int4 v = reinterpret_cast<const int4*>(row4)[c4];
          best = max(best, max(max(v.x, v.y), max(v.z, v.w)));
        }
        j = 15 - (best & 15);
        f0 = __int_as_float(best & ~15);
        fm = __uint_as_float(row[qpsk_word((j - 1) & 15)] & ~15u);
        fp = __uint_as_float(row[qpsk_word((j + 1) & 15)] & ~15u);
        num = fp - fm;  // costs are -gains
        den = 2.f * f0 - fm - fp;
      }
      const float delta = den > 0.f ? fminf(fmaxf(__fdividef(num, 2.f * den), -0.5f), 0.5f) : 0.f;
      const int r = __float2int_rd(fmaf((float)S, delta, 0.5f));
      bh_w[g * kRun + ko] = (uint8_t)((S * j + r + B) & (B - 1));
    }
  };

  const int ybase = grp * SM::GS;  // the group's staged window
  if constexpr (QAM16) {
    float ring[WIN];
#pragma unroll
    for (int u = 0; u < WIN; ++u) ring[u] = 0.f;
    float D = 0.f;
    for (int base = 0; base < SM::STEPS; base += WIN) {
#pragma unroll
      for (int u = 0; u < WIN; ++u) {
        const float4 v = ys4[ybase + base + u];
        const float zx = fmaf(v.x, c0, v.y * s0);
        const float zy = fmaf(v.y, c0, -v.x * s0);
        const float ex = fabsf(fabsf(zx) - 2.f) - 1.f;
        const float ey = fabsf(fabsf(zy) - 2.f) - 1.f;
        const float m = fmaf(ex, ex, ey * ey) * v.z;
        D += m - ring[u];
        ring[u] = m;
        kw[(u % R) * ROWW + grp * C + q] = (__float_as_uint(D) & ~15u) | (uint32_t)q;
        if ((u + 1) % R == 0) {
          __syncwarp();
          reduce_rows(base + u + 1 - R);
          __syncwarp();
        }
      }
    }
  } else {
    // rotation z = y e^{-j phi_q}; packed gains (|zx| + |zy|, sqrt2 max(|zx|, |zy|))
    // of angles q and q + 8
    unsigned long long ring2[WIN];
#pragma unroll
    for (int u = 0; u < WIN; ++u) ring2[u] = 0ull;
    unsigned long long D2 = 0ull;
    const unsigned long long K2 = f2pk(1.f, 1.41421356237309505f);
    const float2* yq = ys2 + ybase;
    uint2* kq = reinterpret_cast<uint2*>(kw + grp * C + 2 * q);
    const uint32_t lo_a = 15u - (uint32_t)q, lo_b = 7u - (uint32_t)q;  // 15 - q, 15 - (q + 8)
    for (int base = 0; base < SM::STEPS; base += WIN) {
      float2 p0 = yq[base], p1 = yq[base + 1];
#pragma unroll
      for (int u = 0; u < WIN; ++u) {
        const float2 v = p0;
        p0 = p1;
        if (u + 2 < WIN) p1 = yq[base + u + 2];
        const float zx = fmaf(v.x, c0, v.y * s0);
        const float zy = fmaf(v.y, c0, -v.x * s0);
        const float ax = fabsf(zx), ay = fabsf(zy);
        const unsigned long long g2 = f2mul(f2pk(ax + ay, fmaxf(ax, ay)), K2);
        D2 = f2add(D2, f2sub(g2, ring2[u]));
        ring2[u] = g2;
        float d0, d1;
        f2up(D2, d0, d1);
        kq[(u % R) * (ROWW / 2)] = make_uint2((__float_as_uint(d0) & ~15u) | lo_a, (__float_as_uint(d1) & ~15u) | lo_b);
        if ((u + 1) % R == 0) {
          __syncwarp();
          reduce_rows(base + u + 1 - R);
          __syncwarp();
        }
      }
    }
  }

  // decisions, unwrap increments and EVM of the warp's runs; block epilogue
  float evn = 0.f, evd = 0.f;
#pragma unroll 1
  for (int g = 0; g < G; ++g) {
    float en, ed;
    const int y0 = g * SM::GS + W;
    bps_finish_run(d, fa, pol, run0 + g, nruns, kw0 + (long long)g * kRun, run_len(g), bh_w + g * kRun, cs_s,
                   [&](int ko) { return QAM16 ? make_float2(ys4[y0 + ko].x, ys4[y0 + ko].y) : ys2[y0 + ko]; }, en,
                   ed);
    evn += en;
    evd += ed;
  }
  bps_finish_block<128>(d, evn, evd);
}

template <int W, bool QAM16>
__global__ void __launch_bounds__(128, Bps2Smem<W, QAM16>::MIN_BLOCKS) bps2_kernel(RxDev d, FrameArgs fa) {
  bps2_body<W, QAM16>(d, fa, own_block());
}

template <int W, bool QAM16>
__global__ void __launch_bounds__(128, Bps2Smem<W, QAM16>::MIN_BLOCKS) bps2_batch_kernel(BView v) {
  int fi;
  VBlock vb;
  if (!batch_block(v, fi, vb)) return;
  const BFrame& f = v.frames[fi];
  bps2_body<W, QAM16>(f.d, f.fa, vb);
}

template <int W, bool Q>
static void launch_bps2_t(const RxDev& d, const FrameArgs& fa, cudaStream_t s) {
  const long long n_dec = fa.k_b - fa.k_a;
  const int nruns = (int)((n_dec + kRun - 1) / kRun);
  dim3 grid((nruns + 15) / 16, 2);
  bps2_kernel<W, Q><<<grid, 128, Bps2Smem<W, Q>::BYTES, s>>>(d, fa);
}

template <int W>
static cudaError_t bps2_attr_t() {
  cudaError_t e = cudaFuncSetAttribute(bps2_kernel<W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Bps2Smem<W, true>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(bps2_kernel<W, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Bps2Smem<W, false>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(bps2_batch_kernel<W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Bps2Smem<W, true>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(bps2_batch_kernel<W, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Bps2Smem<W, false>::BYTES);
  return e;
}

// Opt-in to the dynamic shared memory of every instantiation (once per process).
cudaError_t bps2_set_attributes() {
  cudaError_t e = cudaSuccess;
#define RX_BA(w) if (e == cudaSuccess) e = bps2_attr_t<w>();
  RX_BA(8) RX_BA(12) RX_BA(16) RX_BA(24) RX_BA(32)
#undef RX_BA
  return e;
}

// Two-stage search; d.bps_stride = B/16 (QPSK) or B/8 (16QAM).
cudaError_t launch_bps2(const RxDev& d, const FrameArgs& fa, cudaStream_t s) {
  if (fa.k_b <= fa.k_a) return cudaSuccess;
  const bool q16 = d.bps == 4;
  if (d.bps_stride * (q16 ? 8 : 16) != d.B) return cudaErrorInvalidValue;
#define RX_W(w)                                   \
  if (d.W == w) {                                 \
    if (q16) launch_bps2_t<w, true>(d, fa, s);    \
    else launch_bps2_t<w, false>(d, fa, s);       \
    return cudaGetLastError();                    \
  }
  RX_W(16) RX_W(32) RX_W(8) RX_W(12) RX_W(24)
#undef RX_W
  return cudaErrorInvalidValue;
}

// Batched two-stage search (a cudaError_t value); every frame of v has d's W and modulation.
int launch_bps2_batch(const RxDev& d, const BView& v, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  const bool q16 = d.bps == 4;
  if (d.bps_stride * (q16 ? 8 : 16) != d.B) return cudaErrorInvalidValue;
#define RX_W(w)                                                                                 \
  if (d.W == w) {                                                                               \
    if (q16) return launch_k(bps2_batch_kernel<w, true>, blocks, 128, Bps2Smem<w, true>::BYTES, s, v); \
    return launch_k(bps2_batch_kernel<w, false>, blocks, 128, Bps2Smem<w, false>::BYTES, s, v);        \
  }
  RX_W(16) RX_W(32) RX_W(8) RX_W(12) RX_W(24)
#undef RX_W
  return cudaErrorInvalidValue;
}

}  // namespace rx
