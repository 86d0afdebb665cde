// a4 2x2 butterfly FIR and a5 block-LMS adaptation (CMA acquisition, then
// decision-directed LMS -- paper Sec. II uses a DD-LMS time-domain equaliser).
//
// One warp runs one adaptive chain.  A sub-block of K = 64 symbols:
//   y_p[k] = sum_q sum_t w[p][q][t] r_q[2k + t]            (taps fixed)
//   CMA:  e_p = y_p (|y_p|^2 - R2)
//   DD:   phi_p = arg(-sum_k y_p^4) / 4,  e_p = y_p - e^{j phi} dec(e^{-j phi} y_p)
//   g[p][q][t] = (1/K) sum_k e_p[k] conj(r_q[2k + t]),  w <- w - mu g
// where r_q[i] = rot(i) z_q[i] is the CD output with the frame's AGC gain
// and frequency-offset rotation applied on load (fused, never stored).
//
// Lane l computes the outputs of symbols 2l and 2l+1 (their sample windows
// overlap, so each lane loads T+2 samples per polarisation), then owns the
// tap pairs (q, t) = divmod(l, T) (and l + 32) for the gradient.  The
// sub-block's samples live in shared memory split into 4 planes by index
// mod 4 (conflict-free for the lane stride of 4), the two input
// polarisations' planes 64 bytes apart modulo 128 (conflict-free gradient
// reads); taps are stored as float4 {w[0][q][t], w[1][q][t]} and read as
// broadcasts.
//
// Schedule (both kernels together): the first frame is preceded by one
// sequential acquisition chain over its first acq_syms symbols (CMA while a
// sub-block starts before cma_syms, DD after; singularity check at the
// switch).  Every frame is cut into segments of S symbols; segment j runs
// DD-LMS starting from the final taps of segment j of the previous frame
// (frame 0: from the acquisition taps), so all segments of a frame run in
// parallel, one warp each.
#include "rx_internal.cuh"

namespace rx {

constexpr int kK = 64;

template <int T>
struct ChainSmem {
  static constexpr int NEED = (2 * kK + T - 1 + 3) / 4;
  static constexpr int P4 = NEED + ((4 - NEED % 16) + 16) % 16;  // P4 = 4 mod 16
  static constexpr int QS = 4 * P4 + 8;  // q stride: the q planes 64 bytes apart mod 128
  float2 r[2 * QS];
  float4 w[2][T];
  float4 e[kK];
};

template <int T>
__device__ __forceinline__ float2 sm_r(const ChainSmem<T>& sm, int q, int s) {
  return sm.r[q * ChainSmem<T>::QS + (s & 3) * ChainSmem<T>::P4 + (s >> 2)];
}

// One sub-block update of nk (<= 64) symbols.  mode 0 = CMA, 1 = DD.
// Outputs of the lane's symbols are returned in y[p][j] (j = 0, 1).
template <int T>
__device__ __forceinline__ void sub_block(ChainSmem<T>& sm, int nk, int mode, float mu, float R2, int nl,
                                          float2 (&y)[2][2]) {
  const int lane = threadIdx.x & 31;
  // ---- FIR: symbols 2l, 2l+1
#pragma unroll
  for (int p = 0; p < 2; ++p) y[p][0] = y[p][1] = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    float2 xa = sm_r(sm, q, 4 * lane), xb = sm_r(sm, q, 4 * lane + 1);
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const float2 xn = sm_r(sm, q, 4 * lane + t + 2);
      const float4 w = sm.w[q][t];
      y[0][0].x = fmaf(w.x, xa.x, fmaf(-w.y, xa.y, y[0][0].x));
      y[0][0].y = fmaf(w.x, xa.y, fmaf(w.y, xa.x, y[0][0].y));
      y[1][0].x = fmaf(w.z, xa.x, fmaf(-w.w, xa.y, y[1][0].x));
      y[1][0].y = fmaf(w.z, xa.y, fmaf(w.w, xa.x, y[1][0].y));
      y[0][1].x = fmaf(w.x, xn.x, fmaf(-w.y, xn.y, y[0][1].x));
      y[0][1].y = fmaf(w.x, xn.y, fmaf(w.y, xn.x, y[0][1].y));
      y[1][1].x = fmaf(w.z, xn.x, fmaf(-w.w, xn.y, y[1][1].x));
      y[1][1].y = fmaf(w.z, xn.y, fmaf(w.w, xn.x, y[1][1].y));
      xa = xb;
      xb = xn;
    }
  }
  const bool v0 = 2 * lane < nk, v1 = 2 * lane + 1 < nk;
  // ---- errors
  float2 e[2][2];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    if (mode == 0) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const float2 a = y[p][j];
        e[p][j] = cscale(a, a.x * a.x + a.y * a.y - R2);
      }
    } else {
      float sx = 0.f, sy = 0.f;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        if (j == 0 ? v0 : v1) {
          const float2 a = y[p][j];
          const float2 a2 = make_float2(a.x * a.x - a.y * a.y, 2.f * a.x * a.y);
          sx += a2.x * a2.x - a2.y * a2.y;
          sy += 2.f * a2.x * a2.y;
        }
      }
      sx = warp_sum(sx);
      sy = warp_sum(sy);
      float ph = 0.f;
      if (sx != 0.f || sy != 0.f) ph = 0.25f * atan2f(-sy, -sx);
      float sn, cs;
      sincosf(ph, &sn, &cs);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const float2 a = y[p][j];
        const float2 zr = make_float2(a.x * cs + a.y * sn, a.y * cs - a.x * sn);  // a e^{-j ph}
        const float dx = level_val(level_of(zr.x, nl), nl), dy = level_val(level_of(zr.y, nl), nl);
        const float2 dd = make_float2(dx * cs - dy * sn, dx * sn + dy * cs);      // dec e^{j ph}
        e[p][j] = csub(a, dd);
      }
    }
  }
  if (!v0) e[0][0] = e[1][0] = make_float2(0.f, 0.f);
  if (!v1) e[0][1] = e[1][1] = make_float2(0.f, 0.f);
  sm.e[2 * lane] = make_float4(e[0][0].x, e[0][0].y, e[1][0].x, e[1][0].y);
  sm.e[2 * lane + 1] = make_float4(e[0][1].x, e[0][1].y, e[1][1].x, e[1][1].y);
  __syncwarp();
  // ---- gradient and update of the lane's tap pairs
  const float step = mu / (float)nk;
  for (int pr = lane; pr < 2 * T; pr += 32) {
    const int q = pr / T, t = pr - q * T;
    float g0x = 0.f, g0y = 0.f, g1x = 0.f, g1y = 0.f;
    // e * conj(x) summed over k in order; r_q[2k + t] sits in plane
    // (2k + t) mod 4 at (2k + t) / 4, so even k read one plane and odd k
    // another, each at consecutive entries
    auto acc = [&](const float4& ee, const float2& x) {
      g0x = fmaf(ee.x, x.x, fmaf(ee.y, x.y, g0x));
      g0y = fmaf(ee.y, x.x, fmaf(-ee.x, x.y, g0y));
      g1x = fmaf(ee.z, x.x, fmaf(ee.w, x.y, g1x));
      g1y = fmaf(ee.w, x.x, fmaf(-ee.z, x.y, g1y));
    };
    const float2* xe = &sm.r[q * ChainSmem<T>::QS + (t & 3) * ChainSmem<T>::P4 + (t >> 2)];
    const float2* xo = &sm.r[q * ChainSmem<T>::QS + ((t + 2) & 3) * ChainSmem<T>::P4 + ((t + 2) >> 2)];
    const int npair = nk >> 1;
#pragma unroll 4
    for (int m = 0; m < npair; ++m) {
      acc(sm.e[2 * m], xe[m]);
      acc(sm.e[2 * m + 1], xo[m]);
    }
    if (nk & 1) acc(sm.e[nk - 1], xe[npair]);
    float4 w = sm.w[q][t];
    w.x -= step * g0x;
    w.y -= step * g0y;
    w.z -= step * g1x;
    w.w -= step * g1y;
    sm.w[q][t] = w;
  }
  __syncwarp();
}

template <int T>
__device__ __forceinline__ void load_taps(ChainSmem<T>& sm, const float2* src) {  // src [p][q][t]
  const int lane = threadIdx.x & 31;
  for (int pr = lane; pr < 2 * T; pr += 32) {
    const int q = pr / T, t = pr - q * T;
    const float2 a = src[(0 * 2 + q) * T + t], b = src[(1 * 2 + q) * T + t];
    sm.w[q][t] = make_float4(a.x, a.y, b.x, b.y);
  }
  __syncwarp();
}

template <int T>
__device__ __forceinline__ void store_taps(const ChainSmem<T>& sm, float2* dst) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  for (int pr = lane; pr < 2 * T; pr += 32) {
    const int q = pr / T, t = pr - q * T;
    const float4 w = sm.w[q][t];
    dst[(0 * 2 + q) * T + t] = make_float2(w.x, w.y);
    dst[(1 * 2 + q) * T + t] = make_float2(w.z, w.w);
  }
}

// Sequential acquisition of the first frame, one block of 256 threads
// (the chain is inherently sequential, so its latency is spread over a
// block).  The rotated samples pass through a shared ring of four
// 128-sample blocks per polarisation, kept as even/odd planes (with the
// first 80 entries mirrored past the end, so window reads never wrap);
// blocks are loaded into registers two sub-blocks ahead.
// FIR: thread (q, k, p) = (t & 1, (t >> 1) & 63, t >> 7) forms
// sum_t w[p][q][t] r_q[2k + t]; the q pair is added with a shuffle.
// Gradient: thread (combo, quarter) = (t >> 2, t & 3) sums e_p[k] conj(r_q[2k + t])
// over the sub-block's symbols k = quarter mod 4; the quarters are added
// with shuffles and the quarter-0 thread updates the tap.
template <int T>
__device__ __forceinline__ void acq_body(const RxDev& d, const FrameArgs& fa) {
  constexpr int PL = 344;   // plane stride (float2): 256 + 80 mirror, = 64 B mod 128 B
  __shared__ float2 r_s[4 * PL + 8];
  __shared__ float2 w_s[2][2][T];         // [p][q][t]
  __shared__ float2 e_s[2][kK];
  __shared__ float2 y1_s[kK];             // y_y outputs for the singularity check
  __shared__ float red_s[8][4];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int zlen_f = 2 * fa.Ff + 2 * d.c;
  const int n_acq = min(d.acq_syms, fa.Ff);
  const int nsub = (n_acq + kK - 1) / kK;
  for (int i = tid; i < 4 * T; i += 256) {
    const int p = i / (2 * T), q = (i / T) & 1, t = i % T;
    w_s[p][q][t] = make_float2((p == q && t == (T - 1) / 2) ? 1.f : 0.f, 0.f);
  }
  auto plane = [&](int q, int par) -> float2* { return r_s + (2 * q + par) * PL + q * 8; };
  // one 128-sample block per polarisation: thread (q, s) = (tid >> 7, tid & 127).
  // The raw loads stay in registers until the block is stored (rotation
  // applied then), so nothing waits for them earlier.
  struct Raw { float2 z, h, l; };
  auto load_blk = [&](int b) -> Raw {
    const int q = tid >> 7, n = 128 * b + (tid & 127);
    Raw r{make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    if (b < nsub + 2 && n < zlen_f) {
      r.z = d.z[(long long)q * d.zlen + n];
      r.h = __ldg(&d.rot_hi[n >> 10]);
      r.l = __ldg(&d.rot_lo[n & (kRotLo - 1)]);
    }
    return r;
  };
  auto store_blk = [&](int b, const Raw& r) {
    const int q = tid >> 7, s = tid & 127;
    const int idx = ((64 * b) & 255) + (s >> 1);
    const float2 v = cmul(r.z, cmul(r.h, r.l));
    float2* pl = plane(q, s & 1);
    pl[idx] = v;
    if (idx < 80) pl[idx + 256] = v;
  };
  const int cma_end = min(((d.cma_syms + kK - 1) / kK) * kK, n_acq);
  const int corr_lo = max(cma_end - 1024, 0);
  float cxr = 0.f, cxi = 0.f, pxx = 0.f, pyy = 0.f;
  bool was_cma = false;
  Raw pre0 = load_blk(2), pre1 = load_blk(3);
  store_blk(0, load_blk(0));
  store_blk(1, load_blk(1));
  __syncthreads();
  const int qq = tid & 1, kk = (tid >> 1) & 63, pp = tid >> 7;
  constexpr int NG = 16 * T;  // gradient (combo, quarter) pairs
  for (int i = 0; i < nsub; ++i) {
    const int k0 = i * kK;
    const int nk = min(kK, n_acq - k0);
    const int mode = k0 < d.cma_syms ? 0 : 1;
    // block i + 2 into the ring (slot of block i - 2), block i + 4 into registers
    if (i & 1) {
      store_blk(i + 2, pre1);
      pre1 = load_blk(i + 4);
    } else {
      store_blk(i + 2, pre0);
      pre0 = load_blk(i + 4);
    }
    if (mode == 1 && was_cma) {
      // singularity check over the last CMA outputs
      float v0 = warp_sum(cxr), v1 = warp_sum(cxi), v2 = warp_sum(pxx), v3 = warp_sum(pyy);
      if (lane == 0) { red_s[warp][0] = v0; red_s[warp][1] = v1; red_s[warp][2] = v2; red_s[warp][3] = v3; }
      __syncthreads();
      float sxy = 0.f, syx = 0.f, sxx = 0.f, syy = 0.f;
      for (int w = 0; w < 8; ++w) { sxy += red_s[w][0]; syx += red_s[w][1]; sxx += red_s[w][2]; syy += red_s[w][3]; }
      const float den = sqrtf(sxx * syy);
      const float rho = den > 0.f ? sqrtf(sxy * sxy + syx * syx) / den : 0.f;
      if (rho > 0.5f) {
        float2 a = make_float2(0.f, 0.f), b2 = a;
        if (tid < T) {
          a = w_s[0][1][T - 1 - tid];   // w_xy reversed
          b2 = w_s[0][0][T - 1 - tid];  // w_xx reversed
        }
        __syncthreads();
        if (tid < T) {
          w_s[1][0][tid] = make_float2(-a.x, a.y);    // -conj(w_xy[T-1-t])
          w_s[1][1][tid] = make_float2(b2.x, -b2.y);  // conj(w_xx[T-1-t])
        }
        if (tid == 0) d.st->reinit = 1;
      }
      __syncthreads();
    }
    // ---- FIR over one input polarisation, two accumulators (even/odd taps)
    const int base = (64 * i) & 255;
    const float2* rp0 = plane(qq, 0) + base + kk;
    const float2* rp1 = plane(qq, 1) + base + kk;
    float2 a0 = make_float2(0.f, 0.f), a1 = a0;
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const float2 w = w_s[pp][qq][t];
      const float2 x = (t & 1) ? rp1[t >> 1] : rp0[t >> 1];
      float2& acc = (t & 1) ? a1 : a0;
      acc.x = fmaf(w.x, x.x, fmaf(-w.y, x.y, acc.x));
      acc.y = fmaf(w.x, x.y, fmaf(w.y, x.x, acc.y));
    }
    float2 y = make_float2(a0.x + a1.x, a0.y + a1.y);
    y.x += __shfl_xor_sync(0xffffffffu, y.x, 1);
    y.y += __shfl_xor_sync(0xffffffffu, y.y, 1);
    const bool valid = kk < nk;
    // ---- error
    float2 e;
    if (mode == 0) {
      e = cscale(y, y.x * y.x + y.y * y.y - d.R2);
      if (k0 + nk > corr_lo && k0 < cma_end) {  // sub-block overlaps the correlation range
        if (pp == 1 && qq == 0) y1_s[kk] = y;
        __syncthreads();
        const int k = k0 + kk;
        if (valid && pp == 0 && qq == 0 && k >= corr_lo && k < cma_end) {
          const float2 yo = y1_s[kk];
          cxr += y.x * yo.x + y.y * yo.y;
          cxi += y.y * yo.x - y.x * yo.y;
          pxx += y.x * y.x + y.y * y.y;
          pyy += yo.x * yo.x + yo.y * yo.y;
        }
      }
    } else {
      float sx = 0.f, sy = 0.f;
      if (valid && qq == 0) {
        const float2 a2 = make_float2(y.x * y.x - y.y * y.y, 2.f * y.x * y.y);
        sx = a2.x * a2.x - a2.y * a2.y;
        sy = 2.f * a2.x * a2.y;
      }
      sx = warp_sum(sx);
      sy = warp_sum(sy);
      if (lane == 0) { red_s[warp][0] = sx; red_s[warp][1] = sy; }
      __syncthreads();
      sx = red_s[4 * pp][0] + red_s[4 * pp + 1][0] + red_s[4 * pp + 2][0] + red_s[4 * pp + 3][0];
      sy = red_s[4 * pp][1] + red_s[4 * pp + 1][1] + red_s[4 * pp + 2][1] + red_s[4 * pp + 3][1];
      float ph = 0.f;
      if (sx != 0.f || sy != 0.f) ph = 0.25f * atan2f(-sy, -sx);
      float sn, cs;
      sincosf(ph, &sn, &cs);
      const float2 zr = make_float2(y.x * cs + y.y * sn, y.y * cs - y.x * sn);
      const float dx = level_val(level_of(zr.x, d.nl), d.nl), dy = level_val(level_of(zr.y, d.nl), d.nl);
      e = csub(y, make_float2(dx * cs - dy * sn, dx * sn + dy * cs));
    }
    if (qq == 0) e_s[pp][kk] = valid ? e : make_float2(0.f, 0.f);
    __syncthreads();
    // ---- gradient: thread (combo, quarter) sums over k = quarter mod 4
    // (every lane runs every iteration: shuffles)
    {
      const float step = (mode == 0 ? d.mu_cma : d.mu_dd) / (float)nk;
#pragma unroll
      for (int c0 = 0; c0 < NG; c0 += 256) {
        const int c = c0 + tid;
        const bool act = c < NG;
        const int cg = act ? c >> 2 : 0, qt = c & 3;
        const int gp = cg / (2 * T), gq = (cg / T) & 1, gt = cg % T;
        const float2* rq = plane(gq, gt & 1) + base + qt + (gt >> 1);  // r_q[2k + t] at k = qt + 4m: rq[4m]
        const float2* eq = &e_s[gp][qt];
        float gx0 = 0.f, gy0 = 0.f, gx1 = 0.f, gy1 = 0.f;
        if (act) {
#pragma unroll
          for (int m = 0; m < kK / 4; m += 2) {
            const float2 ea = eq[4 * m], xa = rq[4 * m];
            const float2 eb = eq[4 * m + 4], xb = rq[4 * m + 4];
            gx0 = fmaf(ea.x, xa.x, fmaf(ea.y, xa.y, gx0));
            gy0 = fmaf(ea.y, xa.x, fmaf(-ea.x, xa.y, gy0));
            gx1 = fmaf(eb.x, xb.x, fmaf(eb.y, xb.y, gx1));
            gy1 = fmaf(eb.y, xb.x, fmaf(-eb.x, xb.y, gy1));
          }
        }
        float gx = gx0 + gx1, gy = gy0 + gy1;
        gx += __shfl_xor_sync(0xffffffffu, gx, 1);
        gy += __shfl_xor_sync(0xffffffffu, gy, 1);
        gx += __shfl_xor_sync(0xffffffffu, gx, 2);
        gy += __shfl_xor_sync(0xffffffffu, gy, 2);
        if (act && qt == 0) {
          float2 w = w_s[gp][gq][gt];
          w.x -= step * gx;
          w.y -= step * gy;
          w_s[gp][gq][gt] = w;
        }
      }
    }
    __syncthreads();
    was_cma = mode == 0;
  }
  for (int i = tid; i < 4 * T; i += 256) {
    const int p = i / (2 * T), q = (i / T) & 1, t = i % T;
    d.w_acq[(p * 2 + q) * T + t] = w_s[p][q][t];
  }
}

template <int T>
__global__ void __launch_bounds__(256) acq_kernel(RxDev d, FrameArgs fa) {
  acq_body<T>(d, fa);
}

template <int T>
__global__ void __launch_bounds__(256) acq_batch_kernel(BView v) {
  int fi;
  VBlock vb;
  if (!batch_block(v, fi, vb)) return;
  const BFrame& f = v.frames[fi];
  acq_body<T>(f.d, f.fa);
}

// All segments of one frame, one warp per segment, d.mimo_nw warps per
// block (the block's dynamic shared memory holds one ChainSmem per warp).
template <int T>
__device__ __forceinline__ void mimo_body(const RxDev& d, const FrameArgs& fa, long long hist_base, VBlock vb) {
  extern __shared__ float4 mimo_smem4[];
  ChainSmem<T>* sms = reinterpret_cast<ChainSmem<T>*>(mimo_smem4);
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = vb.x * (int)(blockDim.x >> 5) + wib;
  const int nseg = (fa.Ff + d.S - 1) / d.S;
  if (j >= nseg) return;
  ChainSmem<T>& sm = sms[wib];
  const int zlen_f = 2 * fa.Ff + 2 * d.c;
  float2* chain = d.chains + (long long)j * 4 * T;
  load_taps<T>(sm, fa.f == 0 ? d.w_acq : chain);
  // frame f's equalised symbols go to buffer f % 2 after a copy of the last
  // kYHist symbols of frame f-1 (zeros for the first frame)
  float2* yb = d.y + (long long)(fa.f & 1) * 2 * (kYHist + d.F);
  if (vb.x == 0 && wib == 0) {
    const float2* yp = d.y + (long long)((fa.f + 1) & 1) * 2 * (kYHist + d.F);
    for (int i = lane; i < 2 * kYHist; i += 32) {
      const int p = i / kYHist, t = i % kYHist;
      yb[(long long)p * (kYHist + d.F) + t] =
          fa.f == 0 ? make_float2(0.f, 0.f) : yp[(long long)p * (kYHist + d.F) + d.F + t];
    }
  }
  yb += kYHist;
  const int a = j * d.S, e = min(a + d.S, fa.Ff);
  // the next sub-block's CD samples are loaded into registers while the
  // current one computes; rotation (L1-resident tables) is applied on store
  constexpr int NSP = 2 * kK + T - 1;
  constexpr int PF = (NSP + 31) / 32;
  float2 pz[2][PF];
  auto prefetch = [&](int kf0, int nk) {
    const int ns = 2 * nk + T - 1;
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int r = 0; r < PF; ++r) {
        const int s = lane + 32 * r;
        const int i = 2 * kf0 + s;
        pz[q][r] = (s < ns && i < zlen_f) ? d.z[(long long)q * d.zlen + i] : make_float2(0.f, 0.f);
      }
  };
  auto store = [&](int kf0) {
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int r = 0; r < PF; ++r) {
        const int s = lane + 32 * r;
        if (s < NSP) {
          const int i = 2 * kf0 + s;
          const float2 rot = cmul(__ldg(&d.rot_hi[i >> 10]), __ldg(&d.rot_lo[i & (kRotLo - 1)]));
          sm.r[q * ChainSmem<T>::QS + (s & 3) * ChainSmem<T>::P4 + (s >> 2)] = cmul(pz[q][r], rot);
        }
      }
  };
  if (a < e) prefetch(a, min(kK, e - a));
  for (int k0 = a; k0 < e; k0 += kK) {
    const int nk = min(kK, e - k0);
    store(k0);
    __syncwarp();
    if (k0 + kK < e) prefetch(k0 + kK, min(kK, e - k0 - kK));
    float2 y[2][2];
    sub_block<T>(sm, nk, 1, d.mu_dd, d.R2, d.nl, y);
    const int k = k0 + 2 * lane;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      if (2 * lane + 1 < nk) {
        *reinterpret_cast<float4*>(&yb[(long long)p * (kYHist + d.F) + k]) = make_float4(y[p][0].x, y[p][0].y, y[p][1].x, y[p][1].y);
      } else if (2 * lane < nk) {
        yb[(long long)p * (kYHist + d.F) + k] = y[p][0];
      }
      if (d.hist_syms > 0) {
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const long long ka = hist_base + k + jj;
          if (2 * lane + jj < nk && ka < d.hist_syms) d.hist_y[(long long)p * d.hist_syms + ka] = y[p][jj];
        }
      }
    }
  }
  store_taps<T>(sm, chain);
}

template <int T>
__global__ void __launch_bounds__(256) mimo_kernel(RxDev d, FrameArgs fa, long long hist_base) {
  mimo_body<T>(d, fa, hist_base, own_block());
}

template <int T>
__global__ void __launch_bounds__(256) mimo_batch_kernel(BView v) {
  int fi;
  VBlock vb;
  if (!batch_block(v, fi, vb)) return;
  const BFrame& f = v.frames[fi];
  mimo_body<T>(f.d, f.fa, f.hist_base, vb);
}

// ---- launchers ------------------------------------------------------------

template <int T>
static cudaError_t launch_acq_t(const RxDev& d, const FrameArgs& fa, cudaStream_t s) {
  acq_kernel<T><<<1, 256, 0, s>>>(d, fa);
  return cudaGetLastError();
}

template <int T>
static cudaError_t launch_mimo_t(const RxDev& d, const FrameArgs& fa, cudaStream_t s) {
  const int nseg = (fa.Ff + d.S - 1) / d.S;
  const int nw = d.mimo_nw;
  mimo_kernel<T><<<(nseg + nw - 1) / nw, 32 * nw, nw * sizeof(ChainSmem<T>), s>>>(d, fa, fa.f * (long long)d.F);
  return cudaGetLastError();
}

#define RX_TAPS(X) X(3) X(5) X(7) X(9) X(11) X(13) X(15) X(17) X(19) X(21) X(23) X(25) X(27) X(29) X(31)

cudaError_t launch_acquire(const RxDev& d, const FrameArgs& fa, cudaStream_t s) {
  switch (d.T) {
#define RX_T(t) case t: return launch_acq_t<t>(d, fa, s);
    RX_TAPS(RX_T)
#undef RX_T
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_mimo(const RxDev& d, const FrameArgs& fa, cudaStream_t s) {
  switch (d.T) {
#define RX_T(t) case t: return launch_mimo_t<t>(d, fa, s);
    RX_TAPS(RX_T)
#undef RX_T
    default: return cudaErrorInvalidValue;
  }
}

// ---- batched launchers (every frame of v has d's tap count) ----------------

int mimo_grid_x(const RxDev& d, const FrameArgs& fa) {
  const int nseg = (fa.Ff + d.S - 1) / d.S;
  return (nseg + d.mimo_nw - 1) / d.mimo_nw;
}

cudaError_t launch_acquire_batch(const RxDev& d, const BView& v, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  switch (d.T) {
#define RX_T(t) case t: return launch_k(acq_batch_kernel<t>, blocks, 256, 0, s, v);
    RX_TAPS(RX_T)
#undef RX_T
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_mimo_batch(const RxDev& d, const BView& v, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  switch (d.T) {
#define RX_T(t) \
  case t: return launch_k(mimo_batch_kernel<t>, blocks, 32 * d.mimo_nw, d.mimo_nw * sizeof(ChainSmem<t>), s, v);
    RX_TAPS(RX_T)
#undef RX_T
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rx
