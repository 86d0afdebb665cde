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
// mod 4 (conflict-free for the lane stride of 4); taps are stored as
// float4 {w[0][q][t], w[1][q][t]} and read as broadcasts.
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
  float2 r[2][4 * P4];
  float4 w[2][T];
  float4 e[kK];
};

template <int T>
__device__ __forceinline__ float2 sm_r(const ChainSmem<T>& sm, int q, int s) {
  return sm.r[q][(s & 3) * ChainSmem<T>::P4 + (s >> 2)];
}

// Stage samples [2 kf0, 2 kf0 + 2 nk + T - 1) of the frame buffer, rotated.
template <int T>
__device__ __forceinline__ void stage_samples(ChainSmem<T>& sm, const RxDev& d, int kf0, int nk, int zlen_f) {
  const int lane = threadIdx.x & 31;
  const int ns = 2 * nk + T - 1;
  for (int q = 0; q < 2; ++q) {
    const float2* zq = d.z + (long long)q * d.zlen;
    for (int s = lane; s < ns; s += 32) {
      const int i = 2 * kf0 + s;
      float2 v = make_float2(0.f, 0.f);
      if (i < zlen_f) {
        const float2 rot = cmul(__ldg(&d.rot_hi[i >> 10]), __ldg(&d.rot_lo[i & (kRotLo - 1)]));
        v = cmul(zq[i], rot);
      }
      sm.r[q][(s & 3) * ChainSmem<T>::P4 + (s >> 2)] = v;
    }
  }
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
    for (int k = 0; k < nk; ++k) {
      const float4 ee = sm.e[k];
      const float2 x = sm_r(sm, q, 2 * k + t);
      // e * conj(x)
      g0x = fmaf(ee.x, x.x, fmaf(ee.y, x.y, g0x));
      g0y = fmaf(ee.y, x.x, fmaf(-ee.x, x.y, g0y));
      g1x = fmaf(ee.z, x.x, fmaf(ee.w, x.y, g1x));
      g1y = fmaf(ee.w, x.x, fmaf(-ee.z, x.y, g1y));
    }
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
// block).  FIR: thread (k, p, q) = (t >> 2, (t >> 1) & 1, t & 1) forms
// sum_t w[p][q][t] r_q[2k + t] and the q pair is added with a shuffle.
// Gradient: thread (combo, quarter) sums e_p[k] conj(r_q[2k + t]) over a
// quarter of the sub-block, quarters are added with shuffles.  The next
// sub-block's samples are loaded into registers while the gradient runs.
template <int T>
__global__ void __launch_bounds__(256) acq_kernel(RxDev d, FrameArgs fa) {
  constexpr int NS = 2 * kK + T - 1;      // samples per pol per sub-block
  constexpr int NLD = (2 * NS + 255) / 256;
  __shared__ float2 r_s[2][NS + 1];
  __shared__ float2 w_s[2][2][T];         // [p][q][t]
  __shared__ float2 e_s[2][kK];
  __shared__ float red_s[8][4];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int zlen_f = 2 * fa.Ff + 2 * d.c;
  const int n_acq = min(d.acq_syms, fa.Ff);
  for (int i = tid; i < 4 * T; i += 256) {
    const int p = i / (2 * T), q = (i / T) & 1, t = i % T;
    w_s[p][q][t] = make_float2((p == q && t == (T - 1) / 2) ? 1.f : 0.f, 0.f);
  }
  // prefetch registers for one sub-block's samples
  float2 pre[NLD];
  auto load = [&](int kf0, int nk) {
    const int ns = 2 * nk + T - 1;
#pragma unroll
    for (int j = 0; j < NLD; ++j) {
      const int i = tid + j * 256;
      const int q = i / NS, s = i - q * NS;
      float2 v = make_float2(0.f, 0.f);
      if (q < 2 && s < ns) {
        const int n = 2 * kf0 + s;
        if (n < zlen_f) {
          const float2 rot = cmul(__ldg(&d.rot_hi[n >> 10]), __ldg(&d.rot_lo[n & (kRotLo - 1)]));
          v = cmul(d.z[(long long)q * d.zlen + n], rot);
        }
      }
      pre[j] = v;
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int j = 0; j < NLD; ++j) {
      const int i = tid + j * 256;
      const int q = i / NS, s = i - q * NS;
      if (q < 2) r_s[q][s] = pre[j];
    }
  };
  const int cma_end = min(((d.cma_syms + kK - 1) / kK) * kK, n_acq);
  const int corr_lo = max(cma_end - 1024, 0);
  float cxr = 0.f, cxi = 0.f, pxx = 0.f, pyy = 0.f;
  bool was_cma = false;
  load(0, min(kK, n_acq));
  store();
  __syncthreads();
  const int kk = tid >> 2, pp = (tid >> 1) & 1, qq = tid & 1;
  for (int k0 = 0; k0 < n_acq; k0 += kK) {
    const int nk = min(kK, n_acq - k0);
    const int mode = k0 < d.cma_syms ? 0 : 1;
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
          a = w_s[0][1][T - 1 - tid];  // w_xy reversed
          b2 = w_s[0][0][T - 1 - tid];  // w_xx reversed
        }
        __syncthreads();
        if (tid < T) {
          w_s[1][0][tid] = make_float2(-a.x, a.y);   // -conj(w_xy[T-1-t])
          w_s[1][1][tid] = make_float2(b2.x, -b2.y);  // conj(w_xx[T-1-t])
        }
        if (tid == 0) d.st->reinit = 1;
      }
      __syncthreads();
    }
    // ---- FIR
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const float2 w = w_s[pp][qq][t], x = r_s[qq][2 * kk + t];
      acc.x = fmaf(w.x, x.x, fmaf(-w.y, x.y, acc.x));
      acc.y = fmaf(w.x, x.y, fmaf(w.y, x.x, acc.y));
    }
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
    const float2 y = acc;  // y_pp[kk]
    const bool valid = kk < nk;
    // ---- error
    float2 e;
    if (mode == 0) {
      e = cscale(y, y.x * y.x + y.y * y.y - d.R2);
      // correlation of the two outputs for the singularity check
      const float2 yo = make_float2(__shfl_xor_sync(0xffffffffu, y.x, 2), __shfl_xor_sync(0xffffffffu, y.y, 2));
      const int k = k0 + kk;
      if (valid && pp == 0 && qq == 0 && k >= corr_lo && k < cma_end) {
        cxr += y.x * yo.x + y.y * yo.y;
        cxi += y.y * yo.x - y.x * yo.y;
        pxx += y.x * y.x + y.y * y.y;
        pyy += yo.x * yo.x + yo.y * yo.y;
      }
    } else {
      float s0x = 0.f, s0y = 0.f, s1x = 0.f, s1y = 0.f;
      if (valid && qq == 0) {
        const float2 a2 = make_float2(y.x * y.x - y.y * y.y, 2.f * y.x * y.y);
        const float a4x = a2.x * a2.x - a2.y * a2.y, a4y = 2.f * a2.x * a2.y;
        if (pp == 0) { s0x = a4x; s0y = a4y; } else { s1x = a4x; s1y = a4y; }
      }
      s0x = warp_sum(s0x); s0y = warp_sum(s0y); s1x = warp_sum(s1x); s1y = warp_sum(s1y);
      if (lane == 0) { red_s[warp][0] = s0x; red_s[warp][1] = s0y; red_s[warp][2] = s1x; red_s[warp][3] = s1y; }
      __syncthreads();
      float sx = 0.f, sy = 0.f;
      for (int w = 0; w < 8; ++w) { sx += red_s[w][2 * pp]; sy += red_s[w][2 * pp + 1]; }
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
    // prefetch the next sub-block while the gradient runs
    const int k1 = k0 + kK;
    if (k1 < n_acq) load(k1, min(kK, n_acq - k1));
    // ---- gradient: combo = (p, q, t), quarter of the sub-block
    const float step = (mode == 0 ? d.mu_cma : d.mu_dd) / (float)nk;
    for (int c0 = 0; c0 < 16 * T; c0 += 256) {  // every lane runs every iteration (shuffles)
      const int c = c0 + tid;
      const bool act = c < 16 * T;
      const int combo = act ? c >> 2 : 0, quarter = c & 3;
      const int p = combo / (2 * T), q = (combo / T) & 1, t = combo % T;
      float gx = 0.f, gy = 0.f;
      const int ka = quarter * 16, kb = act ? min(ka + 16, nk) : ka;
      for (int k = ka; k < kb; ++k) {
        const float2 ee = e_s[p][k], x = r_s[q][2 * k + t];
        gx = fmaf(ee.x, x.x, fmaf(ee.y, x.y, gx));
        gy = fmaf(ee.y, x.x, fmaf(-ee.x, x.y, gy));
      }
      gx += __shfl_xor_sync(0xffffffffu, gx, 1);
      gy += __shfl_xor_sync(0xffffffffu, gy, 1);
      gx += __shfl_xor_sync(0xffffffffu, gx, 2);
      gy += __shfl_xor_sync(0xffffffffu, gy, 2);
      if (act && quarter == 0) {
        float2 w = w_s[p][q][t];
        w.x -= step * gx;
        w.y -= step * gy;
        w_s[p][q][t] = w;
      }
    }
    __syncthreads();
    if (k1 < n_acq) {
      store();
      __syncthreads();
    }
    was_cma = mode == 0;
  }
  for (int i = tid; i < 4 * T; i += 256) {
    const int p = i / (2 * T), q = (i / T) & 1, t = i % T;
    d.w_acq[(p * 2 + q) * T + t] = w_s[p][q][t];
  }
}

// All segments of one frame, one warp per segment.
template <int T>
__global__ void __launch_bounds__(128) mimo_kernel(RxDev d, FrameArgs fa, long long hist_base) {
  __shared__ ChainSmem<T> sms[4];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * 4 + wib;
  const int nseg = (fa.Ff + d.S - 1) / d.S;
  if (j >= nseg) return;
  ChainSmem<T>& sm = sms[wib];
  const int zlen_f = 2 * fa.Ff + 2 * d.c;
  float2* chain = d.chains + (long long)j * 4 * T;
  load_taps<T>(sm, fa.f == 0 ? d.w_acq : chain);
  // frame f's equalised symbols go to buffer f % 2 after a copy of the last
  // kYHist symbols of frame f-1 (zeros for the first frame)
  float2* yb = d.y + (long long)(fa.f & 1) * 2 * (kYHist + d.F);
  if (blockIdx.x == 0 && wib == 0) {
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
          sm.r[q][(s & 3) * ChainSmem<T>::P4 + (s >> 2)] = cmul(pz[q][r], rot);
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

// ---- launchers ------------------------------------------------------------

template <int T>
static cudaError_t launch_acq_t(const RxDev& d, const FrameArgs& fa, cudaStream_t s) {
  acq_kernel<T><<<1, 256, 0, s>>>(d, fa);
  return cudaGetLastError();
}

template <int T>
static cudaError_t launch_mimo_t(const RxDev& d, const FrameArgs& fa, cudaStream_t s) {
  const int nseg = (fa.Ff + d.S - 1) / d.S;
  mimo_kernel<T><<<(nseg + 3) / 4, 128, 0, s>>>(d, fa, fa.f * (long long)d.F);
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

}  // namespace rx
