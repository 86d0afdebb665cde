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

// Sequential acquisition of the first frame (one warp).
template <int T>
__global__ void __launch_bounds__(32) acq_kernel(RxDev d, FrameArgs fa) {
  __shared__ ChainSmem<T> sm;
  const int lane = threadIdx.x;
  const int zlen_f = 2 * fa.Ff + 2 * d.c;
  const int n_acq = min(d.acq_syms, fa.Ff);
  // centre spike
  for (int pr = lane; pr < 2 * T; pr += 32) {
    const int q = pr / T, t = pr - q * T;
    const float one = (t == (T - 1) / 2) ? 1.f : 0.f;
    sm.w[q][t] = make_float4(q == 0 ? one : 0.f, 0.f, q == 1 ? one : 0.f, 0.f);
  }
  __syncwarp();
  const int cma_end = min(((d.cma_syms + kK - 1) / kK) * kK, n_acq);
  const int corr_lo = max(cma_end - 1024, 0);
  float cxr = 0.f, cxi = 0.f, pxx = 0.f, pyy = 0.f;
  bool was_cma = false;
  for (int k0 = 0; k0 < n_acq; k0 += kK) {
    const int nk = min(kK, n_acq - k0);
    const int mode = k0 < d.cma_syms ? 0 : 1;
    if (mode == 1 && was_cma) {
      const float sxy = warp_sum(cxr), syx = warp_sum(cxi);
      const float sxx = warp_sum(pxx), syy = warp_sum(pyy);
      const float den = sqrtf(sxx * syy);
      const float rho = den > 0.f ? sqrtf(sxy * sxy + syx * syx) / den : 0.f;
      if (rho > 0.5f) {
        float4 old0[1], old1[1];
        const int t = lane;
        if (t < T) {
          old0[0] = sm.w[0][T - 1 - t];
          old1[0] = sm.w[1][T - 1 - t];
        }
        __syncwarp();
        if (t < T) {
          // w[1][0][t] = -conj(w[0][1][T-1-t]);  w[1][1][t] = conj(w[0][0][T-1-t])
          float4 a = sm.w[0][t], b = sm.w[1][t];
          a.z = -old1[0].x;
          a.w = old1[0].y;
          b.z = old0[0].x;
          b.w = -old0[0].y;
          sm.w[0][t] = a;
          sm.w[1][t] = b;
        }
        __syncwarp();
        if (lane == 0) d.st->reinit = 1;
      }
    }
    stage_samples<T>(sm, d, k0, nk, zlen_f);
    __syncwarp();
    float2 y[2][2];
    sub_block<T>(sm, nk, mode, mode == 0 ? d.mu_cma : d.mu_dd, d.R2, d.nl, y);
    if (mode == 0) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int k = k0 + 2 * lane + j;
        if (2 * lane + j < nk && k >= corr_lo && k < cma_end) {
          const float2 a = y[0][j], b = y[1][j];
          cxr += a.x * b.x + a.y * b.y;  // a conj(b)
          cxi += a.y * b.x - a.x * b.y;
          pxx += a.x * a.x + a.y * a.y;
          pyy += b.x * b.x + b.y * b.y;
        }
      }
    }
    was_cma = mode == 0;
  }
  store_taps<T>(sm, d.w_acq);
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
  float2* yb = d.y + (long long)(fa.f & 1) * 2 * d.F;
  const int a = j * d.S, e = min(a + d.S, fa.Ff);
  for (int k0 = a; k0 < e; k0 += kK) {
    const int nk = min(kK, e - k0);
    stage_samples<T>(sm, d, k0, nk, zlen_f);
    __syncwarp();
    float2 y[2][2];
    sub_block<T>(sm, nk, 1, d.mu_dd, d.R2, d.nl, y);
    const int k = k0 + 2 * lane;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      if (2 * lane + 1 < nk) {
        *reinterpret_cast<float4*>(&yb[(long long)p * d.F + k]) = make_float4(y[p][0].x, y[p][0].y, y[p][1].x, y[p][1].y);
      } else if (2 * lane < nk) {
        yb[(long long)p * d.F + k] = y[p][0];
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
  acq_kernel<T><<<1, 32, 0, s>>>(d, fa);
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
