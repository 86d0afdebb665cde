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
// (Welch average over blocks and polarisations).
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
__global__ void __launch_bounds__(NT) cd_ols_kernel(RxDev d, FrameArgs fa) {
  extern __shared__ float2 buf[];
  __shared__ float scratch[NT / 32];
  __shared__ float2 tw_s[2 * kTwSplit];  // [hi | lo] two-level twiddle table
  for (int i = threadIdx.x; i < 2 * kTwSplit; i += NT) tw_s[i] = d.tw2[i];
  const int pol = blockIdx.y;
  const long long a = fa.s0 + (long long)blockIdx.x * d.L;
  const long long zlen_f = 2LL * fa.Ff + 2 * d.c;
  const int keep = (int)min((long long)d.L, fa.s0 + zlen_f - a);
  const long long lo = a - d.h;
  const long long rbase = (long long)pol * d.ring_cap;

  // load the window (halo included) from the ring
  for (int i = threadIdx.x; i < N; i += NT) {
    const long long n = lo + i;
    float2 v = make_float2(0.f, 0.f);
    if (n >= 0 && n < fa.n_valid) v = load_sample(d.ring, STOR, rbase + (n % d.ring_cap));
    buf[swz(i)] = v;
  }
  __syncthreads();
  fft_smem<N, NT, false>(buf, tw_s, 1);

  // filter; Godard sum over bin pairs Rs apart
  float gr = 0.f, gi = 0.f;
  for (int k = threadIdx.x; k < N / 2; k += NT) {
    float2 y0 = cmul(buf[swz(k)], __ldg(&d.Hf[k]));
    float2 y1 = cmul(buf[swz(k + N / 2)], __ldg(&d.Hf[k + N / 2]));
    const float2 p = cmulc(y0, y1);
    gr += p.x;
    gi += p.y;
    buf[swz(k)] = y0;
    buf[swz(k + N / 2)] = y1;
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
  __syncthreads();
  fft_smem<N, NT, true>(buf, tw_s, 1);

  // kept samples -> z; in-frame power
  float2* zp = d.z + (long long)pol * d.zlen + (a - fa.s0);
  float pw = 0.f;
  for (int i = threadIdx.x; i < keep; i += NT) {
    const float2 v = buf[swz(d.h + i)];
    zp[i] = v;
    const long long n = a + i;
    if (n >= fa.f0 && n < fa.f1) pw += v.x * v.x + v.y * v.y;
  }
  pw = block_sum<NT>(pw, scratch);
  if (threadIdx.x == 0) atomicAdd(&d.acc[fa.acc_slot].P, (double)pw);

  // 4th power of the even in-frame samples, zero padded to N/2
  const long long lo_n = max(a, fa.f0), hi_n = min(a + keep, fa.f1);
  const long long e0 = lo_n + (lo_n & 1);
  const int cnt = hi_n > e0 ? (int)((hi_n - e0 + 1) / 2) : 0;
  if (cnt == 0) return;
  constexpr int PER = (N / 2 + NT - 1) / NT;
  float2 u[PER];
  const int off = d.h + (int)(e0 - a);
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int idx = threadIdx.x + q * NT;
    float2 v = make_float2(0.f, 0.f);
    if (idx < cnt) {
      const float2 x = buf[swz(off + 2 * idx)];
      const float2 x2 = make_float2(x.x * x.x - x.y * x.y, 2.f * x.x * x.y);
      v = make_float2(x2.x * x2.x - x2.y * x2.y, 2.f * x2.x * x2.y);
    }
    u[q] = v;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int idx = threadIdx.x + q * NT;
    if (idx < N / 2) buf[swz(idx)] = u[q];
  }
  __syncthreads();
  fft_smem<N / 2, NT, false>(buf, tw_s, 2);
  for (int k = threadIdx.x; k < N / 2; k += NT) {
    const float2 v = buf[swz(k)];
    atomicAdd(&d.psd[(long long)fa.acc_slot * (N / 2) + k], (double)(v.x * v.x + v.y * v.y));
  }
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
__global__ void __launch_bounds__(1024) est_kernel(RxDev d, FrameArgs fa, int mode) {
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ double sh[4];
  const int tid = threadIdx.x;
  const FrameAcc* acc = d.acc + fa.acc_slot;
  const double* psd = d.psd + (long long)fa.acc_slot * (d.N / 2);
  const double C_re = acc->C[0], C_im = acc->C[1];
  const double resid = (C_re == 0.0 && C_im == 0.0) ? 0.0 : -atan2(C_im, C_re) / (2.0 * M_PI * d.Rs);
  double tau_next;
  if (mode == 1) {
    const EstState es = d.es[fa.f & 1];
    const int n2 = d.N / 2;
    double best = -1.0;
    int bi = 0;
    for (int k = tid; k < n2; k += 1024) {
      const double v = psd[k];
      if (v > best) { best = v; bi = k; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
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
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
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
      if (blockIdx.x == 0) {
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
    for (int l = blockIdx.x * 1024 + tid; l < kRotLo; l += gridDim.x * 1024) {
      float s, c;
      sincosf(omf * (float)l, &s, &c);
      d.rot_lo[l] = make_float2(c, -s);
    }
    const int nhi = (d.zlen + kRotLo - 1) / kRotLo;
    for (int hh = blockIdx.x * 1024 + tid; hh < nhi; hh += gridDim.x * 1024) {
      const double ph = wrap_pi(theta + om * (double)(hh * kRotLo - d.c));
      float s, c;
      sincosf((float)ph, &s, &c);
      d.rot_hi[hh] = make_float2((float)gain * c, -(float)gain * s);
    }
    // clear the other accumulator slot for the next frame's CD pass
    double* psd_n = d.psd + (long long)((fa.f + 1) & 1) * (d.N / 2);
    for (int k = blockIdx.x * 1024 + tid; k < n2; k += gridDim.x * 1024) psd_n[k] = 0.0;
    if (blockIdx.x == 0 && tid == 0) {
      FrameAcc* an = d.acc + ((fa.f + 1) & 1);
      an->C[0] = an->C[1] = an->P = 0.0;
    }
  } else {
    tau_next = resid;
    if (blockIdx.x == 0 && tid == 0) {
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
  for (int k = blockIdx.x * 1024 + tid; k < d.N; k += gridDim.x * 1024) {
    const int kk = k < d.N / 2 ? k : k - d.N;
    float s, c;
    sincospif((float)kk * u2, &s, &c);
    d.Hf[k] = cmul(d.Hs[k], make_float2(c, s));
  }
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
  return e;
}

// Opt-in to the dynamic shared memory of every FFT size (once per process).
cudaError_t cd_set_attributes() {
  cudaError_t e = cd_attr_n<1024, 256>();
  if (e == cudaSuccess) e = cd_attr_n<2048, 256>();
  if (e == cudaSuccess) e = cd_attr_n<4096, 256>();
  if (e == cudaSuccess) e = cd_attr_n<8192, 512>();
  if (e == cudaSuccess) e = cd_attr_n<16384, 1024>();
  return e;
}

cudaError_t launch_cd(const RxDev& d, const FrameArgs& fa, cudaStream_t s) {
  switch (d.N) {
    case 1024: return launch_cd_n<1024, 256>(d, fa, s);
    case 2048: return launch_cd_n<2048, 256>(d, fa, s);
    case 4096: return launch_cd_n<4096, 256>(d, fa, s);
    case 8192: return launch_cd_n<8192, 512>(d, fa, s);
    case 16384: return launch_cd_n<16384, 1024>(d, fa, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_est(const RxDev& d, const FrameArgs& fa, int mode, cudaStream_t s) {
  const int nb = max(1, min(16, (d.N + 1023) / 1024));
  est_kernel<<<nb, 1024, 0, s>>>(d, fa, mode);
  return cudaGetLastError();
}

}  // namespace rx
