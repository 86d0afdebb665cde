// Kramers-Kronig front end (paper Sec. II): 12-bit ADC codes of the
// photocurrent to the reconstructed, downshifted optical field.
//
//   I_t = gain (code_t - offset);  u_t = ln(max(I_t, gain / 2)) / 2
//   phi = Hilbert transform of u, 100 % overlap-save blocks of N samples:
//         segment b = outputs [b L, (b+1) L), L = N/2, from the block of u
//         over [b L - N/4, b L + 3N/4) (u = 0 outside the stream); the
//         block's DFT times -j sgn(k) (0 at k = 0, N/2), transformed back,
//         samples N/4 .. 3N/4 - 1
//   E_t = exp(u_t + j phi_t) exp(-j 2 pi nu t),  nu = f_shift / f_s
//
// Kernel layout: one thread block (N/16 threads) per pair of adjacent
// segments.  The Hilbert transform has a real kernel, so the two real
// blocks go through one complex FFT pair as u_a + j u_b: the real part of
// the result is phi_a, the imaginary part phi_b.  u is staged once for the
// pair's 3L-sample union; the output takes exp(u) and one sincos of
// phi - 2 pi frac(nu t), where frac(nu t) comes from an exact 64-bit
// fixed-point product (nu quantised to 2^-64; no drift over the stream).
#include "fft_smem.cuh"
#include "kk_internal.h"

namespace rx {

// Sample i of the stream: carry codes (absolute index carry_start..) before
// new_start, then the new push; absent (not finite data) outside
// [0, in_end).
__device__ __forceinline__ bool kk_code(const KKArgs& a, long long i, float& code) {
  if (i < 0 || i >= a.in_end) return false;
  code = i < a.new_start ? (float)a.carry[i - a.carry_start] : (float)a.in[i - a.new_start];
  return true;
}

template <int N>
__global__ void __launch_bounds__(N / 16) kk_kernel(KKArgs a) {
  constexpr int NT = N / 16, L = N / 2, U = 3 * L;
  __shared__ __align__(16) float2 buf[N];
  __shared__ float u_s[U];
  __shared__ float2 tw_s[2 * kTwSplit];
  for (int i = threadIdx.x; i < 2 * kTwSplit; i += NT) tw_s[i] = a.tw2[i];

  const long long seg = a.seg0 + 2LL * blockIdx.x;   // first segment of the pair
  const long long lo = seg * L - N / 4;              // stream index of u_s[0]
  for (int i = threadIdx.x; i < U; i += NT) {
    float code;
    const bool in = kk_code(a, lo + i, code);
    u_s[i] = in ? 0.5f * logf(fmaxf(a.gain * (code - a.offset), a.i_min)) : 0.f;
  }
  __syncthreads();
  for (int n = threadIdx.x; n < N; n += NT) buf[swz(n)] = make_float2(u_s[n], u_s[n + L]);
  __syncthreads();
  fft_smem<N, NT, false>(buf, tw_s, 1);
  // -j sgn(k) / N (the inverse transform is unnormalised)
  const float s = 1.f / (float)N;
  for (int k = threadIdx.x; k < N; k += NT) {
    const float2 v = buf[swz(k)];
    float2 r;
    if (k == 0 || k == N / 2) r = make_float2(0.f, 0.f);
    else if (k < N / 2) r = make_float2(v.y * s, -v.x * s);   // * (-j)
    else r = make_float2(-v.y * s, v.x * s);                  // * (+j)
    buf[swz(k)] = r;
  }
  __syncthreads();
  fft_smem<N, NT, true>(buf, tw_s, 1);
  // outputs: segment seg from the real parts, seg + 1 from the imaginary parts
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    for (int n = threadIdx.x; n < L; n += NT) {
      const long long t = (seg + h) * L + n;
      if (t >= a.out_end) break;
      const float2 v = buf[swz(n + N / 4)];
      const float phi = h == 0 ? v.x : v.y;
      const float u = u_s[h * L + n + N / 4];
      const unsigned long long p = a.nu_fx * (unsigned long long)t;  // frac(nu t) in 2^-64
      const float cyc = (float)(p >> 40) * 0x1p-24f;
      float sn, cs;
      sincosf(phi - 6.28318530717958648f * cyc, &sn, &cs);
      const float m = expf(u);
      a.out[t - a.out_start] = make_float2(m * cs, m * sn);
    }
  }
}

// New carry: codes [keep_from, in_end) from the old carry and the push.
__global__ void kk_carry_kernel(KKArgs a, int16_t* dst, long long keep_from) {
  const long long n = a.in_end - keep_from;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long k = keep_from + i;
    dst[i] = k < a.new_start ? a.carry[k - a.carry_start] : a.in[k - a.new_start];
  }
}

cudaError_t launch_kk(const KKArgs& a, int N, long long nseg, cudaStream_t s) {
  if (nseg <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((nseg + 1) / 2);
  switch (N) {
    case 1024: kk_kernel<1024><<<blocks, 64, 0, s>>>(a); break;
    case 2048: kk_kernel<2048><<<blocks, 128, 0, s>>>(a); break;
    case 4096: kk_kernel<4096><<<blocks, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_kk_carry(const KKArgs& a, int16_t* dst, long long keep_from, cudaStream_t s) {
  const long long n = a.in_end - keep_from;
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 1024);
  kk_carry_kernel<<<blocks, 256, 0, s>>>(a, dst, keep_from);
  return cudaGetLastError();
}

}  // namespace rx
