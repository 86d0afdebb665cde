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
// Kernel layout: one thread block per pair of adjacent segments (one warp
// with the one-warp FFT of fft_warp.cuh for N = 1024; N/16 threads with the
// shared-memory FFT otherwise).  The Hilbert transform has a real kernel, so
// the two real blocks go through one complex FFT pair as u_a + j u_b: the
// real part of the result is phi_a, the imaginary part phi_b.  u is staged once for the
// pair's 3L-sample union (16-byte loads of 8 codes when the union lies in
// the push), in log2 units: u2 = u / ln 2, |E| = 2^u2, and the factor
// ln 2 / pi rides on the Hilbert multiplier so the transform returns
// phi / pi.  The output takes one sincospi of phi / pi - 2 frac(nu t),
// where frac(nu t) comes from an exact 64-bit fixed-point product (nu
// quantised to 2^-64; no drift over the stream).
#include <algorithm>
#include <cstring>

#include "fft_smem.cuh"
#include "fft_warp.cuh"
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

// Threads per block: one warp for N = 1024 (the one-warp FFT), N/16 otherwise;
// the one-warp blocks are held to 128 registers so that 16 fit on an SM.
template <int N>
constexpr int kk_threads() { return N == 1024 ? 32 : N / 16; }
template <int N>
constexpr int kk_min_blocks() { return N == 1024 ? 16 : 1; }

// Dynamic shared memory: the FFT buffer (N float2; for N = 1024 the warp's
// 32 x 33 transpose buffer), then u of the pair's 3N/2-sample union.
template <int N>
constexpr size_t kk_smem_bytes() {
  return (N == 1024 ? (size_t)32 * kWarpT * 8 : (size_t)N * 8) + (size_t)3 * (N / 2) * 4;
}

// u2 = u / ln 2 of the codes of [lo, lo + U) into u_s by NT threads (16-byte
// loads of 8 codes when the union lies in the push).
template <int U, int NT>
__device__ __forceinline__ void kk_stage_u(const KKArgs& a, long long lo, float* u_s) {
  static_assert(U % (8 * NT) == 0, "whole 8-code vectors per thread");
  constexpr int PER = U / (8 * NT);
  auto u2_of = [&](float code) { return 0.5f * log2f(fmaxf(a.gain * (code - a.offset), a.i_min)); };
  const long long off = lo - a.new_start;
  if (off >= 0 && lo + U <= a.in_end && (off & 7) == 0 && (reinterpret_cast<uintptr_t>(a.in) & 15) == 0) {
    const int4* src = reinterpret_cast<const int4*>(a.in + off);
    float4* dst = reinterpret_cast<float4*>(u_s);
    int4 w[PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) w[r] = __ldg(src + threadIdx.x + r * NT);
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int v = threadIdx.x + r * NT;
      const int c[4] = {w[r].x, w[r].y, w[r].z, w[r].w};
      float f[8];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        f[2 * j] = u2_of((float)(short)(c[j] & 0xffff));
        f[2 * j + 1] = u2_of((float)(c[j] >> 16));
      }
      dst[2 * v] = make_float4(f[0], f[1], f[2], f[3]);
      dst[2 * v + 1] = make_float4(f[4], f[5], f[6], f[7]);
    }
  } else {
    for (int i = threadIdx.x; i < U; i += NT) {
      float code;
      u_s[i] = kk_code(a, lo + i, code) ? u2_of(code) : 0.f;
    }
  }
}

// The field of output sample t from phi / pi and u2.
__device__ __forceinline__ void kk_store(const KKArgs& a, long long t, float phi_pi, float u2) {
  const unsigned long long p = a.nu_fx * (unsigned long long)t;  // frac(nu t) in 2^-64
  const float cyc = (float)(p >> 40) * 0x1p-23f;                 // 2 frac(nu t)
  float sn, cs;
  sincospif(phi_pi - cyc, &sn, &cs);
  const float m = exp2f(u2);
  a.out[t - a.out_start] = make_float2(m * cs, m * sn);
}

// The pair of segments a.seg0 + 2 pair (+1) with N = 1024 by one warp: the
// two blocks' u as one complex input, the one-warp forward FFT, the Hilbert
// multiplier on the lane-k1 layout in registers, the inverse as the
// conjugate of the forward transform of the conjugate.
__device__ __forceinline__ void kk_pair_1024w(const KKArgs& a, long long pair) {
  constexpr int N = 1024, L = 512, U = 3 * L;
  extern __shared__ __align__(16) float2 kk_smem[];
  float2* t = kk_smem;
  float* u_s = reinterpret_cast<float*>(kk_smem + 32 * kWarpT);
  const int lane = threadIdx.x & 31;
  const long long seg = a.seg0 + 2LL * pair;
  const long long lo = seg * L - N / 4;
  kk_stage_u<U, 32>(a, lo, u_s);
  __syncwarp();
  float2 v[32];
#pragma unroll
  for (int n1 = 0; n1 < 32; ++n1) v[n1] = make_float2(u_s[32 * n1 + lane], u_s[32 * n1 + lane + L]);
  // pass 0: the forward transform, then -j sgn(k) ln2 / (pi N) on bin
  // k = lane + 32 k2 and the conjugate; pass 1: the forward transform again,
  // whose conjugate is the inverse (one copy of the transform's code)
  constexpr float s = 0.693147180559945309f / (3.14159265358979324f * (float)N);
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    fft1024_warp_fwd(v, t);
    if (pass == 0) {
#pragma unroll
      for (int k2 = 0; k2 < 32; ++k2) {
        const int k = lane + 32 * k2;
        const float2 x = v[k2];
        // conj(-j x) = (x.y, x.x), conj(+j x) = (-x.y, -x.x)
        v[k2] = (k == 0 || k == N / 2) ? make_float2(0.f, 0.f)
                : k < N / 2           ? make_float2(x.y * s, x.x * s)
                                      : make_float2(-x.y * s, -x.x * s);
      }
    }
  }
  // lane holds conj(x[lane + 32 n_b]); block samples N/4 .. 3N/4 - 1 are n_b = 8 .. 23:
  // phi_a = Re x = v.x, phi_b = Im x = -v.y
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll
    for (int nb = 8; nb < 24; ++nb) {
      const int n = lane + 32 * nb;
      const long long tt = (seg + h) * L + (n - N / 4);
      if (tt < a.out_end) kk_store(a, tt, h == 0 ? v[nb].x : -v[nb].y, u_s[h * L + n]);
    }
  }
}

// The pair of segments a.seg0 + 2 pair, a.seg0 + 2 pair + 1 by one block of
// N/16 threads with the shared-memory FFT (N = 2048, 4096).
template <int N>
__device__ __forceinline__ void kk_pair_smem(const KKArgs& a, long long pair) {
  constexpr int NT = N / 16, L = N / 2, U = 3 * L;
  extern __shared__ __align__(16) float2 kk_smem[];
  float2* buf = kk_smem;
  float* u_s = reinterpret_cast<float*>(kk_smem + N);
  __shared__ float2 tw_s[2 * kTwSplit];
  for (int i = threadIdx.x; i < 2 * kTwSplit; i += NT) tw_s[i] = a.tw2[i];
  const long long seg = a.seg0 + 2LL * pair;   // first segment of the pair
  const long long lo = seg * L - N / 4;        // stream index of u_s[0]
  kk_stage_u<U, NT>(a, lo, u_s);
  __syncthreads();
  for (int n = threadIdx.x; n < N; n += NT) buf[swz(n)] = make_float2(u_s[n], u_s[n + L]);
  __syncthreads();
  fft_smem<N, NT, false>(buf, tw_s, 1);
  // -j sgn(k) ln2 / (pi N): the inverse transform is unnormalised and u is in log2 units
  constexpr float s = 0.693147180559945309f / (3.14159265358979324f * (float)N);
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
      kk_store(a, t, h == 0 ? v.x : v.y, u_s[h * L + n + N / 4]);
    }
  }
}

template <int N>
__device__ __forceinline__ void kk_pair(const KKArgs& a, long long pair) {
  if constexpr (N == 1024) kk_pair_1024w(a, pair);
  else kk_pair_smem<N>(a, pair);
}

template <int N>
__global__ void __launch_bounds__(kk_threads<N>(), kk_min_blocks<N>()) kk_kernel(KKArgs a) {
  kk_pair<N>(a, blockIdx.x);
}

// Many channels in one launch: block b belongs to the channel c with
// offs[c] <= b < offs[c + 1] (uneven pushes give uneven counts); blocks
// past offs[nch] (the launch may be sized for more) return at once.
template <int N>
__global__ void __launch_bounds__(kk_threads<N>(), kk_min_blocks<N>()) kk_batch_kernel(const KKBatchTable* __restrict__ t) {
  const long long b = blockIdx.x;
  if (b >= t->offs[t->nch]) return;
  int lo = 0, hi = t->nch;  // offs[lo] <= b < offs[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (t->offs[mid] <= b) lo = mid;
    else hi = mid;
  }
  kk_pair<N>(t->args[lo], b - t->offs[lo]);
}

// New carry: codes [keep_from, in_end) from the old carry and the push.
__device__ __forceinline__ void kk_carry_copy(const KKArgs& a, int16_t* dst, long long keep_from, long long i0,
                                              long long step) {
  const long long n = a.in_end - keep_from;
  for (long long i = i0; i < n; i += step) {
    const long long k = keep_from + i;
    dst[i] = k < a.new_start ? a.carry[k - a.carry_start] : a.in[k - a.new_start];
  }
}

__global__ void kk_carry_kernel(KKArgs a, int16_t* dst, long long keep_from) {
  kk_carry_copy(a, dst, keep_from, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

// One block per channel of the table (a carry is shorter than N codes).
__global__ void kk_carry_batch_kernel(const KKBatchTable* __restrict__ t) {
  if ((int)blockIdx.x >= t->nch) return;
  const KKArgs a = t->args[blockIdx.x];
  kk_carry_copy(a, t->carry_dst[blockIdx.x], t->keep_from[blockIdx.x], threadIdx.x, blockDim.x);
}

template <int N>
static cudaError_t kk_attr() {
  constexpr size_t bytes = kk_smem_bytes<N>();
  if (bytes <= 48 * 1024) return cudaSuccess;
  static const cudaError_t attr = [] {  // opt in above the default (once per process)
    cudaError_t e = cudaFuncSetAttribute(kk_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kk_batch_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return e;
  }();
  return attr;
}

template <int N>
static cudaError_t launch_kk_t(const KKArgs& a, unsigned blocks, cudaStream_t s) {
  const cudaError_t e = kk_attr<N>();
  if (e != cudaSuccess) return e;
  kk_kernel<N><<<blocks, kk_threads<N>(), kk_smem_bytes<N>(), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_kk(const KKArgs& a, int N, long long nseg, cudaStream_t s) {
  if (nseg <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((nseg + 1) / 2);
  switch (N) {
    case 1024: return launch_kk_t<1024>(a, blocks, s);
    case 2048: return launch_kk_t<2048>(a, blocks, s);
    case 4096: return launch_kk_t<4096>(a, blocks, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t kk_batch_nodes(int N, cudaKernelNodeParams* field, cudaKernelNodeParams* carry) {
  std::memset(field, 0, sizeof(*field));
  std::memset(carry, 0, sizeof(*carry));
  cudaError_t e = cudaErrorInvalidValue;
  switch (N) {
    case 1024: e = kk_attr<1024>(); field->func = (void*)kk_batch_kernel<1024>; break;
    case 2048: e = kk_attr<2048>(); field->func = (void*)kk_batch_kernel<2048>; break;
    case 4096: e = kk_attr<4096>(); field->func = (void*)kk_batch_kernel<4096>; break;
    default: return cudaErrorInvalidValue;
  }
  field->blockDim = dim3(N == 1024 ? kk_threads<1024>() : N / 16);
  field->sharedMemBytes = (unsigned)(N == 1024 ? kk_smem_bytes<1024>() : N == 2048 ? kk_smem_bytes<2048>()
                                                                                    : kk_smem_bytes<4096>());
  carry->func = (void*)kk_carry_batch_kernel;
  carry->blockDim = dim3(256);
  return e;
}

cudaError_t launch_kk_carry(const KKArgs& a, int16_t* dst, long long keep_from, cudaStream_t s) {
  const long long n = a.in_end - keep_from;
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 1024);
  kk_carry_kernel<<<blocks, 256, 0, s>>>(a, dst, keep_from);
  return cudaGetLastError();
}

}  // namespace rx
