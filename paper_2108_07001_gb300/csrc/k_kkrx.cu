// The paper's KK receiver after the field reconstruction (Sec. II):
//
//   static equaliser + resampling: 100 % overlap-save at 4 samples per
//     symbol; block b (4-sps input [b N4/2 - N4/4, b N4/2 + 3N4/4), zero
//     outside the stream) is transformed with N4 points, cut to the
//     2-sps band (bins -N4/4 .. N4/4 - 1), multiplied by H (CD compensation
//     x RRC matched filter, 1/N4 folded in) and transformed back with N4/2
//     points; samples N4/8 .. 3N4/8 - 1 are the 2-sps outputs
//     [b N4/4, (b+1) N4/4);
//   widely-linear DD-LMS: y_k = sum_t h1[t] x[2k+t-1] + h2[t] conj(x[2k+t-1]),
//     t < 4, block-LMS over sub-blocks of 64 symbols (taps fixed inside a
//     sub-block, e = y - dec(y), h1 -= mu mean(e conj x), h2 -= mu mean(e x)),
//     one chain per segment of S symbols continued from frame to frame;
//   decisions and Gray demapping to packed bits.
//
// Kernel layout: the equaliser runs one block per output segment.  For
// N4 = 1024 the block is one warp: the field straight into registers, the
// one-warp four-step forward FFT, the band times H through shared memory
// into the 512-point inverse.  Otherwise N4/16 threads: 16-byte loads of
// two field samples when the block lies in the step's new field, the
// forward transform's band compacted in place; the inverse reuses the
// table of N4 at stride 2 in both forms.  The DD-LMS runs one warp per
// segment, two symbols per lane and sub-block, the sixteen gradient sums
// all-reduced by shuffles, decisions and bits in the same pass.
#include <cstring>

#include "fft_smem.cuh"
#include "fft_warp.cuh"
#include "kkrx_internal.h"

namespace rx {

__device__ __forceinline__ float2 kkrx_in(const KKEqArgs& a, long long i) {
  if (i < 0 || i >= a.in_end) return make_float2(0.f, 0.f);
  return i < a.new_start ? a.carry[i - a.carry_start] : a.in[i - a.new_start];
}

// Output segment a.seg0 + seg with N4 = 1024 by one warp: the block's 1024
// field samples straight into registers (lane n2 holds samples 32 n1 + n2),
// the one-warp forward FFT, the 2-sps band times H written in the order of
// a 512-point DFT into the freed transpose buffer, the shared-memory
// inverse transform.
__device__ __forceinline__ void kkeq_segment_1024w(const KKEqArgs& a, long long seg) {
  constexpr int N4 = 1024, L4 = 512, L2 = 256;
  __shared__ __align__(16) float2 t[32 * kWarpT];
  __shared__ float2 tw_s[2 * kTwSplit];
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < 2 * kTwSplit; i += 32) tw_s[i] = a.tw2[i];
  const long long b = a.seg0 + seg;
  const long long lo = b * L4 - N4 / 4;
  const long long off = lo - a.new_start;
  float2 v[32];
  if (off >= 0 && lo + N4 <= a.in_end) {
#pragma unroll
    for (int n1 = 0; n1 < 32; ++n1) v[n1] = __ldg(a.in + off + 32 * n1 + lane);
  } else {
#pragma unroll
    for (int n1 = 0; n1 < 32; ++n1) v[n1] = kkrx_in(a, lo + 32 * n1 + lane);
  }
  fft1024_warp_fwd(v, t);
  // lane k1 holds X[k1 + 32 k2]; the band is k2 < 8 (bins k1 + 32 k2) and
  // k2 >= 24 (bins k1 + 32 (k2 - 16) of the 512-point transform)
#pragma unroll
  for (int k2 = 0; k2 < 8; ++k2) t[swz(lane + 32 * k2)] = cmul(v[k2], a.H2[lane + 32 * k2]);
#pragma unroll
  for (int k2 = 24; k2 < 32; ++k2) t[swz(lane + 32 * (k2 - 16))] = cmul(v[k2], a.H2[lane + 32 * (k2 - 16)]);
  __syncthreads();
  fft_smem<N4 / 2, 32, true>(t, tw_s, 2);
  for (int n = lane; n < L2; n += 32) {
    const long long tt = b * L2 + n;
    if (tt < a.out_end) a.out[tt - a.out_base] = t[swz(N4 / 8 + n)];
  }
}

// Output segment a.seg0 + seg by one block of N4/16 threads.
template <int N4>
__device__ __forceinline__ void kkeq_segment_smem(const KKEqArgs& a, long long seg) {
  constexpr int NT = N4 / 16, L4 = N4 / 2, L2 = N4 / 4, NB2 = N4 / 2;
  static_assert(N4 / 2 == 8 * NT, "eight two-sample vectors per thread");
  __shared__ __align__(16) float2 buf[N4];
  __shared__ float2 tw_s[2 * kTwSplit];
  for (int i = threadIdx.x; i < 2 * kTwSplit; i += NT) tw_s[i] = a.tw2[i];
  const long long b = a.seg0 + seg;
  const long long lo = b * L4 - N4 / 4;
  const long long off = lo - a.new_start;
  if (off >= 0 && lo + N4 <= a.in_end && (off & 1) == 0 && (reinterpret_cast<uintptr_t>(a.in) & 15) == 0) {
    // the block lies in this step's field, 16-byte aligned: two samples per
    // load, N4 / 2 = 8 NT loads issued before any is used
    const float4* src = reinterpret_cast<const float4*>(a.in + off);
    float4 w[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) w[r] = __ldg(src + threadIdx.x + r * NT);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int v = threadIdx.x + r * NT;
      buf[swz(2 * v)] = make_float2(w[r].x, w[r].y);
      buf[swz(2 * v + 1)] = make_float2(w[r].z, w[r].w);
    }
  } else {
    for (int n = threadIdx.x; n < N4; n += NT) buf[swz(n)] = kkrx_in(a, lo + n);
  }
  __syncthreads();
  fft_smem<N4, NT, false>(buf, tw_s, 1);
  // the 2-sps band in the order of an N4/2-point DFT, times H
  constexpr int PER = NB2 / NT;
  float2 v[PER];
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int k2 = threadIdx.x + r * NT;
    v[r] = cmul(buf[swz(k2 < N4 / 4 ? k2 : k2 + N4 / 2)], a.H2[k2]);
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < PER; ++r) buf[swz(threadIdx.x + r * NT)] = v[r];
  __syncthreads();
  fft_smem<NB2, NT, true>(buf, tw_s, 2);
  for (int n = threadIdx.x; n < L2; n += NT) {
    const long long t = b * L2 + n;
    if (t < a.out_end) a.out[t - a.out_base] = buf[swz(N4 / 8 + n)];
  }
}

// Threads per equaliser block: one warp for N4 = 1024, else N4/16.
template <int N4>
constexpr int kkeq_threads() {
  return N4 == 1024 ? 32 : N4 / 16;
}

template <int N4>
__device__ __forceinline__ void kkeq_segment(const KKEqArgs& a, long long seg) {
  if constexpr (N4 == 1024) {
    kkeq_segment_1024w(a, seg);
  } else {
    kkeq_segment_smem<N4>(a, seg);
  }
}

// The one-warp form is capped at 128 registers (16 blocks per SM).
template <int N4>
__global__ void __launch_bounds__(kkeq_threads<N4>(), N4 == 1024 ? 16 : 1) kkeq_kernel(KKEqArgs a) {
  kkeq_segment<N4>(a, blockIdx.x);
}

// Many channels in one launch: block b belongs to the channel c with
// offs[c] <= b < offs[c + 1]; blocks past offs[nch] return at once.
template <int N4>
__global__ void __launch_bounds__(kkeq_threads<N4>(), N4 == 1024 ? 16 : 1) kkeq_batch_kernel(const KKEqBatchTable* __restrict__ t) {
  const long long b = blockIdx.x;
  if (b >= t->offs[t->nch]) return;
  int lo = 0, hi = t->nch;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (t->offs[mid] <= b) lo = mid;
    else hi = mid;
  }
  const KKEqArgs a = t->args[lo];
  kkeq_segment<N4>(a, b - t->offs[lo]);
}

template <typename T>
__device__ __forceinline__ void kkrx_tail_copy(const T* carry, long long carry_start, const T* in, long long new_start,
                                               long long keep_from, long long in_end, T* dst, long long i0,
                                               long long step) {
  const long long n = in_end - keep_from;
  for (long long i = i0; i < n; i += step) {
    const long long k = keep_from + i;
    dst[i] = k < new_start ? carry[k - carry_start] : in[k - new_start];
  }
}

template <typename T>
__global__ void kkrx_tail_kernel(const T* carry, long long carry_start, const T* in, long long new_start,
                                 long long keep_from, long long in_end, T* dst) {
  kkrx_tail_copy(carry, carry_start, in, new_start, keep_from, in_end, dst,
                 blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

// The equaliser carries of a batch, one block per channel (fewer than N4 samples each).
__global__ void kkeq_tail_batch_kernel(const KKEqBatchTable* __restrict__ t) {
  if ((int)blockIdx.x >= t->nch) return;
  const KKEqArgs& a = t->args[blockIdx.x];
  kkrx_tail_copy(a.carry, a.carry_start, a.in, a.new_start, t->keep_from[blockIdx.x], a.in_end,
                 t->carry_dst[blockIdx.x], threadIdx.x, blockDim.x);
}

// Nearest level per dimension (a value on a threshold takes the larger
// level) and its Gray label; levels +-1/sqrt2 (QPSK: - -> 1, + -> 0) or
// {-3, -1, 1, 3}/sqrt10 (16QAM: 00, 01, 11, 10).
template <bool Q16>
__device__ __forceinline__ float wl_level(float x, uint32_t& bits) {
  if (Q16) {
    const float t = 0.632455532033675866f;  // 2 / sqrt10
    const int l = (x >= -t) + (x >= 0.f) + (x >= t);
    bits = (uint32_t)(l ^ (l >> 1));
    return (float)(2 * l - 3) * 0.316227766016837933f;
  }
  const int l = x >= 0.f;
  bits = (uint32_t)(1 - l);
  return l ? 0.707106781186547524f : -0.707106781186547524f;
}

// Segment seg of a DD-LMS launch by one warp.
template <bool Q16>
__device__ __forceinline__ void wl_segment(const WLArgs& a, long long seg) {
  constexpr int BPS = Q16 ? 4 : 2;
  const int lane = threadIdx.x;
  const long long s0 = a.k_a + seg * a.seg;
  const long long s1 = min(s0 + a.seg, a.k_end);
  // taps (h1[0..3], h2[0..3]) kept in every lane
  float2 h[8];
  const float2* tin = a.taps_in + seg * a.taps_in_stride;
#pragma unroll
  for (int i = 0; i < 8; ++i) h[i] = tin[i];
  for (long long k0 = s0; k0 < s1; k0 += 64) {
    const int cnt = (int)min(64LL, s1 - k0);
    float g[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) g[i] = 0.f;
    uint32_t lbits = 0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int ks = 2 * lane + q;
      if (ks < cnt) {
        const long long k = k0 + ks;
        float2 X[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const long long i = 2 * k + t - 1;
          X[t] = (i < 0 || i >= a.n2) ? make_float2(0.f, 0.f) : a.x2[i - a.x2_base];
        }
        float yr = 0.f, yi = 0.f;
#pragma unroll
        for (int t = 0; t < 4; ++t) {  // h1 x + h2 conj(x)
          yr += h[t].x * X[t].x - h[t].y * X[t].y + h[4 + t].x * X[t].x + h[4 + t].y * X[t].y;
          yi += h[t].x * X[t].y + h[t].y * X[t].x + h[4 + t].y * X[t].x - h[4 + t].x * X[t].y;
        }
        uint32_t bI, bQ;
        const float dr = wl_level<Q16>(yr, bI), di = wl_level<Q16>(yi, bQ);
        const float er = yr - dr, ei = yi - di;
#pragma unroll
        for (int t = 0; t < 4; ++t) {  // e conj(x) and e x
          g[2 * t] += er * X[t].x + ei * X[t].y;
          g[2 * t + 1] += ei * X[t].x - er * X[t].y;
          g[8 + 2 * t] += er * X[t].x - ei * X[t].y;
          g[8 + 2 * t + 1] += ei * X[t].x + er * X[t].y;
        }
        lbits = (lbits << (2 * (BPS / 2))) | (bI << (BPS / 2)) | bQ;
        if (a.hist && k < a.hist_syms) a.hist[k] = make_float2(yr, yi);
      } else {
        lbits <<= BPS;
      }
    }
    // the lane's two symbols' bits: 4 (QPSK, a nibble) or 8 (16QAM, a byte)
    if (a.bits) {
      const long long bitpos = (k0 + 2 * lane - a.k_bits) * BPS;
      if (Q16) {
        if (2 * lane < cnt) a.bits[bitpos >> 3] = (uint8_t)lbits;
      } else {
        const uint32_t other = __shfl_down_sync(0xffffffffu, lbits, 1);
        if ((lane & 1) == 0 && 2 * lane < cnt) a.bits[bitpos >> 3] = (uint8_t)((lbits << 4) | other);
      }
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) g[i] += __shfl_xor_sync(0xffffffffu, g[i], o);
    }
    const float s = a.mu / (float)cnt;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      h[i].x -= s * g[2 * i];
      h[i].y -= s * g[2 * i + 1];
    }
  }
  if (lane < 8) a.taps_out[seg * 8 + lane] = h[lane];
}

template <bool Q16>
__global__ void __launch_bounds__(32) wl_kernel(WLArgs a) {
  wl_segment<Q16>(a, blockIdx.x);
}

// One DD-LMS step (acquisitions, or the i-th completed frame) of many
// channels: block b belongs to the entry e with offs[e] <= b < offs[e + 1].
template <bool Q16>
__global__ void __launch_bounds__(32) wl_batch_kernel(const WLBatchTable* __restrict__ t, int node) {
  const int ne = t->n[node];
  const long long b = blockIdx.x;
  if (b >= t->offs[node][ne]) return;
  int lo = 0, hi = ne;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (t->offs[node][mid] <= b) lo = mid;
    else hi = mid;
  }
  const WLArgs& a = t->args[node][lo];
  wl_segment<Q16>(a, b - t->offs[node][lo]);
}

// The moves of the remaining 2-sps samples to the other buffer, a block per channel.
__global__ void x2_shift_batch_kernel(const WLBatchTable* __restrict__ t) {
  if ((int)blockIdx.x >= t->nshift) return;
  const float2* src = t->shift_src[blockIdx.x];
  float2* dst = t->shift_dst[blockIdx.x];
  for (long long i = threadIdx.x; i < t->shift_n[blockIdx.x]; i += blockDim.x) dst[i] = src[i];
}

cudaError_t launch_kkeq(const KKEqArgs& a, int N4, long long nseg, cudaStream_t s) {
  if (nseg <= 0) return cudaSuccess;
  switch (N4) {
    case 1024: kkeq_kernel<1024><<<(unsigned)nseg, kkeq_threads<1024>(), 0, s>>>(a); break;
    case 2048: kkeq_kernel<2048><<<(unsigned)nseg, kkeq_threads<2048>(), 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t kkeq_batch_nodes(int N4, cudaKernelNodeParams* eq, cudaKernelNodeParams* tail) {
  std::memset(eq, 0, sizeof(*eq));
  std::memset(tail, 0, sizeof(*tail));
  switch (N4) {
    case 1024:
      eq->func = (void*)kkeq_batch_kernel<1024>;
      eq->blockDim = dim3(kkeq_threads<1024>());
      break;
    case 2048:
      eq->func = (void*)kkeq_batch_kernel<2048>;
      eq->blockDim = dim3(kkeq_threads<2048>());
      break;
    default: return cudaErrorInvalidValue;
  }
  tail->func = (void*)kkeq_tail_batch_kernel;
  tail->blockDim = dim3(256);
  return cudaSuccess;
}

cudaError_t launch_kkeq_tail(const float2* carry, long long carry_start, const float2* in, long long new_start,
                             long long keep_from, long long in_end, float2* dst, cudaStream_t s) {
  const long long n = in_end - keep_from;
  if (n <= 0) return cudaSuccess;
  kkrx_tail_kernel<float2><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(carry, carry_start, in, new_start, keep_from,
                                                                       in_end, dst);
  return cudaGetLastError();
}

cudaError_t launch_wl_batch(const WLBatchTable* t, int node, bool q16, long long blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  if (q16) wl_batch_kernel<true><<<(unsigned)blocks, 32, 0, s>>>(t, node);
  else wl_batch_kernel<false><<<(unsigned)blocks, 32, 0, s>>>(t, node);
  return cudaGetLastError();
}

cudaError_t launch_x2_shift_batch(const WLBatchTable* t, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  x2_shift_batch_kernel<<<(unsigned)n, 256, 0, s>>>(t);
  return cudaGetLastError();
}

cudaError_t launch_wl(const WLArgs& a, bool q16, long long nseg, cudaStream_t s) {
  if (nseg <= 0) return cudaSuccess;
  if (q16) wl_kernel<true><<<(unsigned)nseg, 32, 0, s>>>(a);
  else wl_kernel<false><<<(unsigned)nseg, 32, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace rx
