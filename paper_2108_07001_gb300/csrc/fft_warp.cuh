// A 1024-point complex FFT by one warp: the four-step decomposition
// 1024 = 32 x 32 with each lane's 32-point DFT in registers and one
// transpose through shared memory.
//
// Forward, n = 32 n1 + n2, k = k1 + 32 k2:
//   X[k1 + 32 k2] = sum_n2 W32^(n2 k2) W1024^(n2 k1) sum_n1 x[32 n1 + n2] W32^(n1 k1)
// lane n2 transforms its column over n1 (giving k1), multiplies by
// W1024^(n2 k1), the warp transposes, lane k1 transforms over n2 (giving
// k2): lane k1 ends holding X[k1 + 32 k2] for k2 = 0..31.
// Inverse from that layout, n = n_a + 32 n_b:
//   x[n_a + 32 n_b] = sum_k1 W32^-(n_b k1) W1024^-(n_a k1) sum_k2 X[k1 + 32 k2] W32^-(n_a k2)
// lane k1 transforms over k2 (giving n_a), multiplies by W1024^-(n_a k1),
// the warp transposes, lane n_a transforms over k1 (giving n_b): lane n_a
// ends holding x[n_a + 32 n_b] for n_b = 0..31 (unnormalised).
// The transpose buffer is 32 rows of 33 float2 (the pad keeps each 16-lane
// phase of a 64-bit access on distinct banks).
#pragma once
#include "fft_smem.cuh"

namespace rx {

constexpr int kWarpT = 33;  // padded transpose row (float2)

// exp(-+2 pi i k / 32), k < 16 (forward: minus).
template <bool INV>
__device__ __forceinline__ float2 w32(int k) {
  constexpr float c[16] = {1.f, 0.98078528040323043f, 0.92387953251128674f, 0.83146961230254524f,
                           0.70710678118654752f, 0.55557023301960222f, 0.38268343236508978f, 0.19509032201612827f,
                           0.f, -0.19509032201612827f, -0.38268343236508978f, -0.55557023301960222f,
                           -0.70710678118654752f, -0.83146961230254524f, -0.92387953251128674f, -0.98078528040323043f};
  constexpr float s[16] = {0.f, 0.19509032201612827f, 0.38268343236508978f, 0.55557023301960222f,
                           0.70710678118654752f, 0.83146961230254524f, 0.92387953251128674f, 0.98078528040323043f,
                           1.f, 0.98078528040323043f, 0.92387953251128674f, 0.83146961230254524f,
                           0.70710678118654752f, 0.55557023301960222f, 0.38268343236508978f, 0.19509032201612827f};
  return make_float2(c[k], INV ? s[k] : -s[k]);
}

// 32-point DFT in natural order: two 16-point DFTs of the even and odd
// samples, X[k] = E[k] + W32^k O[k], X[k + 16] = E[k] - W32^k O[k].
template <bool INV>
__device__ __forceinline__ void dft32(float2 (&v)[32]) {
  float2 e[16], o[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    e[i] = v[2 * i];
    o[i] = v[2 * i + 1];
  }
  dft<16, INV>(e);
  dft<16, INV>(o);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const float2 t = k == 0 ? o[0] : cmul(o[k], w32<INV>(k));
    v[k] = cadd(e[k], t);
    v[k + 16] = csub(e[k], t);
  }
}

// v[k] *= w^k for k < 32, w = exp(-+2 pi i m / 1024) (forward: minus), the
// powers from w^(k mod 8) and w^(8 (k / 8)) (each a product of at most four
// correctly rounded values).
template <bool INV>
__device__ __forceinline__ void twiddle32(float2 (&v)[32], int m) {
  float s, c;
  sincospif((float)m / 512.f, &s, &c);
  const float2 w = make_float2(c, INV ? s : -s);
  float2 lo[8], hi[4];
  lo[0] = make_float2(1.f, 0.f);
#pragma unroll
  for (int i = 1; i < 8; ++i) lo[i] = cmul(lo[i - 1], w);
  hi[0] = make_float2(1.f, 0.f);
  hi[1] = cmul(lo[7], w);  // w^8
  hi[2] = cmul(hi[1], hi[1]);
  hi[3] = cmul(hi[2], hi[1]);
#pragma unroll
  for (int k = 1; k < 32; ++k) v[k] = cmul(v[k], (k >> 3) == 0 ? lo[k & 7] : cmul(lo[k & 7], hi[k >> 3]));
}

// Transpose through t (32 x kWarpT float2): lane writes its v[j] to row j,
// column lane; after the barrier lane reads row lane, columns 0..31.
__device__ __forceinline__ void warp_transpose32(float2 (&v)[32], float2* t) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < 32; ++j) t[j * kWarpT + lane] = v[j];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = t[lane * kWarpT + j];
  __syncwarp();
}

// Forward: on entry lane n2 holds v[n1] = x[32 n1 + n2]; on return lane k1
// holds v[k2] = X[k1 + 32 k2].  The two 32-point steps share one body (a
// loop that is not unrolled keeps the code small for the instruction
// cache).  The unnormalised inverse is conj(forward(conj(.))) with the same
// layouts: the input's lane k1, register k2 is index k1 + 32 k2 = 32 k2 + k1,
// the forward's input convention, and the result's lane n_a, register n_b
// is x[n_a + 32 n_b].
__device__ __forceinline__ void fft1024_warp_fwd(float2 (&v)[32], float2* t) {
  const int lane = threadIdx.x & 31;
#pragma unroll 1
  for (int step = 0; step < 2; ++step) {
    dft32<false>(v);
    if (step == 0) {
      twiddle32<false>(v, lane);
      warp_transpose32(v, t);
    }
  }
}

}  // namespace rx
