// In-shared-memory complex FFT for one thread block (power-of-two sizes).
//
// Stockham auto-sort formulation, decimation in time: a pass with radix R
// over sub-transforms of length Ns reads element j + r N/R, multiplies it by
// exp(-+2 pi i r (j mod Ns) / (Ns R)), runs an R-point DFT in registers and
// writes element (j / Ns) Ns R + (j mod Ns) + r Ns.  Passes use radix 16
// until fewer than 16 remain, then one radix 2/4/8 pass; the output is in
// natural order.  Each pass reads all its inputs before a barrier and writes
// after it, so one buffer suffices.  Shared-memory addresses are swizzled
// (i ^ ((i >> 4) & 15)) so the strided writes of the early passes do not
// collide in banks; every access to an FFT buffer goes through swz().
#pragma once
#include "rx_internal.cuh"

namespace rx {

constexpr int kTwSplit = 128;  // two-level twiddle split (N <= 128 * 128)

__device__ __forceinline__ int swz(int i) { return i ^ ((i >> 4) & 15); }

// exp(-2 pi i m / 16) for forward (INV = false), conjugate for inverse.
template <int M, bool INV>
__device__ __forceinline__ float2 w16() {
  constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, r2 = 0.70710678118654752f;
  constexpr int m = M & 15;
  constexpr float cs[16] = {1.f, c1, r2, s1, 0.f, -s1, -r2, -c1, -1.f, -c1, -r2, -s1, 0.f, s1, r2, c1};
  constexpr float sn[16] = {0.f, s1, r2, c1, 1.f, c1, r2, s1, 0.f, -s1, -r2, -c1, -1.f, -c1, -r2, -s1};
  return make_float2(cs[m], INV ? sn[m] : -sn[m]);
}

template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {  // a * (-i) forward, a * (+i) inverse
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& a, float2& b, float2& c, float2& d) {
  float2 t0 = cadd(a, c), t1 = csub(a, c), t2 = cadd(b, d), t3 = mul_mi<INV>(csub(b, d));
  a = cadd(t0, t2);
  c = csub(t0, t2);
  b = cadd(t1, t3);
  d = csub(t1, t3);
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2 (&v)[R]);

template <>
__device__ __forceinline__ void dft<2, false>(float2 (&v)[2]) { dft2<false>(v[0], v[1]); }
template <>
__device__ __forceinline__ void dft<2, true>(float2 (&v)[2]) { dft2<true>(v[0], v[1]); }
template <>
__device__ __forceinline__ void dft<4, false>(float2 (&v)[4]) { dft4<false>(v[0], v[1], v[2], v[3]); }
template <>
__device__ __forceinline__ void dft<4, true>(float2 (&v)[4]) { dft4<true>(v[0], v[1], v[2], v[3]); }

// 8 = 2 (outer) x 4: X[k] = E[k] + W8^k O[k], X[k+4] = E[k] - W8^k O[k].
template <bool INV>
__device__ __forceinline__ void dft8_impl(float2 (&v)[8]) {
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  o1 = cmul(o1, w16<2, INV>());
  o2 = cmul(o2, w16<4, INV>());
  o3 = cmul(o3, w16<6, INV>());
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}
template <>
__device__ __forceinline__ void dft<8, false>(float2 (&v)[8]) { dft8_impl<false>(v); }
template <>
__device__ __forceinline__ void dft<8, true>(float2 (&v)[8]) { dft8_impl<true>(v); }

// 16 = 4 x 4: A_n2 = DFT4 over n1 of x[4 n1 + n2]; B = W16^(n2 k1) A_n2[k1];
// X[k1 + 4 k2] = DFT4 over n2 of B.
template <bool INV>
__device__ __forceinline__ void dft16_impl(float2 (&v)[16]) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
  // v[4*k1 + n2] now holds A_n2[k1]
  v[5] = cmul(v[5], w16<1, INV>());
  v[6] = cmul(v[6], w16<2, INV>());
  v[7] = cmul(v[7], w16<3, INV>());
  v[9] = cmul(v[9], w16<2, INV>());
  v[10] = cmul(v[10], w16<4, INV>());
  v[11] = cmul(v[11], w16<6, INV>());
  v[13] = cmul(v[13], w16<3, INV>());
  v[14] = cmul(v[14], w16<6, INV>());
  v[15] = cmul(v[15], w16<9, INV>());
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  // v[4*k1 + k2] holds X[k1 + 4 k2]: transpose the 4x4 index
  float2 t[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) t[i] = v[i];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[4 * k1 + k2];
}
template <>
__device__ __forceinline__ void dft<16, false>(float2 (&v)[16]) { dft16_impl<false>(v); }
template <>
__device__ __forceinline__ void dft<16, true>(float2 (&v)[16]) { dft16_impl<true>(v); }

// Twiddle exp(-2 pi i m / Nt) from the two-level shared table of the
// transform size Nt = N * tws: tw_s[hi] = exp(-2 pi i (hi kTwSplit)/Nt),
// tw_s[kTwSplit + lo] = exp(-2 pi i lo / Nt), m = hi kTwSplit + lo.
__device__ __forceinline__ float2 twiddle(const float2* tw_s, int m) {
  return cmul(tw_s[m / kTwSplit], tw_s[kTwSplit + (m % kTwSplit)]);
}

// Direct twiddle table of the radix-16 passes with sub-transform length 16
// and 256 (the table option TP): a radix-16 pass at length NS multiplies
// input r of butterfly j by exp(-+2 pi i r (j mod NS) / (16 NS)), which
// does not depend on the transform size, so one table of 15 x 16 + 15 x
// 256 entries, entry (r - 1) NS + (j mod NS) at offset 0 (NS = 16) or 240
// (NS = 256), serves every size; each entry is one correctly rounded value
// instead of a product of table values (kTwPass entries, rx_internal.cuh).

template <int R, int NS>
constexpr bool pass_table() { return R == 16 && (NS == 16 || NS == 256); }

// Sub-transform length of the last pass (passes use radix 16 while at
// least 16 remain) and its radix.
template <int N>
constexpr int last_ns() {
  int ns = 1;
  while (N / ns > 16) ns *= 16;
  return ns;
}

// Twiddles and R-point DFT of butterfly j of the pass with sub-transform
// length NS: inputs v[r] = element j + r N/R, outputs v[r] = element
// (j / NS) NS R + (j mod NS) + r NS.  Inverse passes conjugate the twiddles.
template <int N, int R, int NS, bool INV, bool TP = false>
__device__ __forceinline__ void pass_butterfly(float2 (&v)[R], int j, const float2* __restrict__ tw, int tws,
                                               const float2* __restrict__ tp = nullptr) {
  if constexpr (TP && pass_table<R, NS>()) {
    const float2* t = tp + (NS == 16 ? 0 : 240) + (j & (NS - 1));
#pragma unroll
    for (int r = 1; r < R; ++r) {
      float2 w = t[(r - 1) * NS];
      if (INV) w.y = -w.y;
      v[r] = cmul(v[r], w);
    }
  } else if (NS > 1) {
    // w^r for r < R from the table entries w, w^2, w^4, w^8 (each power is
    // a product of at most four correctly rounded table values)
    constexpr int STEP = N / (NS * R);
    const int m = (j & (NS - 1)) * STEP * tws;
    float2 wp[R];
    wp[1] = twiddle(tw, m);
    if (R > 2) wp[2] = twiddle(tw, 2 * m);
    if (R > 4) wp[4] = twiddle(tw, 4 * m);
    if (R > 8) wp[8] = twiddle(tw, 8 * m);
#pragma unroll
    for (int r = 3; r < R; ++r) {
      if (r == 4 || r == 8) continue;
      const int hb = r >= 8 ? 8 : (r >= 4 ? 4 : 2);
      wp[r] = cmul(wp[hb], wp[r - hb]);
    }
#pragma unroll
    for (int r = 1; r < R; ++r) {
      float2 w = wp[r];
      if (INV) w.y = -w.y;
      v[r] = cmul(v[r], w);
    }
  }
  dft<R, INV>(v);
}

// One Stockham pass through shared memory.
template <int N, int NT, int R, int NS, bool INV, bool TP = false>
__device__ __forceinline__ void fft_pass(float2* buf, const float2* __restrict__ tw, int tws,
                                         const float2* __restrict__ tp = nullptr) {
  constexpr int NB = N / R;
  constexpr int PER = (NB + NT - 1) / NT;
  float2 v[PER][R];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int j = threadIdx.x + u * NT;
    if ((NB % NT) == 0 || j < NB) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[u][r] = buf[swz(j + r * NB)];
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int j = threadIdx.x + u * NT;
    if ((NB % NT) == 0 || j < NB) {
      pass_butterfly<N, R, NS, INV, TP>(v[u], j, tw, tws, tp);
      const int idxD = (j / NS) * NS * R + (j & (NS - 1));
#pragma unroll
      for (int r = 0; r < R; ++r) buf[swz(idxD + r * NS)] = v[u][r];
    }
  }
  __syncthreads();
}

// The passes with sub-transform lengths NS, 16 NS, ... below NS_END.
template <int N, int NT, int NS, int NS_END, bool INV, bool TP = false>
__device__ __forceinline__ void fft_passes(float2* buf, const float2* __restrict__ tw, int tws,
                                           const float2* __restrict__ tp = nullptr) {
  if constexpr (NS < NS_END) {
    constexpr int REM = N / NS;
    constexpr int R = REM >= 16 ? 16 : REM;
    fft_pass<N, NT, R, NS, INV, TP>(buf, tw, tws, tp);
    fft_passes<N, NT, NS * R, NS_END, INV, TP>(buf, tw, tws, tp);
  }
}

// Unnormalised DFT of buf[0..N) (swizzled), forward = exp(-2 pi i k n / N).
// Requires a __syncthreads() between the last write of buf and this call.
template <int N, int NT, bool INV>
__device__ __forceinline__ void fft_smem(float2* buf, const float2* __restrict__ tw, int tws) {
  fft_passes<N, NT, 1, N, INV>(buf, tw, tws);
}

}  // namespace rx
