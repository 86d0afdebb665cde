// a8 BER counting against the known payload (paper Sec. III: the Q-factor
// is estimated from the BER) and the ingest conversion kernel.
//
// Reference bits: PRBS-31, b[i] = (state >> i) & 1 for i < 31, then
// b[n] = b[n-28] ^ b[n-31].  The 31-bit window s_p = b[p..p+30] advances
// as s_{p+1} = A s_p over GF(2); A^(2^i) (columns, host-computed) give
// s_P for any P in O(log P) matrix-vector products, after which the
// sequence is produced 28 bits per step: b[p..p+27] = s & (2^28 - 1),
// s <- (s >> 28) | (((s ^ (s >> 3)) & (2^28 - 1)) << 3).
//
// Sync (once): every delay d in [-Dmax, Dmax] and polarisation order is
// tried on the sync window, each polarisation keeping its best quadrant;
// the smallest total wins (first in (d, order) order on ties).  Counting:
// per slip window, errors under all four quadrants are accumulated; a
// sequential pass then keeps the current quadrant unless its errors exceed
// a quarter of the window's bits, in which case the window's best quadrant
// is taken and a slip is counted.
#include <algorithm>
#include <cstdint>

#include "rx_internal.cuh"

namespace rx {

__device__ __forceinline__ uint32_t gf2_apply(const uint32_t* __restrict__ M, uint32_t s) {
  uint32_t r = 0;
#pragma unroll
  for (int j = 0; j < 31; ++j) r ^= M[j] & (0u - ((s >> j) & 1u));
  return r;
}

__device__ uint32_t prbs_window_at(const uint32_t* jump, uint32_t s, long long P) {
  for (int i = 0; P > 0; ++i, P >>= 1)
    if (P & 1) s = gf2_apply(jump + i * 31, s);
  return s;
}

// Bits [B0, B0 + nbits) of each polarisation's PRBS into d.ref (LSB first).
// B0 = (sym0 - delay) * bps, delay read from the device state if use_delay.
// The jump matrices are staged in shared memory.  Warp 0 jumps the state to
// the block's first chunk (lane j holds column j of each matrix; a product
// is an XOR reduction over the lanes), then every thread jumps the few
// chunks from there to its own (at most log2(blockDim) products).  A chunk
// is kRefChunk bits.
constexpr int kRefChunk = 256;

__device__ __forceinline__ void ref_gen_body(const RxDev& d, long long sym0, int nbits, int use_delay, VBlock vb) {
  __shared__ uint32_t jump_s[48 * 31];
  __shared__ uint32_t base_s;
  for (int i = threadIdx.x; i < 48 * 31; i += blockDim.x) jump_s[i] = d.prbs_jump[i];
  __syncthreads();
  const int pol = vb.y;
  const int chunk0 = vb.x * blockDim.x;
  if ((long long)chunk0 * kRefChunk >= nbits) return;  // whole block past the end (uniform)
  const long long delay = use_delay ? d.st->sync_delay : 0;
  const long long B0 = (sym0 - delay) * d.bps;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    uint32_t st = d.prbs_state0[pol];
    long long P = B0 + (long long)chunk0 * kRefChunk;
    for (int i = 0; P > 0; ++i, P >>= 1) {
      if (P & 1) {
        uint32_t v = (lane < 31 && ((st >> lane) & 1u)) ? jump_s[i * 31 + lane] : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v ^= __shfl_xor_sync(0xffffffffu, v, o);
        st = v;
      }
    }
    if (lane == 0) base_s = st;
  }
  __syncthreads();
  const int chunk = chunk0 + threadIdx.x;
  const int start = chunk * kRefChunk;
  if (start >= nbits) return;
  uint32_t s = prbs_window_at(jump_s, base_s, (long long)threadIdx.x * kRefChunk);
  uint32_t* out = d.ref + (long long)pol * d.ref_words + start / 32;
  const int nw = min(kRefChunk / 32, (nbits - start + 31) / 32);
  unsigned long long acc = 0;
  int nacc = 0, wc = 0;
  while (wc < nw) {
    acc |= (unsigned long long)(s & 0x0FFFFFFFu) << nacc;
    nacc += 28;
    const uint32_t nx = (s ^ (s >> 3)) & 0x0FFFFFFFu;
    s = (s >> 28) | (nx << 3);
    while (nacc >= 32 && wc < nw) {
      out[wc++] = (uint32_t)acc;
      acc >>= 32;
      nacc -= 32;
    }
  }
}

__global__ void __launch_bounds__(128) ref_gen_kernel(RxDev d, long long sym0, int nbits, int use_delay) {
  ref_gen_body(d, sym0, nbits, use_delay, own_block());
}

// Batched: use_delay 0 generates the sync window, 1 the counted range.
__global__ void __launch_bounds__(128) ref_gen_batch_kernel(BView v, int use_delay) {
  int fi;
  VBlock vb;
  if (!batch_block(v, fi, vb)) return;
  const BFrame& f = v.frames[fi];
  ref_gen_body(f.d, use_delay ? f.ref_sym0 : f.sync_sym0, use_delay ? f.ref_nbits : f.sync_nbits, use_delay, vb);
}

__device__ __forceinline__ uint32_t ref_bits(const uint32_t* ref, long long off, int n) {
  const long long w = off >> 5;
  const int sh = (int)(off & 31);
  const unsigned long long v = ((unsigned long long)ref[w + 1] << 32) | ref[w];
  return (uint32_t)(v >> sh) & ((1u << n) - 1u);
}

// Received bits of levels (lI, lQ) rotated by q quarter turns (x j each),
// in payload order: I bits MSB first then Q bits, bit j of the result is
// the j-th bit of the symbol.
__device__ __forceinline__ uint32_t rx_sym_bits(int lI, int lQ, int q, int nl) {
  for (int i = 0; i < q; ++i) {
    const int t = lI;
    lI = nl - 1 - lQ;
    lQ = t;
  }
  if (nl == 2) return (uint32_t)(1 - lI) | ((uint32_t)(1 - lQ) << 1);
  const uint32_t gI = (uint32_t)(lI ^ (lI >> 1)), gQ = (uint32_t)(lQ ^ (lQ >> 1));
  return ((gI >> 1) & 1u) | ((gI & 1u) << 1) | (((gQ >> 1) & 1u) << 2) | ((gQ & 1u) << 3);
}

// One block per (delay, order) candidate over the sync window; the
// reference holds tx symbols [k_s - Dmax, k_s + n_sync + Dmax).
__device__ __forceinline__ void sync_body(const RxDev& d, VBlock vb) {
  __shared__ unsigned red[8][8];
  const int cand = vb.x;
  const int delay = cand / 2 - d.sync_dmax, perm = cand & 1;
  const long long ks = d.ber_skip;
  unsigned err[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
  for (int i = threadIdx.x; i < d.sync_syms; i += 256) {
    const long long k = ks + i;
    const uint8_t v = d.dec[k % d.dec_cap];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int tx = p ^ perm;
      const long long off = (long long)(i - delay + d.sync_dmax) * d.bps;
      const uint32_t rb = ref_bits(d.ref + (long long)tx * d.ref_words, off, d.bps);
      const int lv = (v >> (4 * p)) & 15;
#pragma unroll
      for (int q = 0; q < 4; ++q) err[p][q] += __popc(rx_sym_bits(lv & 3, lv >> 2, q, d.nl) ^ rb);
    }
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      unsigned v = err[p][q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (l == 0) red[w][p * 4 + q] = v;
    }
  __syncthreads();
  if (threadIdx.x < 8) {
    unsigned s = 0;
    for (int ww = 0; ww < 8; ++ww) s += red[ww][threadIdx.x];
    d.sync_err[cand * 8 + threadIdx.x] = s;
  }
  // the last block to finish selects the candidate (atomic counter; no waits)
  __shared__ int am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = atomicAdd(&d.ber_done[0], 1u) == vb.nx - 1;
  __syncthreads();
  if (!am_last || threadIdx.x >= 32) return;
  __threadfence();
  const int ncand = (2 * d.sync_dmax + 1) * 2;
  unsigned best = 0xffffffffu;
  int bc = 0x7fffffff, bq0 = 0, bq1 = 0;
  for (int c = threadIdx.x; c < ncand; c += 32) {
    unsigned tot = 0;
    int qs[2];
    for (int p = 0; p < 2; ++p) {
      unsigned m = 0xffffffffu;
      int qb = 0;
      for (int q = 0; q < 4; ++q) {
        const unsigned e = __ldcg(&d.sync_err[c * 8 + p * 4 + q]);
        if (e < m) { m = e; qb = q; }
      }
      tot += m;
      qs[p] = qb;
    }
    if (tot < best) { best = tot; bc = c; bq0 = qs[0]; bq1 = qs[1]; }
  }
  // smallest total, first candidate on ties
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
    const int o0 = __shfl_xor_sync(0xffffffffu, bq0, o), o1 = __shfl_xor_sync(0xffffffffu, bq1, o);
    if (ob < best || (ob == best && oc < bc)) { best = ob; bc = oc; bq0 = o0; bq1 = o1; }
  }
  if (threadIdx.x == 0) {
    StreamState* st = d.st;
    st->sync_delay = bc / 2 - d.sync_dmax;
    st->sync_perm = bc & 1;
    st->sync_q[0] = st->q_cur[0] = bq0;
    st->sync_q[1] = st->q_cur[1] = bq1;
    st->synced = 1;
    d.ber_done[0] = 0;
  }
}

__global__ void __launch_bounds__(256) sync_kernel(RxDev d) {
  sync_body(d, own_block());
}

__global__ void __launch_bounds__(256) sync_batch_kernel(BView v) {
  int fi;
  VBlock vb;
  if (!batch_block(v, fi, vb)) return;
  sync_body(v.frames[fi].d, vb);
}

// Errors of symbols [ka, kb) under the four quadrants, per slip window.
// The symbols are cut into pieces of at most kBerPiece symbols that never
// cross a window; one warp counts one piece (lane l takes symbols k0 + l of
// each 32-symbol step, so decision bytes load coalesced and the reference
// words are shared by the lanes), reduces its counters with shuffles and
// adds them to its window's slot.  The reference holds tx symbols
// [ka - delay, kb - delay).  The last block to finish runs the slip pass
// over windows [w_from, w_to).
__device__ void slip_pass(const RxDev& d, long long w_from, long long w_to, long long k_lim, int n_win_ring,
                          unsigned* win_s);

constexpr int kBerPiece = 256;  // symbols per warp work item

__host__ __device__ inline long long ber_items(long long ka, long long kb, long long ks, long long sw) {
  const long long k_lo = ka > ks ? ka : ks;
  if (kb <= k_lo) return 0;
  const long long wa = (k_lo - ks) / sw, wb = (kb - 1 - ks) / sw;
  return (wb - wa + 1) * ((sw + kBerPiece - 1) / kBerPiece);
}

__device__ __forceinline__ void ber_count_body(const RxDev& d, long long ka, long long kb, long long w_from,
                                               long long w_to, long long k_lim, int n_win_ring, VBlock vb) {
  __shared__ uint8_t lut[4][16];  // bits of level code (lI | lQ << 2) rotated by q
  __shared__ int am_last;
  if (threadIdx.x < 64) {
    const int q = threadIdx.x >> 4, lv = threadIdx.x & 15;
    lut[q][lv] = (uint8_t)rx_sym_bits(lv & 3, lv >> 2, q, d.nl);
  }
  __syncthreads();
  const long long ks = d.ber_skip, sw = d.slip_win;
  const long long ppw = (sw + kBerPiece - 1) / kBerPiece;  // pieces per window
  const long long k_lo = ka > ks ? ka : ks;
  const int warp = threadIdx.x >> 5, l = threadIdx.x & 31;
  const long long item = (long long)vb.x * 8 + warp;
  bool wrote = false;
  if (item < ber_items(ka, kb, ks, sw)) {  // warp-uniform
    const long long w = (k_lo - ks) / sw + item / ppw;
    const long long pc = item % ppw;
    const long long p0 = max(k_lo, ks + w * sw + pc * kBerPiece);
    const long long p1 = min(kb, min(ks + (w + 1) * sw, ks + w * sw + (pc + 1) * kBerPiece));
    const int perm = d.st->sync_perm;
    unsigned err[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    long long slot = (p0 + l) % d.dec_cap;
#pragma unroll 2
    for (long long k0 = p0; k0 < p1; k0 += 32) {
      const long long k = k0 + l;
      if (k < p1) {
        const uint8_t v = d.dec[slot];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const uint32_t rb = ref_bits(d.ref + (long long)(p ^ perm) * d.ref_words, (k - ka) * d.bps, d.bps);
          const int lv = (v >> (4 * p)) & 15;
#pragma unroll
          for (int q = 0; q < 4; ++q) err[p][q] += __popc((uint32_t)lut[q][lv] ^ rb);
        }
      }
      slot += 32;
      if (slot >= d.dec_cap) slot -= d.dec_cap;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      unsigned e = err[j >> 2][j & 3];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
      if (l == 0 && e) {
        atomicAdd(&d.win_err[(w % n_win_ring) * 8 + j], e);
        wrote = true;
      }
    }
  }
  if (w_to <= w_from) return;
  // threads that added to the window counters make them visible before the
  // block takes its ticket
  if (wrote) __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = atomicAdd(&d.ber_done[1], 1u) == vb.nx - 1;
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  extern __shared__ unsigned win_s[];
  slip_pass(d, w_from, w_to, k_lim, n_win_ring, win_s);
  if (threadIdx.x == 0) d.ber_done[1] = 0;
}

__global__ void __launch_bounds__(256) ber_count_kernel(RxDev d, long long ka, long long kb, long long w_from,
                                                        long long w_to, long long k_lim, int n_win_ring) {
  ber_count_body(d, ka, kb, w_from, w_to, k_lim, n_win_ring, own_block());
}

__global__ void __launch_bounds__(256) ber_count_batch_kernel(BView v) {
  int fi;
  VBlock vb;
  if (!batch_block(v, fi, vb)) return;
  const BFrame& f = v.frames[fi];
  ber_count_body(f.d, f.ka, f.kb, f.w_from, f.w_to, f.k_lim, f.n_win_ring, vb);
}

// Slip pass over windows [w_from, w_to); window w covers symbols
// [ks + w SW, ks + (w+1) SW) clipped to k_lim.  A 4-state automaton (state =
// quadrant in use) per polarisation.  Windows are staged in shared memory in
// chunks of kSlipChunk; each of the 128 threads of a polarisation runs a
// contiguous slice of a chunk from all four start states at once, which
// gives a map start state -> (end state, errors, slips); the maps are
// composed in window order (shuffles within a warp, then the warps in
// order) and the composition is applied to the current state, which gives
// exactly the sequential result.  Window slots are cleared.
constexpr int kSlipChunk = 1024;

struct SlipMap {
  int q[4];
  unsigned e[4], s[4];
};

// a then b: start state i -> b applied to a's end state.
__device__ __forceinline__ void slip_compose(SlipMap& a, const SlipMap& b) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = a.q[i];
    const int bq = m == 0 ? b.q[0] : m == 1 ? b.q[1] : m == 2 ? b.q[2] : b.q[3];
    const unsigned be = m == 0 ? b.e[0] : m == 1 ? b.e[1] : m == 2 ? b.e[2] : b.e[3];
    const unsigned bs = m == 0 ? b.s[0] : m == 1 ? b.s[1] : m == 2 ? b.s[2] : b.s[3];
    a.q[i] = bq;
    a.e[i] += be;
    a.s[i] += bs;
  }
}

__device__ void slip_pass(const RxDev& d, long long w_from, long long w_to, long long k_lim, int n_win_ring,
                          unsigned* win_s) {
  __shared__ SlipMap wmap[8];
  const int pol = threadIdx.x >> 7, lp = threadIdx.x & 127, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  StreamState* st = d.st;
  const long long ks = d.ber_skip;
  int qc = st->q_cur[pol];  // used by the first thread of each polarisation
  unsigned long long E = 0, SL = 0;
  for (long long c0 = w_from; c0 < w_to; c0 += kSlipChunk) {
    const int nw = (int)min((long long)kSlipChunk, w_to - c0);
    const int r0 = (int)(c0 % n_win_ring);  // ring slot of the chunk's first window (nw <= ring size)
    // stage the chunk's counters (eight loads in flight per thread), then
    // clear their slots
    for (int i0 = threadIdx.x; i0 < nw * 8; i0 += 8 * blockDim.x) {
      unsigned v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = i0 + u * blockDim.x;
        int slot = r0 + (i >> 3);
        if (slot >= n_win_ring) slot -= n_win_ring;
        v[u] = i < nw * 8 ? __ldcg(d.win_err + (long long)slot * 8 + (i & 7)) : 0u;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = i0 + u * blockDim.x;
        if (i < nw * 8) win_s[i] = v[u];
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nw * 8; i += blockDim.x) {
      int slot = r0 + (i >> 3);
      if (slot >= n_win_ring) slot -= n_win_ring;
      d.win_err[(long long)slot * 8 + (i & 7)] = 0;
    }
    // this thread's slice of windows, from every start state
    const int per = (nw + 127) / 128;
    const int a0 = min(lp * per, nw), a1 = min(a0 + per, nw);
    SlipMap m;
#pragma unroll
    for (int i = 0; i < 4; ++i) { m.q[i] = i; m.e[i] = 0u; m.s[i] = 0u; }
    for (int i = a0; i < a1; ++i) {
      const long long a = ks + (c0 + i) * d.slip_win;
      const long long nb = (min(a + d.slip_win, k_lim) - a) * d.bps;
      const unsigned* ev = win_s + i * 8 + pol * 4;
      const unsigned e0 = ev[0], e1 = ev[1], e2 = ev[2], e3 = ev[3];
      int qb = 0;
      unsigned eb = e0;
      if (e1 < eb) { qb = 1; eb = e1; }
      if (e2 < eb) { qb = 2; eb = e2; }
      if (e3 < eb) { qb = 3; eb = e3; }
#pragma unroll
      for (int s0 = 0; s0 < 4; ++s0) {
        const int qs = m.q[s0];
        unsigned ec = qs == 0 ? e0 : qs == 1 ? e1 : qs == 2 ? e2 : e3;
        if ((long long)ec * 4 > nb) {
          m.q[s0] = qb;
          ec = eb;
          ++m.s[s0];
        }
        m.e[s0] += ec;
      }
    }
    // compose the 32 maps of the warp in order: lane l takes lane l + o's
    // composition when l is a multiple of 2o
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      SlipMap nb;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        nb.q[i] = __shfl_down_sync(0xffffffffu, m.q[i], o);
        nb.e[i] = __shfl_down_sync(0xffffffffu, m.e[i], o);
        nb.s[i] = __shfl_down_sync(0xffffffffu, m.s[i], o);
      }
      if ((lane & (2 * o - 1)) == 0) slip_compose(m, nb);
    }
    if (lane == 0) wmap[warp] = m;
    __syncthreads();
    if (lp == 0) {
#pragma unroll 1
      for (int w = 4 * pol; w < 4 * pol + 4; ++w) {
        const SlipMap& mw = wmap[w];
        const int i = qc;
        E += i == 0 ? mw.e[0] : i == 1 ? mw.e[1] : i == 2 ? mw.e[2] : mw.e[3];
        SL += i == 0 ? mw.s[0] : i == 1 ? mw.s[1] : i == 2 ? mw.s[2] : mw.s[3];
        qc = i == 0 ? mw.q[0] : i == 1 ? mw.q[1] : i == 2 ? mw.q[2] : mw.q[3];
      }
    }
    __syncthreads();
  }
  if (lp == 0) {
    const long long a = ks + w_from * d.slip_win;
    const long long b = min(ks + w_to * (long long)d.slip_win, k_lim);
    st->q_cur[pol] = qc;
    atomicAdd(&st->errors, E);
    atomicAdd(&st->bits, (unsigned long long)(max(b - a, 0LL) * d.bps));
    atomicAdd(&st->slips, SL);
  }
}

// Push conversion: src planar [2][n] of dtype (0 c128, 1 c64, 2 c16) into
// the ring at absolute sample offset w0 (index mod cap), storage dtype;
// element i of the push.
__device__ __forceinline__ void ingest_one(void* ring, long long ring_cap, int storage, const void* __restrict__ src,
                                           int dtype, long long n, long long j0, long long i) {
  if (i >= 2 * n) return;
  const int pol = i >= n;
  const long long j = i - pol * n;
  float2 v;
  if (dtype == 0) {
    const double2 a = reinterpret_cast<const double2*>(src)[i];
    v = make_float2((float)a.x, (float)a.y);
  } else if (dtype == 1) {
    v = reinterpret_cast<const float2*>(src)[i];
  } else {
    v = __half22float2(reinterpret_cast<const __half2*>(src)[i]);
  }
  long long slot = j0 + j;  // j0 = w0 mod cap, n <= cap
  if (slot >= ring_cap) slot -= ring_cap;
  const long long dst = (long long)pol * ring_cap + slot;
  if (storage == 2) reinterpret_cast<__half2*>(ring)[dst] = __float22half2_rn(v);
  else reinterpret_cast<float2*>(ring)[dst] = v;
}

__global__ void ingest_kernel(RxDev d, const void* __restrict__ src, int dtype, long long n, long long j0) {
  ingest_one(d.ring, d.ring_cap, d.storage, src, dtype, n, j0, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// c64 input into a c64 ring, two samples (16 bytes) per access: pair j of
// polarisation p is src4[p n2 + j] -> ring slot j0 + 2j (mod cap).  Needs
// n, j0 and cap even and a 16-byte aligned source, so a pair never
// straddles the polarisations or the ring's wrap.  Each thread moves four
// pairs, all four loads issued before the stores.
__device__ __forceinline__ void ingest_pairs_body(void* ring, long long ring_cap, const float4* __restrict__ src,
                                                  long long n2, long long j0, VBlock vb) {
  float4* ring4 = reinterpret_cast<float4*>(ring);
  const long long cap2 = ring_cap / 2;
  const long long s0 = j0 / 2;
  const long long stride = (long long)vb.nx * blockDim.x;
  const long long i0 = (long long)vb.x * blockDim.x + threadIdx.x;
  float4 v[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const long long i = i0 + u * stride;
    if (i < 2 * n2) v[u] = __ldcs(&src[i]);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const long long i = i0 + u * stride;
    if (i < 2 * n2) {
      const int pol = i >= n2;
      const long long j = i - pol * n2;
      long long slot = s0 + j;
      if (slot >= cap2) slot -= cap2;
      ring4[pol * cap2 + slot] = v[u];
    }
  }
}

__global__ void __launch_bounds__(256) ingest_pairs_kernel(RxDev d, const float4* __restrict__ src, long long n2,
                                                            long long j0) {
  ingest_pairs_body(d.ring, d.ring_cap, src, n2, j0, own_block());
}

// The pushes of many streams in one launch: entry e of the list (frames
// unused) is ingest e, its nx[e] blocks of 256 threads as in the plain
// launches (pairs: four pairs per thread; else one element).
__global__ void __launch_bounds__(256) ingest_batch_kernel(const BIngest* __restrict__ ing, BView v) {
  int e;
  VBlock vb;
  if (!batch_block(v, e, vb)) return;
  const BIngest& g = ing[e];
  if (g.pairs) {
    ingest_pairs_body(g.ring, g.ring_cap, static_cast<const float4*>(g.src), g.n / 2, g.j0, vb);
  } else {
    ingest_one(g.ring, g.ring_cap, g.storage, g.src, g.dtype, g.n, g.j0, (long long)vb.x * blockDim.x + threadIdx.x);
  }
}

// ---- launchers ------------------------------------------------------------

cudaError_t launch_ref_gen(const RxDev& d, long long sym0, int nbits, int use_delay, cudaStream_t s) {
  const int chunks = (nbits + kRefChunk - 1) / kRefChunk;
  dim3 grid((chunks + 127) / 128, 2);
  ref_gen_kernel<<<grid, 128, 0, s>>>(d, sym0, nbits, use_delay);
  return cudaGetLastError();
}

cudaError_t launch_sync(const RxDev& d, cudaStream_t s) {
  sync_kernel<<<(2 * d.sync_dmax + 1) * 2, 256, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t ber_set_attributes() {
  cudaError_t e = cudaFuncSetAttribute(ber_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(kSlipChunk * 8 * sizeof(unsigned)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(ber_count_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kSlipChunk * 8 * sizeof(unsigned)));
  return e;
}

cudaError_t launch_ber(const RxDev& d, long long ka, long long kb, long long w_from, long long w_to,
                       long long k_lim, int n_win_ring, cudaStream_t s) {
  if (kb <= ka && w_to <= w_from) return cudaSuccess;
  const long long items = ber_items(ka, kb, d.ber_skip, d.slip_win);
  const long long blocks = std::max(1LL, (items + 7) / 8);
  ber_count_kernel<<<(unsigned)blocks, 256, kSlipChunk * 8 * sizeof(unsigned), s>>>(d, ka, kb, w_from, w_to, k_lim,
                                                                                    n_win_ring);
  return cudaGetLastError();
}

cudaError_t launch_ingest(const RxDev& d, const void* src, int dtype, long long n, long long w0, cudaStream_t s) {
  const long long tot = 2 * n;
  if (tot == 0) return cudaSuccess;
  const long long j0 = w0 % d.ring_cap;
  if (dtype == 1 && d.storage == 1 && (n & 1) == 0 && (j0 & 1) == 0 && (d.ring_cap & 1) == 0 &&
      (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    const long long pairs = n;  // 2 pols x n/2 pairs
    const long long blocks = (pairs + 1023) / 1024;
    ingest_pairs_kernel<<<(unsigned)blocks, 256, 0, s>>>(d, static_cast<const float4*>(src), n / 2, j0);
    return cudaGetLastError();
  }
  ingest_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(d, src, dtype, n, j0);
  return cudaGetLastError();
}

// ---- batched launchers (grids as above) -------------------------------------

int ref_grid_x(int nbits) { return ((nbits + kRefChunk - 1) / kRefChunk + 127) / 128; }
int sync_grid_x(const RxDev& d) { return (2 * d.sync_dmax + 1) * 2; }
int ber_grid_x(const RxDev& d, long long ka, long long kb) {
  return (int)std::max(1LL, (ber_items(ka, kb, d.ber_skip, d.slip_win) + 7) / 8);
}
int ingest_grid_x(long long n, bool pairs) { return (int)(pairs ? (n + 1023) / 1024 : (2 * n + 255) / 256); }
// The 16-byte pair path of launch_ingest applies.
bool ingest_pairs_ok(const RxDev& d, const void* src, int dtype, long long n, long long w0) {
  const long long j0 = w0 % d.ring_cap;
  return dtype == 1 && d.storage == 1 && (n & 1) == 0 && (j0 & 1) == 0 && (d.ring_cap & 1) == 0 &&
         (reinterpret_cast<uintptr_t>(src) & 15) == 0;
}

cudaError_t launch_ref_gen_batch(const BView& v, int blocks, int use_delay, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  return launch_k(ref_gen_batch_kernel, blocks, 128, 0, s, v, use_delay);
}

cudaError_t launch_sync_batch(const BView& v, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  return launch_k(sync_batch_kernel, blocks, 256, 0, s, v);
}

cudaError_t launch_ber_batch(const BView& v, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  return launch_k(ber_count_batch_kernel, blocks, 256, kSlipChunk * 8 * sizeof(unsigned), s, v);
}

cudaError_t launch_ingest_batch(const BIngest* ing, const BView& v, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  ingest_batch_kernel<<<blocks, 256, 0, s>>>(ing, v);
  return cudaGetLastError();
}

}  // namespace rx
