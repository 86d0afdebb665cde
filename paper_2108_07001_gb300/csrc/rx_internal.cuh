// Internal definitions shared by the receiver's kernels and its host runtime.
// Device state of one receiver stream lives in HBM; RxDev is passed by value
// to every kernel.  Layouts (per stream):
//   ring   [2][ring_cap]       pushed samples, storage dtype, index n mod cap
//   z      [2][zlen]           CD output of the frame, complex float; index
//                              i <-> absolute sample 2fF - c + i
//   y      [2 buf][2][64 + F]  equaliser output, frame f in buffer f % 2 after
//                              the last 64 symbols of frame f-1
//   bl     [2][F + 2W]         per decided symbol: BPS angle | levels << 8
//   taps   [G][2][2][T]        adaptive chains, complex float
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <tuple>

namespace rx {

constexpr int kMaxTaps = 31;
constexpr int kRotLo = 1024;          // FO rotation table split: n = hi*1024 + lo
constexpr int kRun = 256;             // BPS run / demap tile length (symbols)
constexpr int kMaxTrace = 4096;       // per-frame estimate records kept
constexpr int kYHist = 64;            // equalised-symbol history kept before each frame (>= 2W)
constexpr int kFoeMinSyms = 4096;     // shorter frames reuse the previous FO estimate
constexpr int kTwPass = 15 * 16 + 15 * 256;  // direct twiddles of the radix-16 passes (fft_smem.cuh)

// Per-frame estimates written by the estimator kernel (also the trace).
struct FrameRec {
  double tau;      // timing advance applied to the frame (s)
  double dfo;      // FO estimate (Hz)
  double gain;     // AGC gain
  double theta;    // FO phase at the frame start (rad)
};

// Accumulators filled by the CD kernel, consumed and cleared by the
// estimator kernel.  Block partials are FP32; the sums are FP64, so their
// value does not depend on the order the blocks finish in (the partials
// are exactly representable and the sums stay far from 53-bit rounding).
struct FrameAcc {
  double C[2];     // Godard sum (re, im), both polarisations
  double P;        // sum |z|^2 of in-frame samples, both polarisations
  double pad;
};

// Estimator state entering a frame (double-buffered by frame parity).
struct EstState {
  double tau;          // timing advance of the frame's CD pass (s)
  double theta;        // FO phase at the frame start
  double dfo_prev;     // FO estimate of the previous frame (Hz)
  double pad;
};

// Scalars carried from frame to frame (device resident).
struct StreamState {
  int bhat_last[2];    // BPS angle of the last decided symbol (-1: none)
  int m_last[2];       // unwrap counter of the last decided symbol
  int synced;
  int sync_delay, sync_perm, sync_q[2];
  int q_cur[2];        // BER quadrant in use per polarisation
  int reinit;          // CMA singularity re-initialisation happened
  int pad;
  unsigned long long bits, errors, slips;
  double evm_num, evm_den;
};

struct RxDev {
  // geometry
  int N, halo, h, L, c, T, K, S, F, G, B, W, bps;
  int nl;                      // levels per dimension (2 or 4)
  int bps_stride;              // BPS coarse stride S: 1 full search, > 1 two-stage over B/S angles
  int bps_nw;                  // full-search BPS: runs (warps) per block, 4 or 8
  int mimo_nw;                 // MIMO: segment chains (warps) per block, 1..8
  int zlen;                    // 2F + 2c
  int storage;                 // RX_C64 / RX_C16
  long long ring_cap;          // samples per polarisation
  double Rs, fs;
  float mu_cma, mu_dd, R2;
  float timing_gain;
  int cma_syms, acq_syms;
  int ber_on, ber_skip, sync_syms, sync_dmax, slip_win;
  long long out_cap_bytes;
  long long dec_cap;           // decision ring capacity (symbols)
  long long hist_syms;         // inspection history length (0: off)
  // buffers
  void* ring;
  float2* Hs;                  // static CD x RRC response, 1/N folded in
  float2* Hf;                  // Hs x timing phase of the coming pass
  float2* tw;                  // tw[k] = exp(-2 pi i k / N)
  float2* tw2;                 // [512 + kTwPass]: two-level tables of N and N/2 (each exp(-2 pi i 128 h / Nt),
                               // h < 128, then exp(-2 pi i l / Nt), l < 128), then the direct pass table
  float2* z;
  float2* rot_hi;              // [ceil(zlen/1024)]  gain * exp(-j(theta + w (hi*1024 - c)))
  float2* rot_lo;              // [1024]             exp(-j w lo)
  FrameAcc* acc;               // [3]: frame parity slots + the timing-acquisition pass
  double* psd;                 // [3][N/2] FOE periodogram (FP64 sums of FP32 block terms)
  EstState* es;                // [2]
  FrameRec* rec;               // [kMaxTrace]
  StreamState* st;
  float2* w_acq;               // [2][2][T]
  float2* chains;              // [G][2][2][T]
  float2* y;                   // [2][2][kYHist + F]
  uint16_t* bl;                // [2][F + 2W]
  int* run_int;                // [2][nruns] internal unwrap increment sums
  int* run_m0;                 // [2][nruns] unwrap counter at each run's first symbol
  int* run_edge;               // [2][nruns][2] BPS angle of each run's first and last symbol
  unsigned* bps_done;          // [2] finished-block counters of the BPS kernel
  unsigned* ber_done;          // [2] finished-block counters: sync, count
  uint8_t* dec;                // decision ring [dec_cap]: x levels | y levels << 4
  uint8_t* out;                // output bit ring (bytes)
  uint32_t* prbs_jump;         // [64][31] columns of A^(2^i)
  uint32_t* ref;               // [2][ref_words] reference bits of the frame range
  int ref_words;
  unsigned* sync_err;          // [(2 dmax + 1) * 2][2][4]
  unsigned* win_err;           // [kWinRing][2][4]
  uint32_t prbs_state0[2];     // PRBS start state per polarisation
  // inspection history (optional)
  float2* hist_y;              // [2][hist_syms]
  uint8_t* hist_bhat;          // [2][hist_syms]
  int* hist_m;                 // [2][hist_syms]
};

// Arguments of one frame.
struct FrameArgs {
  long long f;         // frame index
  int Ff;              // symbols in this frame
  long long s0;        // first CD output sample (absolute) = 2fF - c
  long long f0, f1;    // in-frame samples [f0, f1)
  long long n_valid;   // samples per pol that exist (beyond: zero)
  long long k_a, k_b;  // decided symbol range of this frame
  long long k_end;     // BER count limit (exclusive); LLONG_MAX before end of stream
  long long n_sym;     // symbols in the stream if known (final), else LLONG_MAX
  int est_only;        // CD pass that only accumulates the Godard sum
  int acc_slot;        // accumulator slot of this CD pass (f & 1; 2 for est_only)
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Nearest level index per dimension for unit-energy square QAM; values on
// a threshold take the larger level.  nl = 2: levels -1,+1 (/sqrt2);
// nl = 4: -3,-1,1,3 (/sqrt10).
__device__ __forceinline__ int level_of(float x, int nl) {
  if (nl == 2) return x >= 0.f ? 1 : 0;
  const float t = 0.63245553203367588f;  // 2/sqrt(10)
  return (x >= t) ? 3 : (x >= 0.f ? 2 : (x >= -t ? 1 : 0));
}
__device__ __forceinline__ float level_val(int l, int nl) {
  if (nl == 2) return l ? 0.70710678118654752f : -0.70710678118654752f;
  return (2 * l - 3) * 0.31622776601683794f;
}

// Loads one stored sample as complex float.
__device__ __forceinline__ float2 load_sample(const void* ring, int storage, long long idx) {
  if (storage == 2) {  // RX_C16
    __half2 hv = reinterpret_cast<const __half2*>(ring)[idx];
    return __half22float2(hv);
  }
  return reinterpret_cast<const float2*>(ring)[idx];
}

// Packed FP32 pairs (two IEEE single-precision lanes in one 64-bit register,
// element 0 in the low half): add/sub/mul/fma .rn.f32x2.
__device__ __forceinline__ unsigned long long f2pk(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2up(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2fma(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ unsigned long long f2mul(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2add(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2sub(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}


// ---- batched launches (rx_batch_push) -------------------------------------
//
// Every kernel of the chain is a body over block coordinates (x, y) of a
// grid nx blocks wide.  A plain launch passes its own blockIdx / gridDim.x;
// a batched launch runs the grids of many streams' frames one after the
// other in one flat grid, and each block finds its frame and coordinates
// from the launch's prefix sums.

struct VBlock {
  int x, y, nx;
};

__device__ __forceinline__ VBlock own_block() { return VBlock{(int)blockIdx.x, (int)blockIdx.y, (int)gridDim.x}; }

// One frame of one stream in a batched launch: the stream's device state
// with the frame's slot applied and every stage's arguments.
struct BFrame {
  RxDev d;
  FrameArgs fa;                  // the frame (or the decide-only pass at the stream end)
  FrameArgs fe;                  // the timing-acquisition pass of the first frame
  long long hist_base;           // first symbol of the frame (inspection history)
  long long sync_sym0, ref_sym0; // reference bits: the sync window, the counted range
  int sync_nbits, ref_nbits;
  long long ka, kb, w_from, w_to, k_lim;  // BER count
  int n_win_ring, pad;
};

// Ingest of one stream's push in a batched launch.
struct BIngest {
  void* ring;
  long long ring_cap;
  const void* src;
  long long n, j0;
  int storage, dtype, pairs, pad;
};

// A batched launch: list = [n, idx[nmax], nx[nmax], offs[nmax + 1]]; entry
// e runs frame idx[e]'s grid (nx[e] blocks wide) as the launch's blocks
// [offs[e], offs[e + 1]).
struct BView {
  const BFrame* frames;
  const int* list;
  int nmax;
};

// The frame and block coordinates of this block; false for the blocks past
// the last entry (the whole block returns).
__device__ __forceinline__ bool batch_block(const BView& v, int& frame, VBlock& vb) {
  const int n = v.list[0];
  const int* idx = v.list + 1;
  const int* nx = idx + v.nmax;
  const int* offs = nx + v.nmax;
  const int b = (int)blockIdx.x;
  if (n <= 0 || b >= offs[n]) return false;
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (offs[mid] <= b) lo = mid;
    else hi = mid;
  }
  const int r = b - offs[lo];
  vb.nx = nx[lo];
  vb.x = r % vb.nx;
  vb.y = r / vb.nx;
  frame = idx[lo];
  return true;
}

// Batched launches go through launch_k: a kernel launch on s, or, while a
// graph recorder is set on the calling thread, a kernel node added to the
// recorder's graph after the recorder's dependencies (the node becomes the
// only dependency of the next one).  Building a graph this way involves
// no stream capture, so other threads' device-wide calls are unaffected.
struct GraphRecorder {
  cudaGraph_t g = nullptr;
  cudaGraphNode_t deps[4] = {};
  int ndeps = 0;
  cudaGraphNode_t last = nullptr;  // the node added last
};
extern thread_local GraphRecorder* t_graph_rec;

template <typename... P, typename... A>
cudaError_t launch_k(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, const A&... a) {
  // the arguments converted to the kernel's parameter types, and their addresses
  std::tuple<P...> vals(a...);
  void* ptrs[sizeof...(P) > 0 ? sizeof...(P) : 1];
  std::apply([&](auto&... v) {
    int i = 0;
    ((ptrs[i++] = static_cast<void*>(&v)), ...);
  }, vals);
  GraphRecorder* r = t_graph_rec;
  if (!r) return cudaLaunchKernel(reinterpret_cast<const void*>(kern), grid, block, ptrs, smem, s);
  cudaKernelNodeParams p = {};
  p.func = reinterpret_cast<void*>(kern);
  p.gridDim = grid;
  p.blockDim = block;
  p.sharedMemBytes = (unsigned)smem;
  p.kernelParams = ptrs;
  cudaGraphNode_t n = nullptr;
  const cudaError_t e = cudaGraphAddKernelNode(&n, r->g, r->deps, (size_t)r->ndeps, &p);
  if (e != cudaSuccess) return e;
  r->deps[0] = n;
  r->ndeps = 1;
  r->last = n;
  return cudaSuccess;
}

}  // namespace rx
