// Allocation-free entry point: carrier recovery and decisions for one block
// of equalised symbols, with every piece of working memory in one
// file-scope device array instead of cudaMalloc'ed buffers.
//
// It runs the same blind-phase-search and demap kernels as the streaming
// receiver (k_bps.cu) on a block treated as a whole stream: the BPS window
// is truncated at both ends of the block and the unwrap counter starts at 0.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/rx.h"
#include "rx_internal.cuh"

namespace rx {
cudaError_t launch_bps(const RxDev& d, const FrameArgs& fa, cudaStream_t s);
cudaError_t launch_unwrap_demap(const RxDev& d, const FrameArgs& fa, cudaStream_t s);
cudaError_t bps_set_attributes();
void set_last_error(const char* msg);

namespace {

constexpr long long kMaxSyms = RX_NOALLOC_MAX_SYMS;
constexpr long long kF = (kMaxSyms + kRun - 1) / kRun * kRun;  // frame length used for the layout
constexpr long long kW = 32;                                    // largest half window
constexpr long long kRunStride = kF / kRun + 4;

// Layout of the scratch array (byte offsets, each 256-aligned).
constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffY = 0;  // buffer 0 of the [buf][2][kYHist + F] float2 layout (frame 0 only)
constexpr size_t kOffBl = align256(kOffY + 2 * (kYHist + kF) * sizeof(float2));   // [2][F + 2W] u16
constexpr size_t kOffRunInt = align256(kOffBl + 2 * (kF + 2 * kW) * sizeof(uint16_t));
constexpr size_t kOffRunM0 = align256(kOffRunInt + 2 * kRunStride * sizeof(int));
constexpr size_t kOffRunEdge = align256(kOffRunM0 + 2 * kRunStride * sizeof(int));
constexpr size_t kOffDone = align256(kOffRunEdge + 4 * kRunStride * sizeof(int));
constexpr size_t kOffSt = align256(kOffDone + 4 * sizeof(unsigned));
constexpr size_t kOffDec = align256(kOffSt + sizeof(StreamState));
constexpr size_t kScratchBytes = align256(kOffDec + kF);

// The scratch.  Host code must not use this name as an address: the device
// address is looked up per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Copies the caller's planar [2][n] complex float block into buffer 0 of
// the equalised-symbol layout, zeroes the history before it, and resets
// the stream state of the block (unwrap start, counters, EVM sums).
__global__ void noalloc_prepare_kernel(unsigned char* scratch, const float2* __restrict__ y, long long n) {
  float2* yd = reinterpret_cast<float2*>(scratch + kOffY);
  const long long tot = 2 * (kYHist + n);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(i / (kYHist + n));
    const long long j = i - p * (kYHist + n);
    yd[p * (kYHist + kF) + j] = j < kYHist ? make_float2(0.f, 0.f) : y[p * n + (j - kYHist)];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    StreamState* st = reinterpret_cast<StreamState*>(scratch + kOffSt);
    StreamState z = {};
    z.bhat_last[0] = z.bhat_last[1] = -1;
    *st = z;
    unsigned* done = reinterpret_cast<unsigned*>(scratch + kOffDone);
    done[0] = done[1] = done[2] = done[3] = 0;
  }
}

struct DevScratch {
  unsigned char* ptr = nullptr;
  bool ready = false;
};
std::mutex g_mu;
DevScratch g_dev[64];

}  // namespace
}  // namespace rx

using namespace rx;

extern "C" int rx_decide_block_noalloc(const void* y, int64_t n, int modulation, int bps_angles,
                                       int bps_half_window, uint8_t* bits, void* cuda_stream) {
  if (!y || !bits || n < 1) {
    set_last_error("rx_decide_block_noalloc: null buffer or empty block");
    return RX_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(y) % alignof(float2) != 0) {
    set_last_error("rx_decide_block_noalloc: y must be aligned to 8 bytes (complex float)");
    return RX_EINVAL;
  }
  if (n > kMaxSyms) {
    set_last_error("rx_decide_block_noalloc: block longer than RX_NOALLOC_MAX_SYMS symbols");
    return RX_EINVAL;
  }
  if ((modulation != RX_QPSK && modulation != RX_QAM16) || (bps_angles != 32 && bps_angles != 64)) {
    set_last_error("rx_decide_block_noalloc: modulation must be RX_QPSK/RX_QAM16, bps_angles 32 or 64");
    return RX_EINVAL;
  }
  const int W = bps_half_window;
  if (W != 8 && W != 12 && W != 16 && W != 24 && W != 32) {
    set_last_error("rx_decide_block_noalloc: bps_half_window must be one of 8, 12, 16, 24, 32");
    return RX_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    set_last_error("rx_decide_block_noalloc: no current CUDA device");
    return RX_EDEVICE;
  }
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev[dev].ready) {
      // once per device, with that device current
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return RX_EDEVICE;
      }
      e = bps_set_attributes();
      if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return RX_EDEVICE;
      }
      g_dev[dev].ptr = static_cast<unsigned char*>(p);
      g_dev[dev].ready = true;
    }
    scratch = g_dev[dev].ptr;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  RxDev d;
  memset(&d, 0, sizeof(d));
  d.F = (int)kF;
  d.B = bps_angles;
  d.bps_stride = 1;
  d.bps_nw = 8;
  d.W = W;
  d.bps = modulation;
  d.nl = modulation == RX_QPSK ? 2 : 4;
  d.ber_skip = 0;
  d.out_cap_bytes = LLONG_MAX / 4;  // bits land at their stream position in the caller's buffer
  d.dec_cap = kF;
  d.y = reinterpret_cast<float2*>(scratch + kOffY);
  d.bl = reinterpret_cast<uint16_t*>(scratch + kOffBl);
  d.run_int = reinterpret_cast<int*>(scratch + kOffRunInt);
  d.run_m0 = reinterpret_cast<int*>(scratch + kOffRunM0);
  d.run_edge = reinterpret_cast<int*>(scratch + kOffRunEdge);
  d.bps_done = reinterpret_cast<unsigned*>(scratch + kOffDone);
  d.st = reinterpret_cast<StreamState*>(scratch + kOffSt);
  d.dec = scratch + kOffDec;
  d.out = bits;
  FrameArgs fa;
  memset(&fa, 0, sizeof(fa));
  fa.f = 0;
  fa.Ff = (int)n;
  fa.k_a = 0;
  fa.k_b = n;
  fa.k_end = LLONG_MAX;
  fa.n_sym = n;
  const int blocks = (int)((2 * (kYHist + n) + 255) / 256);
  noalloc_prepare_kernel<<<blocks < 1024 ? blocks : 1024, 256, 0, s>>>(scratch, static_cast<const float2*>(y), n);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_bps(d, fa, s);
  if (e == cudaSuccess) e = launch_unwrap_demap(d, fa, s);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return RX_EDEVICE;
  }
  return RX_OK;
}
