// Autotuner for the overlap-save FFT size.
//
// The FFT size N trades the wasted halo fraction (h / N, smaller for larger
// N) against the cost per output sample of a longer transform held in one
// thread block's shared memory.  The paper fixes its block geometry for its
// own GPU (Sec. II: 1024-point blocks, buffers of 2^22 samples); here each
// admissible N is timed on this GPU with the stream's own configuration and
// the fastest is kept.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "../../include/rx.h"

namespace rx {
int cd_halo_samples(const rx_config* cfg);
void set_last_error(const char* msg);
}  // namespace rx

namespace {

// Steady-state time of `frames` frames of a zero stream (no BER) with FFT
// size N: two frames of samples are pushed untimed (the first frame, with
// the acquisition, completes once the second's look-ahead is in), then
// `frames` more frames and the end of the stream are timed.
// Milliseconds, or < 0 on error (*rc set).
double time_chain(const rx_config* base, int N, int frames, void* zeros, size_t block, int* rc) {
  rx_config c = *base;
  c.fft_n = N;
  c.prbs_seed = 0;
  c.history_syms = 0;
  c.profile = 0;
  c.max_block_samples = block;
  rx_handle* h = nullptr;
  *rc = rx_create(&c, &h);
  if (*rc != RX_OK) return -1.0;
  const long long per_frame = 2LL * c.frame_syms;
  auto push = [&](long long total) {
    for (long long a = 0; a < total && *rc == RX_OK; a += (long long)block) {
      const size_t n = (size_t)std::min<long long>((long long)block, total - a);
      *rc = rx_push_block(h, zeros, n, RX_C64, 1, nullptr);
    }
  };
  push(2 * per_frame);
  if (*rc == RX_OK) *rc = rx_join(h, nullptr);
  if (*rc == RX_OK && cudaDeviceSynchronize() != cudaSuccess) *rc = RX_EDEVICE;
  const auto t0 = std::chrono::steady_clock::now();
  push(per_frame * frames);
  if (*rc == RX_OK) *rc = rx_push_block(h, nullptr, 0, RX_C64, 1, nullptr);
  if (*rc == RX_OK) *rc = rx_join(h, nullptr);
  if (*rc == RX_OK && cudaDeviceSynchronize() != cudaSuccess) *rc = RX_EDEVICE;
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  rx_destroy(h);
  return *rc == RX_OK ? ms : -1.0;
}

}  // namespace

extern "C" int rx_autotune_fft(const rx_config* cfg, int frames, int* fft_n, double* ms_per_msample) {
  if (!cfg || !fft_n) {
    rx::set_last_error("rx_autotune_fft: null argument");
    return RX_EINVAL;
  }
  if (frames < 1 || frames > 64) {
    rx::set_last_error("rx_autotune_fft: frames must be in 1..64");
    return RX_EINVAL;
  }
  const int halo = rx::cd_halo_samples(cfg);
  std::vector<int> cand;
  for (int N = 1024; N <= 32768; N *= 2)
    if (N - halo >= 256) cand.push_back(N);
  if (cand.empty()) {
    rx::set_last_error("rx_autotune_fft: CD halo too long for every FFT size");
    return RX_EINVAL;
  }
  if (cudaSetDevice(cfg->device) != cudaSuccess) {
    cudaGetLastError();
    rx::set_last_error("rx_autotune_fft: no such CUDA device");
    return RX_EDEVICE;
  }
  const size_t block = std::min<size_t>(cfg->max_block_samples ? cfg->max_block_samples : (1u << 17), 1u << 20);
  void* zeros = nullptr;
  if (cudaMalloc(&zeros, 2 * block * 8) != cudaSuccess) {
    cudaGetLastError();
    rx::set_last_error("rx_autotune_fft: cudaMalloc failed");
    return RX_ENOMEM;
  }
  cudaMemset(zeros, 0, 2 * block * 8);
  int best_n = 0, rc = RX_OK;
  double best_ms = 0.0;
  for (int N : cand) {
    const double ms = time_chain(cfg, N, frames, zeros, block, &rc);
    if (rc != RX_OK) break;
    if (best_n == 0 || ms < best_ms) {
      best_n = N;
      best_ms = ms;
    }
  }
  cudaFree(zeros);
  if (rc != RX_OK) return rc;
  *fft_n = best_n;
  if (ms_per_msample) *ms_per_msample = best_ms / ((double)frames * 2.0 * cfg->frame_syms / (double)(1 << 20));
  return RX_OK;
}
