// Autotuners: the overlap-save FFT size, and the launch tiles of the
// equaliser and blind-phase-search kernels.
//
// The FFT size N trades the wasted halo fraction (h / N, smaller for larger
// N) against the cost per output sample of a longer transform held in one
// thread block's shared memory.  The paper fixes its block geometry for its
// own GPU (Sec. II: 1024-point blocks, buffers of 2^22 samples); here each
// admissible N is timed on this GPU with the stream's own configuration and
// the fastest is kept.  The tiles (segment chains per block of the
// equaliser, 256-symbol runs per block of the full blind phase search) do
// not change any result, only how the work packs onto the SMs beside the
// other stages; they are timed the same way, one after the other, with the
// size already chosen.
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
  c.fft_n = N;  // tiles as in base
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

// The fastest admissible FFT size (tiles as in cfg); on success *fft_n
// and *best_ms hold it and its time.
int tune_fft(const rx_config* cfg, int frames, void* zeros, size_t block, int* fft_n, double* best_ms) {
  const int halo = rx::cd_halo_samples(cfg);
  std::vector<int> cand;
  for (int N = 1024; N <= 32768; N *= 2)
    if (N - halo >= 256) cand.push_back(N);
  if (cand.empty()) {
    rx::set_last_error("rx_autotune_fft: CD halo too long for every FFT size");
    return RX_EINVAL;
  }
  int best_n = 0, rc = RX_OK;
  double best = 0.0;
  for (int N : cand) {
    const double ms = time_chain(cfg, N, frames, zeros, block, &rc);
    if (rc != RX_OK) return rc;
    if (best_n == 0 || ms < best) {
      best_n = N;
      best = ms;
    }
  }
  *fft_n = best_n;
  *best_ms = best;
  return RX_OK;
}

int check_args(const rx_config* cfg, int frames, const void* out) {
  if (!cfg || !out) {
    rx::set_last_error("rx_autotune: null argument");
    return RX_EINVAL;
  }
  if (frames < 1 || frames > 64) {
    rx::set_last_error("rx_autotune: frames must be in 1..64");
    return RX_EINVAL;
  }
  const int halo = rx::cd_halo_samples(cfg);
  if (32768 - halo < 256) {
    rx::set_last_error("rx_autotune_fft: CD halo too long for every FFT size");
    return RX_EINVAL;
  }
  if (cudaSetDevice(cfg->device) != cudaSuccess) {
    cudaGetLastError();
    rx::set_last_error("rx_autotune: no such CUDA device");
    return RX_EDEVICE;
  }
  return RX_OK;
}

}  // namespace

extern "C" int rx_autotune_fft(const rx_config* cfg, int frames, int* fft_n, double* ms_per_msample) {
  int rc = check_args(cfg, frames, fft_n);
  if (rc != RX_OK) return rc;
  const size_t block = std::min<size_t>(cfg->max_block_samples ? cfg->max_block_samples : (1u << 17), 1u << 20);
  void* zeros = nullptr;
  if (cudaMalloc(&zeros, 2 * block * 8) != cudaSuccess) {
    cudaGetLastError();
    rx::set_last_error("rx_autotune_fft: cudaMalloc failed");
    return RX_ENOMEM;
  }
  cudaMemset(zeros, 0, 2 * block * 8);
  double best = 0.0;
  rc = tune_fft(cfg, frames, zeros, block, fft_n, &best);
  cudaFree(zeros);
  if (rc != RX_OK) return rc;
  if (ms_per_msample) *ms_per_msample = best / ((double)frames * 2.0 * cfg->frame_syms / (double)(1 << 20));
  return RX_OK;
}

extern "C" int rx_autotune_tiles(const rx_config* cfg, int frames, int* fft_n, int* mimo_block_warps,
                                 int* bps_block_runs, double* ms_per_msample) {
  if (!mimo_block_warps || !bps_block_runs) {
    rx::set_last_error("rx_autotune_tiles: null argument");
    return RX_EINVAL;
  }
  int rc = check_args(cfg, frames, fft_n);
  if (rc != RX_OK) return rc;
  const size_t block = std::min<size_t>(cfg->max_block_samples ? cfg->max_block_samples : (1u << 17), 1u << 20);
  void* zeros = nullptr;
  if (cudaMalloc(&zeros, 2 * block * 8) != cudaSuccess) {
    cudaGetLastError();
    rx::set_last_error("rx_autotune_tiles: cudaMalloc failed");
    return RX_ENOMEM;
  }
  cudaMemset(zeros, 0, 2 * block * 8);
  rx_config c = *cfg;
  c.mimo_block_warps = 4;
  c.bps_block_runs = 8;
  double best = 0.0;
  rc = tune_fft(&c, frames, zeros, block, &c.fft_n, &best);
  // each tile in turn, the others at their current best; a candidate is
  // kept only if it beats the incumbent's time by more than 1 %
  const int mimo_cand[] = {1, 2, 4, 8};
  const int bps_cand[] = {4, 8};
  for (int pass = 0; pass < 2 && rc == RX_OK; ++pass) {
    const int* cand = pass == 0 ? mimo_cand : bps_cand;
    const int nc = pass == 0 ? 4 : 2;
    if (pass == 1 && c.bps_coarse_stride > 1) break;  // the two-stage search has one layout
    for (int k = 0; k < nc && rc == RX_OK; ++k) {
      rx_config t = c;
      (pass == 0 ? t.mimo_block_warps : t.bps_block_runs) = cand[k];
      if ((pass == 0 ? c.mimo_block_warps : c.bps_block_runs) == cand[k]) continue;
      const double ms = time_chain(&t, t.fft_n, frames, zeros, block, &rc);
      if (rc == RX_OK && ms < 0.99 * best) {
        c = t;
        best = ms;
      }
    }
  }
  cudaFree(zeros);
  if (rc != RX_OK) return rc;
  *fft_n = c.fft_n;
  *mimo_block_warps = c.mimo_block_warps;
  *bps_block_runs = c.bps_block_runs;
  if (ms_per_msample) *ms_per_msample = best / ((double)frames * 2.0 * cfg->frame_syms / (double)(1 << 20));
  return RX_OK;
}
