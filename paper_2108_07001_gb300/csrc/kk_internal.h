// Arguments of the Kramers-Kronig front-end kernels (k_kk.cu), filled by
// the host runtime (rx_kk.cu) for every push.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rx {

struct KKArgs {
  const int16_t* carry;          // codes of stream samples [carry_start, new_start)
  const int16_t* in;             // codes of stream samples [new_start, in_end) (this push)
  long long carry_start, new_start, in_end;
  long long seg0;                // first segment of the launch (segment b = samples [b L, (b+1) L))
  long long out_start, out_end;  // field of sample t goes to out[t - out_start], t < out_end
  float2* out;
  const float2* tw2;             // two-level twiddle table of the FFT size
  float gain, offset, i_min;     // I = gain (code - offset), floor i_min
  unsigned long long nu_fx;      // downshift frequency / sample rate, fixed point 2^-64
};

// Arguments of many channels' pushes in one launch (rx_kk_batch_push):
// channel c's blocks are [offs[c], offs[c + 1]).
constexpr int kKKBatchMax = 256;
struct KKBatchTable {
  int nch;
  int pad;
  long long offs[kKKBatchMax + 1];
  KKArgs args[kKKBatchMax];
  int16_t* carry_dst[kKKBatchMax];
  long long keep_from[kKKBatchMax];
};

cudaError_t launch_kk(const KKArgs& a, int N, long long nseg, cudaStream_t s);
// Kernel-node templates (function, block, shared memory) of the batched
// field and carry kernels for a graph; grid and arguments are the caller's.
cudaError_t kk_batch_nodes(int N, cudaKernelNodeParams* field, cudaKernelNodeParams* carry);
cudaError_t launch_kk_carry(const KKArgs& a, int16_t* dst, long long keep_from, cudaStream_t s);

}  // namespace rx
