// Arguments of the KK receiver's equaliser and DD-LMS kernels (k_kkrx.cu),
// filled by the chain's host runtime (rx_kkrx.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rx {

struct KKEqArgs {
  const float2* carry;           // 4-sps field of stream samples [carry_start, new_start)
  const float2* in;              // field of [new_start, in_end) (this step's new samples)
  long long carry_start, new_start, in_end;
  long long seg0;                // first output segment (segment b = 2-sps samples [b N4/4, (b+1) N4/4))
  float2* out;                   // 2-sps sample t goes to out[t - out_base], t < out_end
  long long out_base, out_end;
  const float2* H2;              // N4/2 bins: CD compensation x RRC, 1/N4 folded in
  const float2* tw2;             // two-level twiddle table of N4
};

struct WLArgs {
  const float2* x2;              // 2-sps samples: x[i] = x2[i - x2_base] for 0 <= i < n2, else 0
  long long x2_base, n2;
  long long k_a, k_end;          // symbols of the launch; block j = segment [k_a + j seg, ...)
  long long seg;
  const float2* taps_in;         // (h1[4], h2[4]) per segment, taps_in_stride apart (0: shared)
  long long taps_in_stride;
  float2* taps_out;              // 8 per segment
  float mu;
  uint8_t* bits;                 // packed bits, symbol k at bit (k - k_bits) * bits per symbol; null: none
  long long k_bits;
  float2* hist;                  // equalised symbols k < hist_syms; null: none
  long long hist_syms;
};

// Equaliser arguments of many channels in one launch: channel c's blocks
// are [offs[c], offs[c + 1]); its carry goes to carry_dst[c] from keep_from[c].
constexpr int kKKEqBatchMax = 256;
struct KKEqBatchTable {
  int nch;
  int pad;
  long long offs[kKKEqBatchMax + 1];
  KKEqArgs args[kKKEqBatchMax];
  float2* carry_dst[kKKEqBatchMax];
  long long keep_from[kKKEqBatchMax];
};

// DD-LMS work of many channels: node 0 holds the acquisitions, node 1 + i
// the i-th frame each channel completed (a channel's frames run in order,
// one node after the other); entry e of a node has blocks
// [offs[node][e], offs[node][e + 1]).  Then the moves of the channels'
// remaining 2-sps samples.
constexpr int kWLNodes = 5;
struct WLBatchTable {
  int n[kWLNodes];
  int nshift;
  long long offs[kWLNodes][kKKEqBatchMax + 1];
  WLArgs args[kWLNodes][kKKEqBatchMax];
  const float2* shift_src[kKKEqBatchMax];
  float2* shift_dst[kKKEqBatchMax];
  long long shift_n[kKKEqBatchMax];
};

cudaError_t launch_wl_batch(const WLBatchTable* t, int node, bool q16, long long blocks, cudaStream_t s);
cudaError_t launch_x2_shift_batch(const WLBatchTable* t, int n, cudaStream_t s);

cudaError_t launch_kkeq(const KKEqArgs& a, int N4, long long nseg, cudaStream_t s);
// Kernel-node templates of the batched equaliser and its carries (grid and
// arguments are the caller's).
cudaError_t kkeq_batch_nodes(int N4, cudaKernelNodeParams* eq, cudaKernelNodeParams* tail);
cudaError_t launch_kkeq_tail(const float2* carry, long long carry_start, const float2* in, long long new_start,
                             long long keep_from, long long in_end, float2* dst, cudaStream_t s);
cudaError_t launch_wl(const WLArgs& a, bool q16, long long nseg, cudaStream_t s);

}  // namespace rx
