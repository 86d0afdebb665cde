// Host runtime of the Kramers-Kronig front end: stream positions, the carry
// of samples that later segments still need, staging of host pushes and the
// launches (paper Sec. II: a kernel joins each buffer to the end of the
// previous one so that the overlap-save blocks see a contiguous stream).
//
// Positions: in_pos samples pushed, out_pos field samples written (a whole
// number of segments of L = N/2 until the end).  Segment b needs input up
// to b L + 3N/4, so after a push out_pos = floor((in_pos - N/4) / L) L.
// The carry holds the codes of [max(0, out_pos - N/4), in_pos): the left
// half-block of the next segment and every sample not yet output (fewer
// than N).  Two carry buffers alternate: the field kernel of a push reads
// one while the carry kernel after it fills the other, in stream order.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/rx.h"
#include "kk_internal.h"

namespace rx {
void set_last_error(const char* msg);
}

struct rx_kk {
  rx_kk_config cfg;
  int N = 0, L = 0;
  long long in_pos = 0, out_pos = 0;
  bool ended = false;
  int cur = 0;                      // carry buffer holding [carry_start, in_pos)
  int16_t* carry[2] = {nullptr, nullptr};
  int16_t* stage = nullptr;         // host pushes land here
  float2* tw2 = nullptr;
  unsigned long long nu_fx = 0;
};

namespace {

int fail(const char* msg, int rc) {
  rx::set_last_error(msg);
  return rc;
}

int check_cuda(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return RX_OK;
  static thread_local char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  cudaGetLastError();
  return fail(buf, RX_EDEVICE);
}

// frac(f_shift / fs) as a 64-bit binary fraction: exact for integral rates
// (both below 2^53 Hz), else to double precision.
unsigned long long nu_fixed(double f_shift, double fs) {
  if (f_shift == std::floor(f_shift) && fs == std::floor(fs) && std::fabs(f_shift) < 9.0e15 && fs < 9.0e15) {
    const long long F = (long long)fs;
    long long r = (long long)f_shift % F;
    if (r < 0) r += F;
    return (unsigned long long)(((unsigned __int128)r << 64) / (unsigned __int128)F);
  }
  double x = f_shift / fs;
  x -= std::floor(x);
  return (unsigned long long)std::ldexp(x, 64);
}

rx::KKArgs base_args(const rx_kk* h, const int16_t* in, long long n_new, float2* out, long long out_new) {
  rx::KKArgs a;
  a.carry = h->carry[h->cur];
  a.in = in;
  a.carry_start = h->out_pos - h->N / 4 > 0 ? h->out_pos - h->N / 4 : 0;
  a.new_start = h->in_pos;
  a.in_end = h->in_pos + n_new;
  a.seg0 = h->out_pos / h->L;
  a.out_start = h->out_pos;
  a.out_end = out_new;
  a.out = out;
  a.tw2 = h->tw2;
  a.gain = (float)h->cfg.adc_gain;
  a.offset = (float)h->cfg.adc_offset;
  a.i_min = (float)(0.5 * h->cfg.adc_gain);
  a.nu_fx = h->nu_fx;
  return a;
}

}  // namespace

extern "C" void rx_kk_config_default(rx_kk_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->fs_hz = 4e9;
  c->f_shift_hz = 0.516e9;
  c->adc_gain = 1.0;
  c->adc_offset = 0.0;
  c->fft_n = 1024;
  c->max_block_samples = (size_t)1 << 22;
  c->device = 0;
}

extern "C" int rx_kk_create(const rx_kk_config* cfg, rx_kk** out) {
  if (!cfg || !out) return fail("rx_kk_create: null argument", RX_EINVAL);
  *out = nullptr;
  if (cfg->fft_n != 1024 && cfg->fft_n != 2048 && cfg->fft_n != 4096)
    return fail("rx_kk_create: fft_n must be 1024, 2048 or 4096", RX_EINVAL);
  if (!(cfg->fs_hz > 0.0)) return fail("rx_kk_create: fs_hz must be > 0", RX_EINVAL);
  if (!(cfg->adc_gain > 0.0)) return fail("rx_kk_create: adc_gain must be > 0", RX_EINVAL);
  if (!std::isfinite(cfg->f_shift_hz) || !std::isfinite(cfg->adc_offset))
    return fail("rx_kk_create: f_shift_hz and adc_offset must be finite", RX_EINVAL);
  if (cfg->max_block_samples < 1 || cfg->max_block_samples > ((size_t)1 << 31))
    return fail("rx_kk_create: max_block_samples must be in 1..2^31", RX_EINVAL);
  if (cudaSetDevice(cfg->device) != cudaSuccess) {
    cudaGetLastError();
    return fail("rx_kk_create: no such CUDA device", RX_EDEVICE);
  }
  rx_kk* h = new rx_kk;
  h->cfg = *cfg;
  h->N = cfg->fft_n;
  h->L = cfg->fft_n / 2;
  h->nu_fx = nu_fixed(cfg->f_shift_hz, cfg->fs_hz);
  bool ok = cudaMalloc(&h->carry[0], h->N * sizeof(int16_t)) == cudaSuccess &&
            cudaMalloc(&h->carry[1], h->N * sizeof(int16_t)) == cudaSuccess &&
            cudaMalloc(&h->stage, cfg->max_block_samples * sizeof(int16_t)) == cudaSuccess &&
            cudaMalloc(&h->tw2, 256 * sizeof(float2)) == cudaSuccess;
  if (ok) {
    // two-level twiddles exp(-2 pi i m / N), m = hi 128 + lo, in FP64
    std::vector<float2> tw(256);
    for (int i = 0; i < 128; ++i) {
      const double ah = -2.0 * M_PI * (double)(i * 128) / h->N, al = -2.0 * M_PI * (double)i / h->N;
      tw[i] = make_float2((float)std::cos(ah), (float)std::sin(ah));
      tw[128 + i] = make_float2((float)std::cos(al), (float)std::sin(al));
    }
    ok = cudaMemcpy(h->tw2, tw.data(), 256 * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    rx_kk_destroy(h);
    return fail("rx_kk_create: device allocation failed", RX_ENOMEM);
  }
  *out = h;
  return RX_OK;
}

namespace {

// One push of n > 0 codes (already on the device at `in`), planned without
// launching: the field kernel's arguments and segment pairs, the carry
// copy's destination and start, and the positions after it.
struct KKPlan {
  rx::KKArgs a;
  long long pairs, keep_from, in_end, out_new;
  int16_t* carry_dst;
};

int kk_check(const rx_kk* h, size_t n, float* out, size_t out_cap, long long* count) {
  if (h->ended) return fail("rx_kk push: stream already ended (rx_kk_reset starts a new one)", RX_ESTATE);
  if (n > h->cfg.max_block_samples) return fail("rx_kk push: n exceeds max_block_samples", RX_EINVAL);
  const long long in_end = h->in_pos + (long long)n;
  const long long q = in_end - h->N / 4;
  const long long out_new = q >= h->L ? q / h->L * h->L : 0;
  *count = out_new - h->out_pos;
  if (*count > 0 && (!out || (long long)out_cap < *count))
    return fail("rx_kk push: out is null or out_cap is smaller than the field samples the push completes",
                RX_EINVAL);
  return RX_OK;
}

KKPlan kk_plan(const rx_kk* h, const int16_t* in, size_t n, float* out) {
  KKPlan p;
  p.in_end = h->in_pos + (long long)n;
  const long long q = p.in_end - h->N / 4;
  p.out_new = q >= h->L ? q / h->L * h->L : 0;
  p.a = base_args(h, in, (long long)n, reinterpret_cast<float2*>(out), p.out_new);
  p.pairs = ((p.out_new - h->out_pos) / h->L + 1) / 2;
  p.keep_from = p.out_new - h->N / 4 > 0 ? p.out_new - h->N / 4 : 0;
  p.carry_dst = h->carry[h->cur ^ 1];
  return p;
}

void kk_commit(rx_kk* h, const KKPlan& p) {
  h->cur ^= 1;
  h->in_pos = p.in_end;
  h->out_pos = p.out_new;
}

}  // namespace

extern "C" int rx_kk_push(rx_kk* h, const int16_t* codes, size_t n, int on_device, float* out, size_t out_cap,
                          size_t* n_out, void* cuda_stream) {
  if (!h || !n_out || (n > 0 && !codes)) return fail("rx_kk_push: null argument", RX_EINVAL);
  *n_out = 0;
  if (on_device != 0 && on_device != 1) return fail("rx_kk_push: on_device must be 0 or 1", RX_EINVAL);
  long long count = 0;
  int rc = kk_check(h, n, out, out_cap, &count);
  if (rc) return rc;
  if (n == 0) return RX_OK;
  if (cudaSetDevice(h->cfg.device) != cudaSuccess) return check_cuda(cudaGetLastError(), "rx_kk_push");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int16_t* in = codes;
  if (on_device == 0) {
    rc = check_cuda(cudaMemcpyAsync(h->stage, codes, n * sizeof(int16_t), cudaMemcpyHostToDevice, s),
                    "rx_kk_push: host copy");
    if (rc) return rc;
    in = h->stage;
  }
  const KKPlan p = kk_plan(h, in, n, out);
  rc = check_cuda(rx::launch_kk(p.a, h->N, count / h->L, s), "rx_kk_push: field kernel");
  if (rc) return rc;
  rc = check_cuda(rx::launch_kk_carry(p.a, p.carry_dst, p.keep_from, s), "rx_kk_push: carry kernel");
  if (rc) return rc;
  kk_commit(h, p);
  *n_out = (size_t)count;
  return RX_OK;
}

extern "C" int rx_kk_end(rx_kk* h, float* out, size_t out_cap, size_t* n_out, void* cuda_stream) {
  if (!h || !n_out) return fail("rx_kk_end: null argument", RX_EINVAL);
  *n_out = 0;
  if (h->ended) return fail("rx_kk_end: stream already ended", RX_ESTATE);
  const long long count = h->in_pos - h->out_pos;
  if (count > 0 && (!out || (long long)out_cap < count))
    return fail("rx_kk_end: out is null or out_cap is smaller than the remaining field samples", RX_EINVAL);
  if (count > 0) {
    if (cudaSetDevice(h->cfg.device) != cudaSuccess) return check_cuda(cudaGetLastError(), "rx_kk_end");
    // every sample still needed is in the carry; past in_pos is absent
    rx::KKArgs a = base_args(h, nullptr, 0, reinterpret_cast<float2*>(out), h->in_pos);
    const int rc = check_cuda(rx::launch_kk(a, h->N, (count + h->L - 1) / h->L, (cudaStream_t)cuda_stream),
                              "rx_kk_end: field kernel");
    if (rc) return rc;
  }
  h->out_pos = h->in_pos;
  h->ended = true;
  *n_out = (size_t)count;
  return RX_OK;
}

extern "C" int rx_kk_reset(rx_kk* h) {
  if (!h) return fail("rx_kk_reset: null handle", RX_EINVAL);
  h->in_pos = h->out_pos = 0;
  h->ended = false;
  h->cur = 0;
  return RX_OK;
}

extern "C" int rx_kk_position(const rx_kk* h, int64_t* samples_in, int64_t* samples_out) {
  if (!h) return fail("rx_kk_position: null handle", RX_EINVAL);
  if (samples_in) *samples_in = h->in_pos;
  if (samples_out) *samples_out = h->out_pos;
  return RX_OK;
}

extern "C" void rx_kk_destroy(rx_kk* h) {
  if (!h) return;
  cudaSetDevice(h->cfg.device);
  cudaFree(h->carry[0]);
  cudaFree(h->carry[1]);
  cudaFree(h->stage);
  cudaFree(h->tw2);
  delete h;
}

// ---- many channels in one graph launch ------------------------------------
//
// A batch push plans every channel's push on the host, writes the plans to
// a table in page-locked memory and replays a graph of three nodes: the
// table's copy to the device, the batched field kernel (one block per
// segment pair of any channel; a block finds its channel from the
// prefix sums of the channels' uneven pair counts) and the batched carry
// kernel (one block per channel).  Only the field node's grid changes
// between replays.  Two table slots, each with its own graph, alternate;
// a slot's host table is rewritten only after its previous copy ran.

struct rx_kk_batch {
  std::vector<rx_kk*> ch;
  int N = 0, device = 0, slot = 0;
  rx::KKBatchTable* host_tab[2] = {nullptr, nullptr};
  rx::KKBatchTable* dev_tab[2] = {nullptr, nullptr};
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaGraphNode_t field_node[2] = {nullptr, nullptr};
  cudaKernelNodeParams field_params[2];
  cudaEvent_t done[2] = {nullptr, nullptr};
  bool used[2] = {false, false};
};

extern "C" int rx_kk_batch_create(rx_kk* const* channels, int n_channels, rx_kk_batch** out) {
  if (!channels || !out || n_channels < 1) return fail("rx_kk_batch_create: null argument or no channels", RX_EINVAL);
  *out = nullptr;
  if (n_channels > rx::kKKBatchMax) return fail("rx_kk_batch_create: at most 256 channels", RX_EINVAL);
  for (int c = 0; c < n_channels; ++c) {
    if (!channels[c]) return fail("rx_kk_batch_create: null channel", RX_EINVAL);
    if (channels[c]->N != channels[0]->N || channels[c]->cfg.device != channels[0]->cfg.device)
      return fail("rx_kk_batch_create: channels must share fft_n and device", RX_EINVAL);
    for (int d = 0; d < c; ++d)
      if (channels[d] == channels[c]) return fail("rx_kk_batch_create: a channel appears twice", RX_EINVAL);
  }
  rx_kk_batch* b = new rx_kk_batch;
  b->ch.assign(channels, channels + n_channels);
  b->N = channels[0]->N;
  b->device = channels[0]->cfg.device;
  int rc = check_cuda(cudaSetDevice(b->device), "rx_kk_batch_create");
  for (int k = 0; k < 2 && rc == RX_OK; ++k) {
    rc = check_cuda(cudaHostAlloc(&b->host_tab[k], sizeof(rx::KKBatchTable), cudaHostAllocDefault), "table");
    if (!rc) rc = check_cuda(cudaMalloc(&b->dev_tab[k], sizeof(rx::KKBatchTable)), "table");
    if (!rc) rc = check_cuda(cudaEventCreateWithFlags(&b->done[k], cudaEventDisableTiming), "event");
    if (!rc) {
      std::memset(b->host_tab[k], 0, sizeof(rx::KKBatchTable));
      cudaKernelNodeParams field, carry;
      rc = check_cuda(rx::kk_batch_nodes(b->N, &field, &carry), "rx_kk_batch_create: kernels");
      if (!rc) rc = check_cuda(cudaGraphCreate(&b->graph[k], 0), "graph");
      cudaGraphNode_t copy = nullptr, cnode = nullptr;
      if (!rc)
        rc = check_cuda(cudaGraphAddMemcpyNode1D(&copy, b->graph[k], nullptr, 0, b->dev_tab[k], b->host_tab[k],
                                                 sizeof(rx::KKBatchTable), cudaMemcpyHostToDevice),
                        "graph copy node");
      // kernelParams holds the address of the table pointer; the value is copied when the node is added
      void* tab_arg[1] = {&b->dev_tab[k]};
      field.gridDim = dim3(1);
      field.kernelParams = tab_arg;
      carry.gridDim = dim3((unsigned)n_channels);
      carry.kernelParams = tab_arg;
      if (!rc) rc = check_cuda(cudaGraphAddKernelNode(&b->field_node[k], b->graph[k], &copy, 1, &field), "field node");
      if (!rc) rc = check_cuda(cudaGraphAddKernelNode(&cnode, b->graph[k], &b->field_node[k], 1, &carry), "carry node");
      if (!rc) rc = check_cuda(cudaGraphInstantiate(&b->exec[k], b->graph[k], 0), "graph instantiate");
      b->field_params[k] = field;
    }
  }
  if (rc) {
    rx_kk_batch_destroy(b);
    return rc;
  }
  *out = b;
  return RX_OK;
}

extern "C" int rx_kk_batch_push(rx_kk_batch* b, const int16_t* const* codes, const size_t* n, float* const* out,
                                const size_t* out_cap, size_t* n_out, void* cuda_stream) {
  if (!b || !codes || !n || !out || !out_cap || !n_out) return fail("rx_kk_batch_push: null argument", RX_EINVAL);
  const int nch = (int)b->ch.size();
  for (int c = 0; c < nch; ++c) {  // all or nothing: check every channel first
    n_out[c] = 0;
    long long count = 0;
    if (n[c] > 0 && !codes[c]) return fail("rx_kk_batch_push: null codes", RX_EINVAL);
    const int rc = kk_check(b->ch[c], n[c], out[c], out_cap[c], &count);
    if (rc) return rc;
  }
  int rc = check_cuda(cudaSetDevice(b->device), "rx_kk_batch_push");
  if (rc) return rc;
  const int k = b->slot;
  if (b->used[k]) {
    rc = check_cuda(cudaEventSynchronize(b->done[k]), "rx_kk_batch_push: table slot");
    if (rc) return rc;
  }
  rx::KKBatchTable* t = b->host_tab[k];
  std::vector<KKPlan> plans(nch);
  t->nch = nch;
  t->offs[0] = 0;
  for (int c = 0; c < nch; ++c) {
    rx_kk* h = b->ch[c];
    if (n[c] == 0) {  // nothing new: no blocks, an empty carry copy, no position change
      plans[c].a = base_args(h, nullptr, 0, reinterpret_cast<float2*>(out[c]), h->out_pos);
      plans[c].pairs = 0;
      plans[c].keep_from = h->in_pos;
      plans[c].carry_dst = h->carry[h->cur ^ 1];
    } else {
      plans[c] = kk_plan(h, codes[c], n[c], out[c]);
    }
    t->args[c] = plans[c].a;
    t->offs[c + 1] = t->offs[c] + plans[c].pairs;
    t->carry_dst[c] = plans[c].carry_dst;
    t->keep_from[c] = plans[c].keep_from;
  }
  const long long blocks = t->offs[nch];
  if (blocks > 0x7fffffffLL) return fail("rx_kk_batch_push: too many segments in one batch", RX_EINVAL);
  cudaKernelNodeParams fp = b->field_params[k];
  void* arg[1] = {&b->dev_tab[k]};
  fp.kernelParams = arg;
  fp.gridDim = dim3((unsigned)std::max(1LL, blocks));
  rc = check_cuda(cudaGraphExecKernelNodeSetParams(b->exec[k], b->field_node[k], &fp), "rx_kk_batch_push: grid");
  if (!rc) rc = check_cuda(cudaGraphLaunch(b->exec[k], (cudaStream_t)cuda_stream), "rx_kk_batch_push: graph");
  if (!rc) rc = check_cuda(cudaEventRecord(b->done[k], (cudaStream_t)cuda_stream), "rx_kk_batch_push: event");
  if (rc) return rc;
  b->used[k] = true;
  b->slot ^= 1;
  for (int c = 0; c < nch; ++c) {
    if (n[c] == 0) continue;
    n_out[c] = (size_t)(plans[c].out_new - b->ch[c]->out_pos);
    kk_commit(b->ch[c], plans[c]);
  }
  return RX_OK;
}

extern "C" void rx_kk_batch_destroy(rx_kk_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  for (int k = 0; k < 2; ++k) {
    if (b->done[k]) cudaEventSynchronize(b->done[k]);
    if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
    if (b->graph[k]) cudaGraphDestroy(b->graph[k]);
    if (b->done[k]) cudaEventDestroy(b->done[k]);
    cudaFreeHost(b->host_tab[k]);
    cudaFree(b->dev_tab[k]);
  }
  delete b;
}
