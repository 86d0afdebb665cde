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

extern "C" int rx_kk_push(rx_kk* h, const int16_t* codes, size_t n, int on_device, float* out, size_t out_cap,
                          size_t* n_out, void* cuda_stream) {
  if (!h || !n_out || (n > 0 && !codes)) return fail("rx_kk_push: null argument", RX_EINVAL);
  *n_out = 0;
  if (h->ended) return fail("rx_kk_push: stream already ended (rx_kk_reset starts a new one)", RX_ESTATE);
  if (n > h->cfg.max_block_samples) return fail("rx_kk_push: n exceeds max_block_samples", RX_EINVAL);
  if (on_device != 0 && on_device != 1) return fail("rx_kk_push: on_device must be 0 or 1", RX_EINVAL);
  if (n == 0) return RX_OK;
  const long long in_end = h->in_pos + (long long)n;
  const long long q = in_end - h->N / 4;
  const long long out_new = q >= h->L ? q / h->L * h->L : 0;
  const long long count = out_new - h->out_pos;
  if (count > 0 && (!out || (long long)out_cap < count))
    return fail("rx_kk_push: out is null or out_cap is smaller than the field samples this push completes",
                RX_EINVAL);
  if (cudaSetDevice(h->cfg.device) != cudaSuccess) return check_cuda(cudaGetLastError(), "rx_kk_push");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int16_t* in = codes;
  if (on_device == 0) {
    int rc = check_cuda(cudaMemcpyAsync(h->stage, codes, n * sizeof(int16_t), cudaMemcpyHostToDevice, s),
                        "rx_kk_push: host copy");
    if (rc) return rc;
    in = h->stage;
  }
  rx::KKArgs a = base_args(h, in, (long long)n, reinterpret_cast<float2*>(out), out_new);
  int rc = check_cuda(rx::launch_kk(a, h->N, count / h->L, s), "rx_kk_push: field kernel");
  if (rc) return rc;
  const long long keep_from = out_new - h->N / 4 > 0 ? out_new - h->N / 4 : 0;
  rc = check_cuda(rx::launch_kk_carry(a, h->carry[h->cur ^ 1], keep_from, s), "rx_kk_push: carry kernel");
  if (rc) return rc;
  h->cur ^= 1;
  h->in_pos = in_end;
  h->out_pos = out_new;
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
