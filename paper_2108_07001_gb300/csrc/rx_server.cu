// Serving layer: many channel streams on one GPU behind one worker thread.
//
// The paper processes its ADC buffers on several CUDA streams so that
// consecutive buffers overlap on the GPU (Sec. II).  Here each channel
// stream has its own receiver (rx_handle: ring, taps, phase, timing and BER
// state stay on the device between blocks) and its own CUDA streams; the
// worker admits queued capture blocks in arrival order, round-robin over
// the streams, as soon as a stream's receiver can take them, so frames of
// different streams run concurrently.  Streams are admitted by the device
// memory their receiver holds.  Nothing here waits on the device except
// where a caller asks for it (sync, stats, close).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/rx.h"

namespace rx {
size_t handle_dev_bytes(const rx_handle* h);
void handle_progress(rx_handle* h, long long* launched, long long* done, long long* pending);
void set_last_error(const char* msg);
}  // namespace rx

namespace {

using Clock = std::chrono::steady_clock;

double now_ms() { return std::chrono::duration<double, std::milli>(Clock::now().time_since_epoch()).count(); }

int err(int code, const char* msg) {
  rx::set_last_error(msg);
  return code;
}

struct Block {
  const void* p = nullptr;    // device block, or the host copy below
  std::vector<uint8_t> host;  // host blocks are copied at submit
  size_t n = 0;
  int dtype = 0;
  int on_device = 0;
  double t_submit = 0.0;
  bool end = false;           // end-of-stream marker
};

struct Wait {
  long long frame;  // frames up to this index complete the latency sample
  double t_submit;
};

struct Stream {
  int id = 0;
  rx_handle* h = nullptr;
  int64_t bytes = 0;
  cudaStream_t cs = nullptr;  // stream the blocks are pushed on
  std::mutex hm;              // serialises every call on h
  // guarded by the server mutex
  std::deque<Block> q;
  std::vector<uint8_t> bits;  // decided bytes not yet pulled
  size_t bits_tail = 0;       // bits in the last byte of a flushed stream (0: whole bytes)
  int64_t submitted = 0, pushed = 0;
  bool end_queued = false, flushed = false, closing = false, busy = false;
  long long f_launched = 0, f_done = 0, pending = 0;
  // worker only
  std::deque<Wait> waits;
};

}  // namespace

struct rx_server {
  rx_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv;       // wakes the workers
  std::condition_variable done_cv;  // wakes sync/close waiters
  std::vector<std::thread> workers; // worker k serves the streams with id % workers == k
  bool stop = false;
  std::map<int, Stream*> streams;
  int next_id = 0;
  int64_t mem_used = 0;
  std::vector<double> lat;
  int64_t submitted = 0, pushed = 0, samples = 0, frames_done = 0;
  int werr = 0;
  std::string werr_msg;
};

namespace {

const size_t kPullChunk = 1 << 20;

// Moves decided bytes of one stream into its host buffer (worker, stream
// lock held; scratch is the worker's own buffer).  Returns RX_OK or the
// receiver's error.
int drain_bits(rx_server* s, Stream* st, std::vector<uint8_t>& scratch) {
  for (;;) {
    size_t room;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      room = (size_t)s->cfg.bits_cap_bytes > st->bits.size() ? (size_t)s->cfg.bits_cap_bytes - st->bits.size() : 0;
    }
    if (room == 0) return RX_OK;
    const size_t want = std::min(room, kPullChunk);
    if (scratch.size() < want) scratch.resize(want);
    size_t nb = 0;
    const int rc = rx_pull_bits(st->h, scratch.data(), want, &nb, 0);
    if (rc != RX_OK) return rc;
    if (nb == 0) return RX_OK;
    std::lock_guard<std::mutex> lk(s->mu);
    st->bits.insert(st->bits.end(), scratch.begin(), scratch.begin() + (nb + 7) / 8);
    if (nb % 8) st->bits_tail = nb % 8;
    if (nb < want * 8) return RX_OK;
  }
}

// Latency samples of frames completed since the last poll (worker, stream
// lock held).
void poll_frames(rx_server* s, Stream* st) {
  long long fl = 0, fd = 0, pn = 0;
  rx::handle_progress(st->h, &fl, &fd, &pn);
  const double t = now_ms();
  std::lock_guard<std::mutex> lk(s->mu);
  st->f_launched = fl;
  st->pending = pn;
  s->frames_done += fd - st->f_done;
  st->f_done = fd;
  while (!st->waits.empty() && st->waits.front().frame < fd) {
    s->lat.push_back(t - st->waits.front().t_submit);
    st->waits.pop_front();
  }
}

void set_worker_error(rx_server* s, int rc) {
  std::lock_guard<std::mutex> lk(s->mu);
  if (!s->werr) {
    s->werr = rc;
    s->werr_msg = rx_last_error();
  }
}

// One pass of worker k over its streams; true if anything was pushed.
bool worker_pass(rx_server* s, int k, std::vector<uint8_t>& scratch) {
  bool progressed = false;
  std::vector<Stream*> order;
  const int nw = (int)s->workers.size();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& kv : s->streams)
      if (!kv.second->closing && kv.first % nw == k) {
        kv.second->busy = true;
        order.push_back(kv.second);
      }
  }
  for (Stream* st : order) {
    std::lock_guard<std::mutex> hl(st->hm);
    int rc = drain_bits(s, st, scratch);
    // push queued blocks while the receiver takes them
    while (rc == RX_OK) {
      Block* b = nullptr;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        if (!st->q.empty()) b = &st->q.front();
      }
      if (!b) break;
      long long fl0 = 0, fd0 = 0, pn0 = 0;
      rx::handle_progress(st->h, &fl0, &fd0, &pn0);
      const int prc = b->end ? rx_push_block(st->h, nullptr, 0, RX_C64, 1, st->cs)
                             : rx_push_block(st->h, b->p, b->n, b->dtype, b->on_device, st->cs);
      if (prc == RX_EAGAIN) {  // output ring full: make room, try again next pass
        rc = drain_bits(s, st, scratch);
        break;
      }
      if (prc != RX_OK) {
        rc = prc;
        break;
      }
      long long fl1 = 0, fd1 = 0, pn1 = 0;
      rx::handle_progress(st->h, &fl1, &fd1, &pn1);
      if (fl1 > fl0) st->waits.push_back(Wait{fl1 - 1, b->t_submit});
      std::lock_guard<std::mutex> lk(s->mu);
      if (b->end) {
        st->flushed = true;
      } else {
        st->pushed++;
        s->pushed++;
        s->samples += (int64_t)b->n;
      }
      st->q.pop_front();
      progressed = true;
    }
    if (rc == RX_OK) {
      poll_frames(s, st);
      rc = drain_bits(s, st, scratch);
    }
    if (rc != RX_OK) set_worker_error(s, rc);
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (Stream* st : order) st->busy = false;
  }
  s->done_cv.notify_all();
  return progressed;
}

void worker_main(rx_server* s, int k) {
  cudaSetDevice(s->cfg.device);
  std::vector<uint8_t> scratch;
  const int nw = (int)s->workers.size();
  for (;;) {
    bool work;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop) return;
      work = false;
      for (auto& kv : s->streams)
        if (kv.first % nw == k && (!kv.second->q.empty() || kv.second->pending > 0)) work = true;
      if (!work) s->cv.wait_for(lk, std::chrono::microseconds(200));
      if (s->stop) return;
    }
    if (!worker_pass(s, k, scratch)) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

Stream* find(rx_server* s, int id) {
  auto it = s->streams.find(id);
  return it == s->streams.end() ? nullptr : it->second;
}

double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const size_t i = std::min(v.size() - 1, (size_t)(p * (double)(v.size() - 1) + 0.5));
  return v[i];
}

}  // namespace

extern "C" {

void rx_server_config_default(rx_server_config* c) {
  std::memset(c, 0, sizeof(*c));
  c->mem_budget_bytes = 0;
  c->max_streams = 64;
  c->device = 0;
  c->bits_cap_bytes = 64LL << 20;
  c->workers = 4;
}

int rx_server_create(const rx_server_config* cfg, rx_server** out) {
  if (!cfg || !out) return err(RX_EINVAL, "null argument");
  *out = nullptr;
  if (cfg->max_streams < 1 || cfg->max_streams > 1024) return err(RX_EINVAL, "max_streams must be in 1..1024");
  if (cfg->bits_cap_bytes < 4096) return err(RX_EINVAL, "bits_cap_bytes must be >= 4096");
  if (cfg->workers < 1 || cfg->workers > 64) return err(RX_EINVAL, "workers must be in 1..64");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
    cudaGetLastError();
    return err(RX_EDEVICE, "no such CUDA device");
  }
  if (cudaSetDevice(cfg->device) != cudaSuccess) return err(RX_EDEVICE, "cudaSetDevice failed");
  rx_server* s = new rx_server;
  s->cfg = *cfg;
  if (s->cfg.mem_budget_bytes <= 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete s;
      return err(RX_EDEVICE, "cudaMemGetInfo failed");
    }
    s->cfg.mem_budget_bytes = std::max<int64_t>((int64_t)fr - (1LL << 30), 0);
  }
  s->workers.resize(s->cfg.workers);
  for (int k = 0; k < s->cfg.workers; ++k) s->workers[k] = std::thread(worker_main, s, k);
  *out = s;
  return RX_OK;
}

int rx_server_open(rx_server* s, const rx_config* cfg, int* stream_id) {
  if (!s || !cfg || !stream_id) return err(RX_EINVAL, "null argument");
  if (cfg->device != s->cfg.device) return err(RX_EINVAL, "stream device differs from the server's");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if ((int)s->streams.size() >= s->cfg.max_streams) return err(RX_EAGAIN, "max_streams are open");
  }
  rx_handle* h = nullptr;
  int rc = rx_create(cfg, &h);
  if (rc == RX_ENOMEM) return err(RX_EAGAIN, "device memory exhausted");
  if (rc != RX_OK) return rc;
  const int64_t bytes = (int64_t)rx::handle_dev_bytes(h);
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    rx_destroy(h);
    return err(RX_EDEVICE, "cudaStreamCreate failed");
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->mem_used + bytes > s->cfg.mem_budget_bytes) {
    rx_destroy(h);
    cudaStreamDestroy(cs);
    return err(RX_EAGAIN, "stream does not fit in the remaining device memory budget");
  }
  Stream* st = new Stream;
  st->id = s->next_id++;
  st->h = h;
  st->bytes = bytes;
  st->cs = cs;
  s->streams[st->id] = st;
  s->mem_used += bytes;
  *stream_id = st->id;
  return RX_OK;
}

int64_t rx_server_submit(rx_server* s, int stream_id, const void* samples, size_t n_per_pol, int dtype,
                         int on_device) {
  if (!s || !samples || n_per_pol == 0) return err(RX_EINVAL, "null or empty block");
  if (dtype != RX_C128 && dtype != RX_C64 && dtype != RX_C16) return err(RX_EINVAL, "bad dtype");
  Block b;
  b.n = n_per_pol;
  b.dtype = dtype;
  b.on_device = on_device ? 1 : 0;
  b.t_submit = now_ms();
  if (on_device) {
    b.p = samples;
  } else {
    const size_t esz = dtype == RX_C128 ? 16 : (dtype == RX_C64 ? 8 : 4);
    b.host.assign(static_cast<const uint8_t*>(samples), static_cast<const uint8_t*>(samples) + 2 * n_per_pol * esz);
    b.p = b.host.data();
  }
  int64_t seq;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    Stream* st = find(s, stream_id);
    if (!st || st->closing) return err(RX_EINVAL, "no such stream");
    if (st->end_queued) return err(RX_ESTATE, "submit after end of stream");
    seq = st->submitted++;
    s->submitted++;
    st->q.push_back(std::move(b));
  }
  s->cv.notify_all();
  return seq;
}

int rx_server_end(rx_server* s, int stream_id) {
  if (!s) return err(RX_EINVAL, "null server");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    Stream* st = find(s, stream_id);
    if (!st || st->closing) return err(RX_EINVAL, "no such stream");
    if (st->end_queued) return err(RX_ESTATE, "stream already ended");
    st->end_queued = true;
    Block b;
    b.end = true;
    b.t_submit = now_ms();
    st->q.push_back(std::move(b));
  }
  s->cv.notify_all();
  return RX_OK;
}

int rx_server_sync(rx_server* s, int stream_id, int timeout_ms) {
  if (!s) return err(RX_EINVAL, "null server");
  const auto t_end = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    Stream* st = find(s, stream_id);
    if (!st) return err(RX_EINVAL, "no such stream");
    if (s->werr) {
      rx::set_last_error(s->werr_msg.c_str());
      return s->werr;
    }
    if (st->q.empty() && st->pending == 0 && !st->busy) break;
    if (timeout_ms >= 0 && Clock::now() >= t_end) return err(RX_ETIMEDOUT, "sync timed out");
    s->cv.notify_all();
    s->done_cv.wait_for(lk, std::chrono::microseconds(200));
  }
  return RX_OK;
}

int rx_server_pull_bits(rx_server* s, int stream_id, uint8_t* out, size_t cap_bytes, size_t* n_bits) {
  if (!s || !n_bits || (!out && cap_bytes)) return err(RX_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  Stream* st = find(s, stream_id);
  if (!st) return err(RX_EINVAL, "no such stream");
  const size_t nb = std::min(cap_bytes, st->bits.size());
  if (nb) std::memcpy(out, st->bits.data(), nb);
  size_t bits = nb * 8;
  if (nb == st->bits.size() && st->bits_tail) bits = nb * 8 - (8 - st->bits_tail);
  if (nb == st->bits.size()) st->bits_tail = 0;
  st->bits.erase(st->bits.begin(), st->bits.begin() + nb);
  *n_bits = bits;
  s->cv.notify_all();
  return RX_OK;
}

int rx_server_stream_stats(rx_server* s, int stream_id, rx_stats_t* out) {
  if (!s || !out) return err(RX_EINVAL, "null argument");
  Stream* st;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    st = find(s, stream_id);
    if (!st) return err(RX_EINVAL, "no such stream");
  }
  std::lock_guard<std::mutex> hl(st->hm);
  return rx_stats(st->h, out);
}

rx_handle* rx_server_handle(rx_server* s, int stream_id) {
  if (!s) return nullptr;
  std::lock_guard<std::mutex> lk(s->mu);
  Stream* st = find(s, stream_id);
  return st ? st->h : nullptr;
}

int rx_server_close(rx_server* s, int stream_id) {
  if (!s) return err(RX_EINVAL, "null server");
  Stream* st;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    st = find(s, stream_id);
    if (!st) return err(RX_EINVAL, "no such stream");
    st->closing = true;  // the worker takes it no more
    while (st->busy) s->done_cv.wait_for(lk, std::chrono::microseconds(200));
    s->streams.erase(stream_id);
    s->mem_used -= st->bytes;
  }
  int rc;
  {
    std::lock_guard<std::mutex> hl(st->hm);
    rc = rx_destroy(st->h);
    cudaStreamDestroy(st->cs);
  }
  delete st;
  return rc;
}

int rx_server_stats(rx_server* s, rx_server_stats_t* out) {
  if (!s || !out) return err(RX_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->blocks_submitted = s->submitted;
  out->blocks_pushed = s->pushed;
  int64_t queued = 0;
  for (auto& kv : s->streams) queued += (int64_t)kv.second->q.size();
  out->blocks_queued = queued;
  out->samples_pushed = s->samples;
  out->frames_done = s->frames_done;
  out->latency_p50_ms = percentile(s->lat, 0.50);
  out->latency_p99_ms = percentile(s->lat, 0.99);
  out->latency_max_ms = s->lat.empty() ? 0.0 : *std::max_element(s->lat.begin(), s->lat.end());
  out->latency_samples = (int64_t)s->lat.size();
  out->mem_in_use_bytes = s->mem_used;
  out->mem_budget_bytes = s->cfg.mem_budget_bytes;
  out->streams_open = (int)s->streams.size();
  out->worker_error = s->werr;
  return RX_OK;
}

int rx_server_destroy(rx_server* s) {
  if (!s) return err(RX_EINVAL, "null server");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  for (auto& w : s->workers)
    if (w.joinable()) w.join();
  int rc = RX_OK;
  for (auto& kv : s->streams) {
    const int r = rx_destroy(kv.second->h);
    if (rc == RX_OK) rc = r;
    cudaStreamDestroy(kv.second->cs);
    delete kv.second;
  }
  delete s;
  return rc;
}

}  // extern "C"
