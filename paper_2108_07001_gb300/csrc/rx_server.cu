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
//
// Batched mode (rx_server_config.batch = 1): one worker forms rounds.  A
// round takes the first queued block of every stream that has one and
// pushes the device-memory blocks of one input type together through one
// rx_batch_push, so each stage of every stream's completed frames runs in
// one launch (rx_batch); pageable host blocks, and blocks of the round's
// other input types, go through the stream's own rx_push_block.  The batch
// holds the open streams' receivers; when a stream opens or closes, the
// worker replaces it (rx_batch_destroy waits for the old batch's work), so
// a stream's receiver is destroyed only after no batch refers to it.
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
int pull_bits_begin(rx_handle* h, uint8_t* out, size_t cap_bytes, size_t* n_bits, cudaStream_t cs);
void pull_bits_commit(rx_handle* h, size_t n_bits);
long long handle_launched(const rx_handle* h);
long long batch_calls_done(rx_batch* b);
bool batch_try_free(rx_batch* b);
void handle_bits(const rx_handle* h, long long* ready, long long* ring_bits);
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
  bool in_batch = false;      // batched mode: the current batch refers to this stream's receiver
  bool undrained = false;     // batched mode: decided bits the worker still has to move to `bits`
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
  // batched mode (worker only, except members' in_batch flags under mu)
  rx_batch* batch = nullptr;
  std::vector<Stream*> members;     // the batch's streams, in its order
  // replaced batches whose work may still run, with their streams
  std::vector<std::pair<rx_batch*, std::vector<Stream*>>> retired;
  cudaStream_t bcs = nullptr;       // stream the batched ingests run on
  cudaStream_t dcs = nullptr;       // stream of the bit copies to the host
  uint8_t* pinned = nullptr;        // page-locked landing area of those copies
  size_t pinned_bytes = 0;
  cudaEvent_t drain_ev = nullptr;   // end of the bit copies in flight
  struct Landing {
    Stream* st;
    size_t off, nbits;
  };
  std::vector<Landing> inflight;    // bit copies queued and not yet committed
  int64_t batch_calls = 0;
  double last_drain_ms = 0.0;
  double round_ms = 0.0, push_ms = 0.0, poll_ms = 0.0;  // worker time in passes, push calls, polls (under mu)
  long long polled_calls = -1;      // batch calls complete at the last poll of every stream
  double last_poll_ms = 0.0;
  bool poll_due = true;             // a push outside the batch since the last poll
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
      const double tp = now_ms();
      const int prc = b->end ? rx_push_block(st->h, nullptr, 0, RX_C64, 1, st->cs)
                             : rx_push_block(st->h, b->p, b->n, b->dtype, b->on_device, st->cs);
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->push_ms += now_ms() - tp;
      }
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

// Batched mode: the decided bits of the batch's streams reach their host
// buffers in two steps that never stall a round: drain_begin queues one
// copy per stream into the page-locked landing area and records an event;
// a later round's drain_finish, once the event has passed (or waiting for
// it when asked), marks the bits pulled and appends them to the buffers.
// Worker only, the streams' handle locks held.
int drain_finish(rx_server* s, bool wait) {
  if (s->inflight.empty()) return RX_OK;
  const cudaError_t e = wait ? cudaEventSynchronize(s->drain_ev) : cudaEventQuery(s->drain_ev);
  if (e == cudaErrorNotReady) return RX_OK;
  if (e != cudaSuccess) return err(RX_EDEVICE, "bit copy failed");
  std::lock_guard<std::mutex> lk(s->mu);
  for (const auto& l : s->inflight) {
    rx::pull_bits_commit(l.st->h, l.nbits);
    const uint8_t* p = s->pinned + l.off;
    l.st->bits.insert(l.st->bits.end(), p, p + (l.nbits + 7) / 8);
    if (l.nbits % 8) l.st->bits_tail = l.nbits % 8;
  }
  s->inflight.clear();
  s->poll_due = true;  // the streams' drained state changed
  return RX_OK;
}

int drain_begin(rx_server* s, const std::vector<Stream*>& m) {
  size_t used = 0;
  for (Stream* st : m) {
    size_t room;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      room = (size_t)s->cfg.bits_cap_bytes > st->bits.size() ? (size_t)s->cfg.bits_cap_bytes - st->bits.size() : 0;
    }
    room = std::min(room, s->pinned_bytes - used);
    if (room == 0) continue;
    size_t nb = 0;
    const int rc = rx::pull_bits_begin(st->h, s->pinned + used, room, &nb, s->dcs);
    if (rc != RX_OK) return rc;
    if (nb == 0) continue;
    s->inflight.push_back({st, used, nb});
    used += (nb + 7) / 8;
  }
  if (!s->inflight.empty() && cudaEventRecord(s->drain_ev, s->dcs) != cudaSuccess)
    return err(RX_EDEVICE, "cudaEventRecord failed");
  return RX_OK;
}

// Batched mode: a stream's receiver stays alive while the current or a
// replaced batch refers to it (under mu).
void mark_members(rx_server* s) {
  for (auto& kv : s->streams) kv.second->in_batch = false;
  for (Stream* st : s->members) st->in_batch = true;
  for (auto& r : s->retired)
    for (Stream* st : r.second) st->in_batch = true;
}

// Batched mode: frees the replaced batches whose work is complete (never
// waits).
void free_retired(rx_server* s) {
  if (s->retired.empty()) return;
  bool freed = false;
  for (size_t i = 0; i < s->retired.size();) {
    bool done;
    {
      std::vector<std::unique_lock<std::mutex>> locks;
      for (Stream* st : s->retired[i].second) locks.emplace_back(st->hm);
      done = rx::batch_try_free(s->retired[i].first);
    }
    if (done) {
      s->retired.erase(s->retired.begin() + i);
      freed = true;
    } else {
      ++i;
    }
  }
  if (freed) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      mark_members(s);
    }
    s->done_cv.notify_all();
  }
}

// Batched mode: when the set of open streams changed (a stream opened, or
// one is closing), the batch is replaced by one over the open streams.
// The old batch is not waited for: it is freed once its work has run
// (free_retired), so admission never stalls the other streams; work
// stays ordered per stream across the two batches.
int refresh_batch(rx_server* s) {
  free_retired(s);
  std::vector<Stream*> want;
  bool leaving_in_flight = false;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& kv : s->streams)
      if (!kv.second->closing) want.push_back(kv.second);
    for (const auto& l : s->inflight) leaving_in_flight |= l.st->closing;
  }
  if (want == s->members && (s->batch || want.empty())) return RX_OK;
  if (leaving_in_flight) {  // bit copies of a leaving stream complete first
    std::vector<std::unique_lock<std::mutex>> locks;
    for (Stream* st : s->members) locks.emplace_back(st->hm);
    const int rc = drain_finish(s, true);
    if (rc != RX_OK) return rc;
  }
  rx_batch* nb = nullptr;
  if (!want.empty()) {
    std::vector<rx_handle*> hs;
    for (Stream* st : want) hs.push_back(st->h);
    int rc = rx_batch_create(hs.data(), (int)hs.size(), &nb);
    if (rc != RX_OK) return rc;
    if (s->cfg.batch == 2) rc = rx_batch_set_graph(nb, 1);
    if (rc != RX_OK) {
      rx_batch_destroy(nb);
      return rc;
    }
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->batch) s->retired.push_back({s->batch, s->members});
    s->batch = nb;
    s->members = want;
    s->polled_calls = -1;
    mark_members(s);
  }
  s->done_cv.notify_all();
  free_retired(s);
  return RX_OK;
}

// Marks the frames a push launched for the latency statistics and counts
// the block (worker, handle lock held).
void account_push(rx_server* s, Stream* st, const Block& b, long long fl0) {
  const long long fl1 = rx::handle_launched(st->h);
  if (fl1 > fl0) st->waits.push_back(Wait{fl1 - 1, b.t_submit});
  std::lock_guard<std::mutex> lk(s->mu);
  // the push may have queued work: the stream counts as busy on the device
  // until the next poll says otherwise
  st->pending = std::max<long long>(st->pending, 1);
  if (b.end) {
    st->flushed = true;
  } else {
    st->pushed++;
    s->pushed++;
    s->samples += (int64_t)b.n;
  }
  st->q.pop_front();
}

// One round of the batched worker; true if anything was pushed.
bool batch_round(rx_server* s, std::vector<uint8_t>& scratch) {
  int rc = refresh_batch(s);
  if (rc != RX_OK) {
    set_worker_error(s, rc);
    return false;
  }
  if (!s->batch) return false;
  std::vector<Stream*> m = s->members;
  const int n = (int)m.size();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (Stream* st : m) st->busy = true;
  }
  bool progressed = false;
  {
    std::vector<std::unique_lock<std::mutex>> locks;
    for (Stream* st : m) locks.emplace_back(st->hm);
    rc = drain_finish(s, false);
    // the round: every stream's first queued block
    std::vector<Block*> fr(n, nullptr);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (int c = 0; c < n; ++c)
        if (!m[c]->q.empty()) fr[c] = &m[c]->q.front();
    }
    // the batched call takes the device blocks of the first one's input type, and ends
    int gd = -1, go = -1;
    for (int c = 0; c < n; ++c)
      if (fr[c] && !fr[c]->end && fr[c]->on_device) {
        gd = fr[c]->dtype;
        go = fr[c]->on_device;
        break;
      }
    static const unsigned char kNothing = 0;  // a non-null pointer for "no block"
    std::vector<const void*> ptrs(n, &kNothing);
    std::vector<size_t> ns(n, 0);
    std::vector<char> inb(n, 0);
    std::vector<long long> fl0(n, 0);
    bool any = false;
    for (int c = 0; c < n; ++c) {
      Block* b = fr[c];
      if (!b) continue;
      if (b->end) {
        ptrs[c] = nullptr;
      } else if (b->on_device && b->dtype == gd && b->on_device == go) {
        ptrs[c] = b->p;
        ns[c] = b->n;
      } else {
        continue;
      }
      inb[c] = 1;
      any = true;
      fl0[c] = rx::handle_launched(m[c]->h);
    }
    bool batched = false, refused = false;
    if (rc == RX_OK && any) {
      const double tp = now_ms();
      const int prc = rx_batch_push(s->batch, ptrs.data(), ns.data(), gd < 0 ? RX_C64 : gd, go < 0 ? 1 : go, s->bcs);
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->push_ms += now_ms() - tp;
      }
      if (prc == RX_OK) {
        batched = true;
        std::lock_guard<std::mutex> lk(s->mu);
        s->batch_calls++;
      } else if (prc != RX_EAGAIN) {
        rc = prc;  // RX_EAGAIN: a stream's output ring is full; its blocks go one by one below
      } else {
        refused = true;
      }
    }
    for (int c = 0; c < n && rc == RX_OK; ++c) {
      Block* b = fr[c];
      if (!b) continue;
      Stream* st = m[c];
      if (inb[c] && batched) {
        account_push(s, st, *b, fl0[c]);
        progressed = true;
        continue;
      }
      const long long f0 = rx::handle_launched(st->h);
      const int prc = b->end ? rx_push_block(st->h, nullptr, 0, RX_C64, 1, st->cs)
                             : rx_push_block(st->h, b->p, b->n, b->dtype, b->on_device, st->cs);
      if (prc == RX_EAGAIN) {  // drained below, pushed in a later round
        refused = true;
        continue;
      }
      (void)scratch;
      if (prc != RX_OK) {
        rc = prc;
        break;
      }
      account_push(s, st, *b, f0);
      s->poll_due = true;
      progressed = true;
    }
    // the streams are polled (frames done, latency samples, bits ready)
    // when a batch call completed, after a push outside the batch, or
    // 1 ms after the last poll: one event query per round otherwise
    const long long cd = rx::batch_calls_done(s->batch);
    const double t_now = now_ms();
    struct PollTime {
      rx_server* s;
      double t0;
      ~PollTime() {
        std::lock_guard<std::mutex> lk(s->mu);
        s->poll_ms += now_ms() - t0;
      }
    } poll_time{s, t_now};
    if (rc == RX_OK && (cd != s->polled_calls || s->poll_due || refused || !s->inflight.empty() ||
                        t_now - s->last_poll_ms > 1.0)) {
      s->polled_calls = cd;
      s->poll_due = false;
      s->last_poll_ms = t_now;
      // bits go to the host buffers when a ring is refused or a quarter
      // full, a stream is idle, or 2 ms after the last drain
      bool drain = refused || t_now - s->last_drain_ms > 2.0;
      std::vector<char> ready_bits(n, 0);
      for (int c = 0; c < n && rc == RX_OK; ++c) {
        poll_frames(s, m[c]);
        long long ready = 0, ring = 1;
        rx::handle_bits(m[c]->h, &ready, &ring);
        ready_bits[c] = ready > 0;
        if (ready > 0 && (4 * ready > ring || m[c]->pending == 0)) drain = true;
      }
      if (rc == RX_OK && drain && s->inflight.empty()) {
        rc = drain_begin(s, m);
        s->last_drain_ms = t_now;
      }
      // a stream is drained once no bits of it wait on the device (or its
      // host buffer is full: its bits wait there until the client pulls)
      std::vector<char> fly(n, 0);
      for (const auto& l : s->inflight)
        for (int c = 0; c < n; ++c) fly[c] |= l.st == m[c];
      std::lock_guard<std::mutex> lk(s->mu);
      for (int c = 0; c < n; ++c) {
        const bool room = (size_t)s->cfg.bits_cap_bytes > m[c]->bits.size();
        m[c]->undrained = fly[c] || (ready_bits[c] && room);
      }
    }
  }
  if (rc != RX_OK) set_worker_error(s, rc);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (Stream* st : m) st->busy = false;
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
        if (kv.first % nw == k && (!kv.second->q.empty() || kv.second->pending > 0 || kv.second->undrained ||
                                   (kv.second->closing && kv.second->in_batch)))
          work = true;
      if (s->cfg.batch && !s->retired.empty()) work = true;
      if (!work) s->cv.wait_for(lk, std::chrono::microseconds(200));
      if (s->stop) return;
    }
    const double t0 = now_ms();
    const bool pushed = s->cfg.batch ? batch_round(s, scratch) : worker_pass(s, k, scratch);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->round_ms += now_ms() - t0;
    }
    if (!pushed) std::this_thread::sleep_for(std::chrono::microseconds(20));
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
  c->batch = 0;
}

int rx_server_create(const rx_server_config* cfg, rx_server** out) {
  if (!cfg || !out) return err(RX_EINVAL, "null argument");
  *out = nullptr;
  if (cfg->max_streams < 1 || cfg->max_streams > 1024) return err(RX_EINVAL, "max_streams must be in 1..1024");
  if (cfg->bits_cap_bytes < 4096) return err(RX_EINVAL, "bits_cap_bytes must be >= 4096");
  if (cfg->workers < 1 || cfg->workers > 64) return err(RX_EINVAL, "workers must be in 1..64");
  if (cfg->batch < 0 || cfg->batch > 2) return err(RX_EINVAL, "batch must be 0, 1 or 2");
  if (cfg->batch && cfg->max_streams > RX_BATCH_MAX) return err(RX_EINVAL, "batched rounds take at most RX_BATCH_MAX streams");
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
  if (s->cfg.batch) {
    s->cfg.workers = 1;  // one worker forms the rounds
    s->pinned_bytes = (size_t)std::min<int64_t>(s->cfg.bits_cap_bytes, 64LL << 20);
    if (cudaStreamCreateWithFlags(&s->bcs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->dcs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->drain_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&s->pinned, s->pinned_bytes) != cudaSuccess) {
      if (s->bcs) cudaStreamDestroy(s->bcs);
      if (s->dcs) cudaStreamDestroy(s->dcs);
      delete s;
      return err(RX_EDEVICE, "batched server: stream or page-locked buffer creation failed");
    }
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
    if (st->q.empty() && st->pending == 0 && !st->busy && !st->undrained) break;
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
    st->closing = true;  // the worker takes it no more (batched mode: and drops it from the batch)
    s->cv.notify_all();
    while (st->busy || st->in_batch) s->done_cv.wait_for(lk, std::chrono::microseconds(200));
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
  out->batch_calls = s->batch_calls;
  out->worker_round_ms = s->round_ms;
  out->worker_push_ms = s->push_ms;
  out->worker_poll_ms = s->poll_ms;
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
  for (auto& r : s->retired) rx_batch_destroy(r.first);  // before the receivers they refer to
  if (s->batch) rx_batch_destroy(s->batch);
  if (s->bcs) cudaStreamDestroy(s->bcs);
  if (s->dcs) {
    cudaStreamSynchronize(s->dcs);
    cudaStreamDestroy(s->dcs);
  }
  if (s->drain_ev) cudaEventDestroy(s->drain_ev);
  if (s->pinned) cudaFreeHost(s->pinned);
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
