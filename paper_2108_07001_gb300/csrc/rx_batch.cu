// Batched pushes of many dual-polarisation streams (rx_batch_* in
// include/rx.h), on top of the plain path's frame planning.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "rx_handle.h"

using namespace rx;
using namespace rxrt;

namespace rx {
thread_local GraphRecorder* t_graph_rec = nullptr;
}

// ---- batched pushes of many streams (rx_batch_*) ---------------------------
//
// One call ingests every stream's block with one launch on the caller's
// stream, then runs the frames the blocks complete by ordinal: the i-th
// frame of every stream that completes at least i + 1 frames goes through
// each stage in one launch (streams with another FFT size, tap count or
// BPS form in a launch of their own).  The stages are pipelined over four
// streams of the batch like the plain path's: front (CD + estimators), mid
// (acquisition + MIMO), back (BPS) and demap + BER; ordinal q's stage waits
// for the same ordinal's previous stage and for the ordinals whose buffers
// it reuses (front: the MIMO of q - kZSlots, whose CD output slot it
// overwrites; mid: the BPS of q - 2, whose equalised-symbol buffer it
// overwrites; back: the demap of q - 2, whose decision buffers it
// overwrites), and the ingest of the next call waits for this call's
// front work (ring slots).  The arguments of a call (ingest list,
// per-ordinal launch lists and frames) are written to a page-locked table
// and copied to the device once.

namespace {

enum BStageId { BS_CD0, BS_EST0, BS_CD, BS_EST1, BS_ACQ, BS_MIMO, BS_BPS, BS_SCAN, BS_DEMAP, BS_REF0, BS_SYNC, BS_REF1,
                BS_BER, BS_N };

// Work of one stream at one ordinal.
struct BPlan {
  FrameArgs fa;
  RxDev d;
  bool frame;   // a whole frame (else the decide-only pass at the end)
  bool final_;
  BerPlan ber;
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct rx_batch {
  std::vector<rx_handle*> h;
  int nh = 0;
  int device = 0;
  // launch groups: streams whose kernels share template parameters
  std::vector<int> grp[BS_N];         // group of each stream per stage
  std::vector<int> rep[BS_N];         // a stream of each group per stage
  int slot0[BS_N + 1] = {};           // first launch-list slot of each stage
  int nslots = 0;
  int max_ord = 0;
  size_t list_ints = 0;               // ints per launch list: 1 + 2 nh + (nh + 1)
  size_t ing_bytes = 0, ord_bytes = 0, lists_bytes = 0, blob_bytes = 0;
  static constexpr int kSlots = 4;    // tables in flight
  static constexpr int kQ = 8;        // ordinal events kept per pipeline stage
  void* host[kSlots] = {};
  void* dev[kSlots] = {};
  cudaEvent_t ev_slot[kSlots] = {};   // last call that used table slot s is done
  cudaStream_t s_stage[4] = {};       // front, mid, back, BER
  cudaEvent_t ev_stage[4][kQ] = {};   // stage done, by ordinal sequence number mod kQ
  cudaEvent_t ev_ing = nullptr;       // the call's table copy and ingest done (caller's stream)
  cudaEvent_t ev_front_last = nullptr;  // front work of the last ordinal so far
  long long q = 0;                    // ordinals launched so far
  std::vector<cudaEvent_t> ev_ring;   // call start / end events (round robin)
  size_t ev_i = 0;
  long long calls = 0, launches = 0, frames = 0;
  long long calls_done = 0;          // calls seen complete (batch_calls_done)
  double wait_s = 0.0;                // host time spent waiting for table slots
  // graph replay (rx_batch_set_graph): one graph of every stage launch of
  // max_ord ordinals, a kernel node per (ordinal, launch list)
  struct GNode {
    cudaGraphNode_t node = nullptr;
    cudaKernelNodeParams p = {};      // as captured (argument values held by the graph)
    int o = 0, list = 0;              // ordinal and launch-list slot
    int grid = 0;                     // grid now set in the executable graph
    bool on = true;                   // enabled in the executable graph
  };
  bool graph = false;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t gx = nullptr;
  std::vector<GNode> gnodes;
  void* gdev = nullptr;               // the graph's device table (table layout, ordinal part used)
  long long replays = 0;
};

namespace {

// Launch list slot l of ordinal o in a table.
int* blob_list(const rx_batch* b, char* base, int o, int l) {
  return reinterpret_cast<int*>(base + b->ing_bytes + (size_t)o * b->ord_bytes + (size_t)l * b->list_ints * 4);
}
BFrame* blob_frames(const rx_batch* b, char* base, int o) {
  return reinterpret_cast<BFrame*>(base + b->ing_bytes + (size_t)o * b->ord_bytes + b->lists_bytes);
}

// Appends an entry (frame fi, grid nx wide, nblk blocks) to a launch list.
void list_add(const rx_batch* b, int* L, int fi, int nx, int nblk) {
  const int n = L[0];
  int* idx = L + 1;
  int* nxa = idx + b->nh;
  int* offs = nxa + b->nh;
  if (n == 0) offs[0] = 0;
  idx[n] = fi;
  nxa[n] = nx;
  offs[n + 1] = offs[n] + nblk;
  L[0] = n + 1;
}
int list_blocks(const rx_batch* b, const int* L) { return L[0] ? L[1 + 2 * b->nh + L[0]] : 0; }

// Frames (and whether the decide-only pass follows) a push of n samples,
// or the end of stream (n < 0), makes stream h launch.
int count_work(const rx_handle* h, long long n) {
  const long long F = h->d.F;
  if (n >= 0) {
    const long long pushed = h->pushed + n;
    long long f = h->f_next;
    while (pushed >= 2 * (f + 1) * F + h->la) ++f;
    return (int)(f - h->f_next);
  }
  const long long n_sym = h->pushed / 2;
  int k = 0;
  bool fin = false;
  for (long long f = h->f_next; f * F < n_sym; ++f) {
    ++k;
    if ((f + 1) * F >= n_sym) fin = true;
  }
  if (!fin && !h->tail_launched) ++k;  // at most one decide-only pass
  return k;
}

// Plans frame f of h (host state advanced as launch_frame does).
BPlan plan_frame(rx_handle* h, long long f, bool final_) {
  BPlan p;
  p.fa = frame_args(h, f, final_);
  p.d = decide_dev(slot_dev(h, f), h->n_decide);
  p.frame = true;
  p.final_ = final_;
  h->n_decide++;
  if (h->d.ber_on) p.ber = plan_ber(h, p.fa, final_);
  h->decided = p.fa.k_b;
  h->f_next = f + 1;
  return p;
}

// Adds plan p of stream c as frame fi of ordinal o.
void add_plan(rx_batch* b, char* base, int o, int fi, int c, const BPlan& p) {
  const rx_handle* h = b->h[c];
  BFrame& fr = blob_frames(b, base, o)[fi];
  std::memset(&fr, 0, sizeof(fr));
  fr.d = p.d;
  fr.fa = p.fa;
  fr.fe = est_pass_args(p.fa);
  fr.hist_base = p.fa.f * (long long)h->d.F;
  fr.sync_sym0 = p.ber.sync_sym0;
  fr.sync_nbits = p.ber.sync_nbits;
  fr.ref_sym0 = p.ber.ref_sym0;
  fr.ref_nbits = p.ber.ref_nbits;
  fr.ka = p.ber.ka;
  fr.kb = p.ber.kb;
  fr.w_from = p.ber.w_from;
  fr.w_to = p.ber.w_to;
  fr.k_lim = p.ber.k_lim;
  fr.n_win_ring = h->n_win_ring;
  const RxDev& d = p.d;
  const FrameArgs& fa = p.fa;
  auto L = [&](int st) { return blob_list(b, base, o, b->slot0[st] + b->grp[st][c]); };
  if (p.frame) {
    const int ncd = cd_grid_x(d, fa);
    if (fa.f == 0) {
      const FrameArgs fe = est_pass_args(fa);
      list_add(b, L(BS_CD0), fi, cd_grid_x(d, fe), 2 * cd_grid_x(d, fe));
      list_add(b, L(BS_EST0), fi, est_grid_x(d), est_grid_x(d));
    }
    list_add(b, L(BS_CD), fi, ncd, 2 * ncd);
    list_add(b, L(BS_EST1), fi, est_grid_x(d), est_grid_x(d));
    if (fa.f == 0) list_add(b, L(BS_ACQ), fi, 1, 1);
    list_add(b, L(BS_MIMO), fi, mimo_grid_x(d, fa), mimo_grid_x(d, fa));
  }
  if (fa.k_b > fa.k_a) {
    list_add(b, L(BS_BPS), fi, bps_grid_x(d, fa), 2 * bps_grid_x(d, fa));
    list_add(b, L(BS_SCAN), fi, 2, 2);  // one block per polarisation
    list_add(b, L(BS_DEMAP), fi, demap_grid_x(fa), demap_grid_x(fa));
  }
  if (p.ber.sync) {
    list_add(b, L(BS_REF0), fi, ref_grid_x(p.ber.sync_nbits), 2 * ref_grid_x(p.ber.sync_nbits));
    list_add(b, L(BS_SYNC), fi, sync_grid_x(d), sync_grid_x(d));
  }
  if (p.ber.ref) list_add(b, L(BS_REF1), fi, ref_grid_x(p.ber.ref_nbits), 2 * ref_grid_x(p.ber.ref_nbits));
  if (p.ber.count && !(p.ber.kb <= p.ber.ka && p.ber.w_to <= p.ber.w_from))
    list_add(b, L(BS_BER), fi, ber_grid_x(d, p.ber.ka, p.ber.kb), ber_grid_x(d, p.ber.ka, p.ber.kb));
}

// Orders stream h's earlier work (its own streams, the pushes on another
// stream, a reset) before work queued next on cs; the batch's own earlier
// calls (last_cs = its end stream) are ordered by the batch itself.
int join_stream(rx_handle* h, cudaStream_t cs, cudaStream_t batch_end) {
  if (h->copy_dirty && h->last_cs != cs && h->last_cs != batch_end) {
    RX_CK(mark_copy(h));
    RX_CK(cudaStreamWaitEvent(cs, h->ev_copy, 0));
  }
  if (h->own_work) {
    cudaStream_t ss[6] = {h->s_front, h->s_mid, h->s_comp, h->s_comp2, h->s_dem, h->s_ber};
    cudaEvent_t e = get_event(h);
    for (cudaStream_t x : ss) {
      RX_CK(cudaEventRecord(e, x));
      RX_CK(cudaStreamWaitEvent(cs, e, 0));
    }
    h->ev_pool.push_back(e);
    h->own_work = false;
  }
  if (h->reset_pending) {
    RX_CK(cudaStreamWaitEvent(cs, h->ev_reset, 0));
    h->reset_pending = false;
  }
  return RX_OK;
}

// Pipeline stage of each launch.
int stage_of(int st) {
  // demap with the BER work: the next ordinal's BPS overlaps it (the two
  // use the decision buffers of different decide passes)
  return st <= BS_EST1 ? 0 : (st <= BS_MIMO ? 1 : (st <= BS_BPS ? 2 : 3));
}

// The launches of one ordinal's lists that belong to pipeline stage ps.
// capture (a graph recorder set on this thread): every list gets a kernel
// node (the smallest grid: the lists are empty until a call fills them),
// kept for graph replay.
int launch_ordinal(rx_batch* b, char* dbase, char* hbase, int o, int ps, cudaStream_t cs, bool capture = false) {
  BView v;
  v.frames = blob_frames(b, dbase, o);
  v.nmax = b->nh;
  for (int st = 0; st < BS_N; ++st) {
    if (stage_of(st) != ps) continue;
    for (int g = 0; g < b->slot0[st + 1] - b->slot0[st]; ++g) {
      const RxDev& d = b->h[b->rep[st][g]]->d;
      int blocks;
      if (capture) {
        blocks = (st == BS_CD0 || st == BS_CD) && d.N == 32768 ? 2 : 1;  // 32768: clusters of two CTAs
      } else {
        blocks = list_blocks(b, blob_list(b, hbase, o, b->slot0[st] + g));
        if (blocks <= 0) continue;
      }
      v.list = blob_list(b, dbase, o, b->slot0[st] + g);
      cudaError_t e = cudaSuccess;
      switch (st) {
        case BS_CD0: e = launch_cd_batch(d, v, blocks, 0, cs); break;
        case BS_EST0: e = launch_est_batch(v, blocks, 0, cs); break;
        case BS_CD: e = launch_cd_batch(d, v, blocks, 1, cs); break;
        case BS_EST1: e = launch_est_batch(v, blocks, 1, cs); break;
        case BS_ACQ: e = launch_acquire_batch(d, v, blocks, cs); break;
        case BS_MIMO: e = launch_mimo_batch(d, v, blocks, cs); break;
        case BS_BPS: e = launch_bps_batch(d, v, blocks, cs); break;
        case BS_SCAN: e = launch_scan_batch(v, blocks, cs); break;
        case BS_DEMAP: e = launch_demap_batch(v, blocks, cs); break;
        case BS_REF0: e = launch_ref_gen_batch(v, blocks, 0, cs); break;
        case BS_SYNC: e = launch_sync_batch(v, blocks, cs); break;
        case BS_REF1: e = launch_ref_gen_batch(v, blocks, 1, cs); break;
        case BS_BER: e = launch_ber_batch(v, blocks, cs); break;
      }
      if (e != cudaSuccess) return cuda_fail(e, "rx_batch_push: launch");
      if (!capture) {
        b->launches++;
        continue;
      }
      rx_batch::GNode n;
      n.node = t_graph_rec->last;  // the node launch_k just added
      n.o = o;
      n.list = b->slot0[st] + g;
      n.grid = blocks;
      b->gnodes.push_back(n);
    }
  }
  return RX_OK;
}

void graph_free(rx_batch* b) {
  if (b->gx) cudaGraphExecDestroy(b->gx);
  if (b->g) cudaGraphDestroy(b->g);
  b->gx = nullptr;
  b->g = nullptr;
  b->gnodes.clear();
}

// Builds the graph of every stage launch of max_ord ordinals, node by node
// (no stream capture).  Each pipeline stage is a chain of nodes in launch
// order, and the first node of stage ps at ordinal o also depends on the
// stream mode's in-call waits: front on the MIMO kZSlots ordinals back,
// every later stage on the ordinal's previous stage, mid and back on the
// next stage two ordinals back.  The waits across calls are not needed:
// replays run one after another on one stream.
int graph_build(rx_batch* b) {
  b->gnodes.clear();
  cudaGraph_t g = nullptr;
  RX_CK(cudaGraphCreate(&g, 0));
  const int M = b->max_ord;
  std::vector<cudaGraphNode_t> done(4 * (size_t)M, nullptr);  // last node of stage ps at ordinal o
  cudaGraphNode_t tail[4] = {};
  GraphRecorder rec;
  rec.g = g;
  char* gd = static_cast<char*>(b->gdev);
  int rc = RX_OK;
  t_graph_rec = &rec;
  for (int o = 0; o < M && rc == RX_OK; ++o)
    for (int ps = 0; ps < 4 && rc == RX_OK; ++ps) {
      rec.ndeps = 0;
      auto dep = [&](cudaGraphNode_t n) {
        if (n) rec.deps[rec.ndeps++] = n;
      };
      dep(tail[ps]);
      if (ps == 0) {
        if (o >= kZSlots) dep(done[1 * (size_t)M + o - kZSlots]);
      } else {
        dep(done[(ps - 1) * (size_t)M + o]);
        if (ps < 3 && o >= 2) dep(done[(ps + 1) * (size_t)M + o - 2]);
      }
      rec.last = nullptr;
      rc = launch_ordinal(b, gd, nullptr, o, ps, nullptr, true);
      if (rc == RX_OK && !rec.last) {  // a stage without launches keeps its place in the chain
        const cudaError_t e = cudaGraphAddEmptyNode(&rec.last, g, rec.deps, (size_t)rec.ndeps);
        if (e != cudaSuccess) rc = cuda_fail(e, "rx_batch_set_graph: empty node");
      }
      tail[ps] = done[ps * (size_t)M + o] = rec.last;
    }
  t_graph_rec = nullptr;
  b->g = g;
  if (rc == RX_OK) {
    const cudaError_t e = cudaGraphInstantiate(&b->gx, g, 0);
    if (e != cudaSuccess) rc = cuda_fail(e, "rx_batch_set_graph: instantiate");
  }
  for (size_t i = 0; i < b->gnodes.size() && rc == RX_OK; ++i) {
    const cudaError_t e = cudaGraphKernelNodeGetParams(b->gnodes[i].node, &b->gnodes[i].p);
    if (e != cudaSuccess) rc = cuda_fail(e, "rx_batch_set_graph: node parameters");
  }
  if (rc != RX_OK) {
    cudaGetLastError();
    graph_free(b);
  }
  return rc;
}

// Per call: grids of the nodes whose block count changed, and the nodes
// without work (no frame in the list, ordinal beyond the call's) disabled.
int graph_update(rx_batch* b, char* hb, int n_ord) {
  for (rx_batch::GNode& n : b->gnodes) {
    const int blocks = n.o < n_ord ? list_blocks(b, blob_list(b, hb, n.o, n.list)) : 0;
    const bool on = blocks > 0;
    if (on && blocks != n.grid) {
      cudaKernelNodeParams p = n.p;
      p.gridDim = dim3((unsigned)blocks, 1, 1);
      RX_CK(cudaGraphExecKernelNodeSetParams(b->gx, n.node, &p));
      n.grid = blocks;
    }
    if (on != n.on) {
      RX_CK(cudaGraphNodeSetEnabled(b->gx, n.node, on ? 1u : 0u));
      n.on = on;
    }
    if (on) b->launches++;
  }
  return RX_OK;
}

void batch_free(rx_batch* b) {
  for (int i = 0; i < rx_batch::kSlots; ++i) {
    if (b->host[i]) cudaFreeHost(b->host[i]);
    if (b->dev[i]) cudaFree(b->dev[i]);
    if (b->ev_slot[i]) cudaEventDestroy(b->ev_slot[i]);
  }
  for (int p = 0; p < 4; ++p) {
    for (int i = 0; i < rx_batch::kQ; ++i)
      if (b->ev_stage[p][i]) cudaEventDestroy(b->ev_stage[p][i]);
    if (b->s_stage[p]) cudaStreamDestroy(b->s_stage[p]);
  }
  if (b->ev_ing) cudaEventDestroy(b->ev_ing);
  for (cudaEvent_t e : b->ev_ring) cudaEventDestroy(e);
  graph_free(b);
  if (b->gdev) cudaFree(b->gdev);
}

}  // namespace

namespace rx {
// Calls of the batch whose device work is complete (polled, nothing waits):
// at most kSlots calls are in flight, so the slot events of the calls not
// yet seen complete are all distinct.
long long batch_calls_done(rx_batch* b) {
  while (b->calls_done < b->calls &&
         cudaEventQuery(b->ev_slot[b->calls_done % rx_batch::kSlots]) == cudaSuccess)
    ++b->calls_done;
  cudaGetLastError();
  return b->calls_done;
}

// Frees the batch without waiting when its device work is complete: true
// when freed, false while some of it still runs (try again later).  The
// handles may meanwhile carry work of another batch or of plain pushes;
// the caller holds no other call on them.
bool batch_try_free(rx_batch* b) {
  cudaSetDevice(b->device);
  if (batch_calls_done(b) < b->calls) return false;
  for (int p = 0; p < 4; ++p)
    if (cudaStreamQuery(b->s_stage[p]) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
  for (rx_handle* h : b->h) {
    harvest(h);  // the batch's entries are complete, so they leave the queue
    for (const PendingFrame& pf : h->pend)
      for (cudaEvent_t e : b->ev_ring)
        if (pf.ev_done == e || pf.ev_in == e) return false;
  }
  for (rx_handle* h : b->h) {
    bool mine = false;
    for (cudaEvent_t e : b->ev_ring) mine |= h->batch_done == e;
    if (mine) h->batch_done = nullptr;
    if (h->last_cs == b->s_stage[3]) {  // its work is complete: nothing to join
      h->last_cs = nullptr;
      h->copy_dirty = false;
    }
  }
  batch_free(b);
  delete b;
  return true;
}
}  // namespace rx

extern "C" {

int rx_batch_create(rx_handle* const* streams, int n_streams, rx_batch** out) {
  if (!streams || !out || n_streams < 1 || n_streams > RX_BATCH_MAX) return fail(RX_EINVAL, "need 1..RX_BATCH_MAX streams and out");
  *out = nullptr;
  for (int c = 0; c < n_streams; ++c) {
    if (!streams[c]) return fail(RX_EINVAL, "null stream handle");
    for (int k = 0; k < c; ++k)
      if (streams[k] == streams[c]) return fail(RX_EINVAL, "a stream appears twice in the batch");
    if (streams[c]->cfg.device != streams[0]->cfg.device) return fail(RX_EINVAL, "streams on different devices");
  }
  rx_batch* b = new rx_batch();
  b->h.assign(streams, streams + n_streams);
  b->nh = n_streams;
  b->device = streams[0]->cfg.device;
  // launch groups by the kernels' template parameters
  auto key = [](const RxDev& d, int st) -> long long {
    switch (st) {
      case BS_CD0: case BS_CD: return (long long)d.N * 4 + d.storage;
      case BS_ACQ: return d.T;
      case BS_MIMO: return (long long)d.T * 16 + d.mimo_nw;  // the launch's block size is the group's
      case BS_BPS: return ((((long long)d.B * 64 + d.W) * 8 + d.bps) * 64 + d.bps_stride) * 16 + d.bps_nw;
      default: return 0;
    }
  };
  int slot = 0;
  for (int st = 0; st < BS_N; ++st) {
    std::vector<long long> keys;
    b->slot0[st] = slot;
    for (int c = 0; c < n_streams; ++c) {
      const long long k = key(b->h[c]->d, st);
      int g = (int)(std::find(keys.begin(), keys.end(), k) - keys.begin());
      if (g == (int)keys.size()) {
        keys.push_back(k);
        b->rep[st].push_back(c);
      }
      b->grp[st].push_back(g);
    }
    slot += (int)keys.size();
  }
  b->slot0[BS_N] = slot;
  b->nslots = slot;
  // ordinals per call: frames a block of max_block_samples completes, or
  // the frames and decide-only pass of an end of stream
  for (rx_handle* h : b->h) {
    const long long F2 = 2LL * h->d.F;
    const long long blk = (long long)h->cfg.max_block_samples;
    const int o1 = (int)((blk + F2 - 1) / F2) + 2;
    const int o2 = (int)((F2 + h->la + F2 - 1) / F2) + 3;
    b->max_ord = std::max(b->max_ord, std::max(o1, o2));
  }
  b->list_ints = 2 + 3 * (size_t)n_streams;
  b->ing_bytes = align_up(sizeof(BIngest) * n_streams + b->list_ints * 4, 256);
  b->lists_bytes = align_up((size_t)b->nslots * b->list_ints * 4, 256);
  b->ord_bytes = b->lists_bytes + align_up(sizeof(BFrame) * n_streams, 256);
  b->blob_bytes = b->ing_bytes + (size_t)b->max_ord * b->ord_bytes;
  cudaError_t e = cudaSetDevice(b->device);
  for (int i = 0; i < rx_batch::kSlots && e == cudaSuccess; ++i) {
    e = cudaMallocHost(&b->host[i], b->blob_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->dev[i], b->blob_bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_slot[i], cudaEventDisableTiming);
  }
  for (int p = 0; p < 4 && e == cudaSuccess; ++p) {
    e = cudaStreamCreateWithFlags(&b->s_stage[p], cudaStreamNonBlocking);
    for (int i = 0; i < rx_batch::kQ && e == cudaSuccess; ++i)
      e = cudaEventCreateWithFlags(&b->ev_stage[p][i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_ing, cudaEventDisableTiming);
  for (int i = 0; i < 512 && e == cudaSuccess; ++i) {
    cudaEvent_t ev = nullptr;
    e = cudaEventCreate(&ev);
    if (e == cudaSuccess) b->ev_ring.push_back(ev);
  }
  if (e != cudaSuccess) {
    batch_free(b);
    delete b;
    return cuda_fail(e, "rx_batch_create");
  }
  *out = b;
  return RX_OK;
}

int rx_batch_push(rx_batch* b, const void* const* samples, const size_t* n_per_pol, int dtype, int on_device,
                  void* cuda_stream) {
  if (!b || !samples || !n_per_pol) return fail(RX_EINVAL, "null argument");
  if (dtype < RX_C128 || dtype > RX_C16) return fail(RX_EINVAL, "bad dtype");
  if (on_device < 1 || on_device > 3)
    return fail(RX_EINVAL, "batched pushes take device memory (on_device = 1) or mapped page-locked host memory (2, 3)");
  RX_CK(cudaSetDevice(b->device));
  const int nh = b->nh;
  std::vector<const void*> src(nh, nullptr);
  std::vector<int> work(nh, 0);
  // every check before any side effect: a refused call changes nothing
  for (int c = 0; c < nh; ++c) {
    rx_handle* h = b->h[c];
    const size_t n = n_per_pol[c];
    if (!samples[c] && n == 0) {
      if (h->ended) return fail(RX_ESTATE, "end of a stream that has ended");
      work[c] = count_work(h, -1);
      continue;
    }
    if (n == 0) continue;  // nothing for this stream (valid after its end too)
    if (h->ended) return fail(RX_ESTATE, "push after end of stream");
    if (!samples[c]) return fail(RX_EINVAL, "samples is NULL");
    if (n > h->cfg.max_block_samples) return fail(RX_EINVAL, "n_per_pol exceeds max_block_samples");
    src[c] = samples[c];
    if (on_device >= 2) {
      cudaPointerAttributes pa;
      if (cudaPointerGetAttributes(&pa, samples[c]) != cudaSuccess || pa.type != cudaMemoryTypeHost ||
          pa.devicePointer == nullptr) {
        cudaGetLastError();
        return fail(RX_EINVAL, "on_device = 2 or 3 needs page-locked host memory mapped for the device");
      }
      src[c] = pa.devicePointer;
    }
    work[c] = count_work(h, (long long)n);
    harvest(h);
    const long long dec = work[c] ? (h->f_next + work[c]) * h->d.F - h->d.W : h->decided;
    if (2LL * h->d.bps * dec - h->bits_pulled + 64 > 8LL * h->d.out_cap_bytes)
      return fail(RX_EAGAIN, "output ring full: pull bits first");
  }
  for (int c = 0; c < nh; ++c)
    if (work[c] > b->max_ord) return fail(RX_EINVAL, "more frames in one call than the batch was sized for");
  cudaStream_t cs = (cudaStream_t)cuda_stream;
  for (int c = 0; c < nh; ++c) {
    if (!work[c] && !src[c]) continue;
    int rc = join_stream(b->h[c], cs, b->s_stage[3]);
    if (rc != RX_OK) return rc;
  }
  // the ingest overwrites ring slots the earlier calls' CD passes read
  if (b->ev_front_last) RX_CK(cudaStreamWaitEvent(cs, b->ev_front_last, 0));
  const int sl = (int)(b->calls % rx_batch::kSlots);
  {
    const auto t0 = std::chrono::steady_clock::now();
    RX_CK(cudaEventSynchronize(b->ev_slot[sl]));  // the call kSlots back is done with both copies of the table
    b->wait_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  char* hb = static_cast<char*>(b->host[sl]);
  char* db = static_cast<char*>(b->dev[sl]);
  // ingests
  BIngest* ing = reinterpret_cast<BIngest*>(hb);
  int* ing_list = reinterpret_cast<int*>(hb + sizeof(BIngest) * nh);
  ing_list[0] = 0;
  for (int c = 0; c < nh; ++c) {
    if (!src[c]) continue;
    rx_handle* h = b->h[c];
    const long long n = (long long)n_per_pol[c];
    BIngest& g = ing[c];
    g.ring = h->d.ring;
    g.ring_cap = h->d.ring_cap;
    g.src = src[c];
    g.n = n;
    g.j0 = h->pushed % h->d.ring_cap;
    g.storage = h->d.storage;
    g.dtype = dtype;
    g.pairs = ingest_pairs_ok(h->d, src[c], dtype, n, h->pushed) ? 1 : 0;
    g.pad = 0;
    const int nx = ingest_grid_x(n, g.pairs != 0);
    list_add(b, ing_list, c, nx, nx);
    h->pushed += n;
  }
  // frames by ordinal
  int n_ord = 0;
  for (int o = 0; o < b->max_ord; ++o)
    for (int l = 0; l < b->nslots; ++l) blob_list(b, hb, o, l)[0] = 0;
  std::vector<int> nfr(b->max_ord, 0);
  std::vector<long long> nframes(nh, 0), last_f(nh, -1);
  for (int c = 0; c < nh; ++c) {
    if (!work[c] && samples[c]) continue;
    rx_handle* h = b->h[c];
    const long long F = h->d.F;
    int o = 0;
    auto put = [&](const BPlan& p) {
      add_plan(b, hb, o, nfr[o]++, c, p);
      if (p.frame) {
        nframes[c]++;
        last_f[c] = p.fa.f;
      }
      n_ord = std::max(n_ord, o + 1);
      ++o;
    };
    if (!samples[c] && n_per_pol[c] == 0) {
      h->ended = true;
      h->n_total = h->pushed;
      const long long n_sym = h->n_total / 2;
      for (long long f = h->f_next; f * F < n_sym; ++f) {
        const bool fin = (f + 1) * F >= n_sym;
        put(plan_frame(h, f, fin));
        if (fin) h->tail_launched = true;
      }
      if (!h->tail_launched && h->f_next != 0 && h->decided < n_sym) {
        BPlan p;
        p.fa = tail_args(h);
        p.d = decide_dev(h->d, h->n_decide);
        p.frame = false;
        p.final_ = true;
        h->n_decide++;
        if (h->d.ber_on) p.ber = plan_ber(h, p.fa, true);
        h->decided = n_sym;
        put(p);
      }
    } else {
      while (h->pushed >= 2 * (h->f_next + 1) * F + h->la) put(plan_frame(h, h->f_next, false));
    }
  }
  // one copy of the table's used part, then the launches
  const size_t used = b->ing_bytes + (size_t)n_ord * b->ord_bytes;
  cudaEvent_t ev_a = b->ev_ring[b->ev_i++ % b->ev_ring.size()];
  cudaEvent_t ev_b = b->ev_ring[b->ev_i++ % b->ev_ring.size()];
  RX_CK(cudaEventRecord(ev_a, cs));
  if (b->graph) {  // the ordinal part to the graph's table (the previous replay is done with it)
    RX_CK(cudaMemcpyAsync(db, hb, b->ing_bytes, cudaMemcpyHostToDevice, cs));
    if (n_ord > 0)
      RX_CK(cudaMemcpyAsync(static_cast<char*>(b->gdev) + b->ing_bytes, hb + b->ing_bytes,
                            (size_t)n_ord * b->ord_bytes, cudaMemcpyHostToDevice, cs));
  } else {
    RX_CK(cudaMemcpyAsync(db, hb, used, cudaMemcpyHostToDevice, cs));
  }
  {
    BView v;
    v.frames = nullptr;
    v.list = reinterpret_cast<const int*>(db + sizeof(BIngest) * nh);
    v.nmax = nh;
    const int blocks = list_blocks(b, ing_list);
    if (blocks > 0) {
      RX_CK(launch_ingest_batch(reinterpret_cast<const BIngest*>(db), v, blocks, cs));
      b->launches++;
    }
  }
  RX_CK(cudaEventRecord(b->ev_ing, cs));
  cudaStream_t se = b->s_stage[3];
  if (b->graph && n_ord > 0) {
    int rc = graph_update(b, hb, n_ord);
    if (rc != RX_OK) return rc;
    RX_CK(cudaStreamWaitEvent(se, b->ev_ing, 0));
    RX_CK(cudaGraphLaunch(b->gx, se));
    b->replays++;
  }
  constexpr int kQ = rx_batch::kQ;
  for (int o = 0; o < n_ord && !b->graph; ++o) {
    const long long q = b->q++;
    for (int ps = 0; ps < 4; ++ps) {
      cudaStream_t sp = b->s_stage[ps];
      if (ps == 0) {
        if (o == 0) RX_CK(cudaStreamWaitEvent(sp, b->ev_ing, 0));
        if (q >= kZSlots) RX_CK(cudaStreamWaitEvent(sp, b->ev_stage[1][(q - kZSlots) % kQ], 0));
      } else {
        RX_CK(cudaStreamWaitEvent(sp, b->ev_stage[ps - 1][q % kQ], 0));
        if (ps < 3 && q >= 2) RX_CK(cudaStreamWaitEvent(sp, b->ev_stage[ps + 1][(q - 2) % kQ], 0));
      }
      int rc = launch_ordinal(b, db, hb, o, ps, sp);
      if (rc != RX_OK) return rc;
      RX_CK(cudaEventRecord(b->ev_stage[ps][q % kQ], sp));
    }
    b->ev_front_last = b->ev_stage[0][q % kQ];
  }
  // the call's end on the BER stream (after its last ordinal, or the ingest alone)
  RX_CK(cudaStreamWaitEvent(se, b->ev_ing, 0));
  RX_CK(cudaEventRecord(ev_b, se));
  RX_CK(cudaEventRecord(b->ev_slot[sl], se));
  if (b->graph) b->ev_front_last = ev_b;  // the next call's ingest and table copy wait for the whole replay
  b->calls++;
  for (int c = 0; c < nh; ++c) {
    rx_handle* h = b->h[c];
    if (!src[c] && !work[c]) continue;
    h->last_cs = se;  // later plain pushes and frames are ordered after the call's end
    h->copy_dirty = true;
    h->f_waited = h->f_next;
    h->batch_done = ev_b;
    if (!work[c]) continue;
    PendingFrame pf;
    pf.f = last_f[c];
    pf.gen = h->gen;
    pf.ev_in = ev_a;
    pf.ev_start = ev_b;  // device time of a call is the batch's, not a stream's
    pf.ev_done = ev_b;
    pf.nframes = nframes[c];
    pf.shared = true;
    pf.dec_after = h->decided;
    pf.bits_after = 2LL * h->d.bps * h->decided;
    h->pend.push_back(pf);
    b->frames += nframes[c];
  }
  return RX_OK;
}

int rx_batch_info(const rx_batch* b, int64_t* calls, int64_t* launches, int64_t* frames, double* wait_ms) {
  if (!b) return fail(RX_EINVAL, "null batch");
  if (calls) *calls = b->calls;
  if (launches) *launches = b->launches;
  if (frames) *frames = b->frames;
  if (wait_ms) *wait_ms = 1e3 * b->wait_s;
  return RX_OK;
}

int rx_batch_set_graph(rx_batch* b, int on) {
  if (!b) return fail(RX_EINVAL, "null batch");
  if (b->calls > 0) return fail(RX_ESTATE, "rx_batch_set_graph: the batch has pushed");
  RX_CK(cudaSetDevice(b->device));
  if (!on) {
    graph_free(b);
    b->graph = false;
    return RX_OK;
  }
  if (b->graph) return RX_OK;
  cudaError_t e = cudaSuccess;
  if (!b->gdev) e = cudaMalloc(&b->gdev, b->blob_bytes);
  if (e != cudaSuccess) return cuda_fail(e, "rx_batch_set_graph");
  const int rc = graph_build(b);
  if (rc != RX_OK) return rc;
  b->graph = true;
  return RX_OK;
}

int rx_batch_graph_info(const rx_batch* b, int64_t* replays, int64_t* nodes) {
  if (!b) return fail(RX_EINVAL, "null batch");
  if (replays) *replays = b->replays;
  if (nodes) *nodes = b->graph ? (int64_t)b->gnodes.size() : 0;
  return RX_OK;
}

void rx_batch_destroy(rx_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  for (int i = 0; i < rx_batch::kSlots; ++i) cudaEventSynchronize(b->ev_slot[i]);
  for (int p = 0; p < 4; ++p) cudaStreamSynchronize(b->s_stage[p]);
  for (rx_handle* h : b->h) {
    // every pending entry complete, so none keeps one of the batch's events
    sync_all(h);
    harvest(h);
    bool mine = false;
    for (cudaEvent_t e : b->ev_ring) mine |= h->batch_done == e;
    if (mine) h->batch_done = nullptr;
    // the batch's streams go away: the stream's work is complete, so its
    // next plain push starts from the legacy stream with nothing to join
    if (h->last_cs == b->s_stage[3]) {
      h->last_cs = nullptr;
      h->copy_dirty = false;
    }
  }
  batch_free(b);
  delete b;
}

}  // extern "C"
