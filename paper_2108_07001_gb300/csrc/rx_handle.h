// The receiver handle behind rx_create .. rx_destroy and the host-runtime
// helpers shared by the plain path (rx_runtime.cu) and the batched path
// (rx_batch.cu).  Library-internal: not part of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <deque>
#include <string>
#include <vector>

#include "../../include/rx.h"
#include "rx_internal.cuh"

namespace rx {
cudaError_t launch_cd(const RxDev& d, const FrameArgs& fa, cudaStream_t s);
cudaError_t launch_est(const RxDev& d, const FrameArgs& fa, int mode, cudaStream_t s);
cudaError_t launch_acquire(const RxDev& d, const FrameArgs& fa, cudaStream_t s);
cudaError_t launch_mimo(const RxDev& d, const FrameArgs& fa, cudaStream_t s);
cudaError_t launch_bps(const RxDev& d, const FrameArgs& fa, cudaStream_t s);
cudaError_t launch_unwrap_demap(const RxDev& d, const FrameArgs& fa, cudaStream_t s);
cudaError_t launch_ref_gen(const RxDev& d, long long sym0, int nbits, int use_delay, cudaStream_t s);
cudaError_t launch_sync(const RxDev& d, cudaStream_t s);
cudaError_t launch_ber(const RxDev& d, long long ka, long long kb, long long w_from, long long w_to,
                       long long k_lim, int n_win_ring, cudaStream_t s);
cudaError_t launch_ingest(const RxDev& d, const void* src, int dtype, long long n, long long w0, cudaStream_t s);
cudaError_t cd_set_attributes();
cudaError_t bps_set_attributes();
cudaError_t ber_set_attributes();
// batched launches (rx_batch_push): grid widths per frame and launchers
int cd_grid_x(const RxDev& d, const FrameArgs& fa);
int est_grid_x(const RxDev& d);
int mimo_grid_x(const RxDev& d, const FrameArgs& fa);
int bps_grid_x(const RxDev& d, const FrameArgs& fa);
int demap_grid_x(const FrameArgs& fa);
int ref_grid_x(int nbits);
int sync_grid_x(const RxDev& d);
int ber_grid_x(const RxDev& d, long long ka, long long kb);
int ingest_grid_x(long long n, bool pairs);
bool ingest_pairs_ok(const RxDev& d, const void* src, int dtype, long long n, long long w0);
cudaError_t launch_ingest_batch(const BIngest* ing, const BView& v, int blocks, cudaStream_t s);
cudaError_t launch_cd_batch(const RxDev& d, const BView& v, int blocks, int pass, cudaStream_t s);
cudaError_t launch_est_batch(const BView& v, int blocks, int mode, cudaStream_t s);
cudaError_t launch_acquire_batch(const RxDev& d, const BView& v, int blocks, cudaStream_t s);
cudaError_t launch_mimo_batch(const RxDev& d, const BView& v, int blocks, cudaStream_t s);
cudaError_t launch_bps_batch(const RxDev& d, const BView& v, int blocks, cudaStream_t s);
cudaError_t launch_demap_batch(const BView& v, int blocks, cudaStream_t s);
cudaError_t launch_scan_batch(const BView& v, int blocks, cudaStream_t s);
cudaError_t launch_ref_gen_batch(const BView& v, int blocks, int use_delay, cudaStream_t s);
cudaError_t launch_sync_batch(const BView& v, int blocks, cudaStream_t s);
cudaError_t launch_ber_batch(const BView& v, int blocks, cudaStream_t s);
int cd_halo_samples(const rx_config* cfg);
}  // namespace rx

namespace rxrt {

using namespace rx;

// Sets the message of rx_last_error() and returns code.
int fail(int code, const std::string& msg);
// RX_EDEVICE with the CUDA error's text.
int cuda_fail(cudaError_t e, const char* where);

#define RX_CK(call)                                    \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

constexpr double kC = 299792458.0;
constexpr int kZSlots = 6;      // frames in flight between the front and back streams
constexpr int kRingFrames = 3;  // frames of input the ring holds (plus look-ahead and one push): the
                                // pushes of the next frames land while the CD reads the current one
constexpr int kStageSlots = 8;  // device staging buffers of host pushes

struct StageEv {
  int stage;
  cudaEvent_t a, b;
};

struct PendingFrame {
  long long f;
  long long gen;         // stream generation (rx_reset increments it)
  long long bits_after;  // bits produced once this frame completes
  long long dec_after;
  cudaEvent_t ev_in, ev_start, ev_done;
  std::vector<StageEv> sev;
  long long nframes = 1; // frames it completes (a batched push: all of the stream's frames of the round)
  bool shared = false;   // the events belong to a batch (not returned to the handle's pool)
};

}  // namespace rxrt

struct rx_handle {
  rx_config cfg;
  rx::RxDev d;
  cudaStream_t s_copy = nullptr;
  cudaStream_t s_front = nullptr;  // CD + estimator of each frame
  cudaStream_t s_mid = nullptr;    // acquisition and MIMO
  cudaStream_t s_comp = nullptr;   // BPS of even decide passes ("back")
  cudaStream_t s_comp2 = nullptr;  // BPS of odd decide passes (consecutive frames' BPS overlap)
  cudaEvent_t ev_mid[2] = {};      // MIMO of a frame done (its y buffer written), by frame parity
  cudaEvent_t ev_bpsd[2] = {};     // BPS of a frame done (its y buffer free again), by frame parity
  cudaEvent_t ev_bpsp[2] = {};     // BPS of a decide pass done (its decision buffers written), by pass parity
  cudaEvent_t ev_front[rxrt::kZSlots] = {};  // front work of the frame in slot done
  cudaEvent_t ev_mimo[rxrt::kZSlots] = {};   // MIMO of the frame in slot done (slot reusable)
  cudaStream_t s_dem = nullptr;        // unwrap scan and demap, after the BPS
  cudaStream_t s_ber = nullptr;        // BER counting (metrics), after the demap
  cudaEvent_t ev_dem[2] = {};          // demap of a decide pass done (its decision buffers free), by pass parity
  cudaEvent_t ev_berd[2] = {};         // BER work of a frame done (its ring slots reusable)
  long long n_decide = 0;              // decision passes launched in this stream
  cudaEvent_t ev_copy = nullptr;   // last ingest (recorded on the pushing stream)
  cudaEvent_t ev_reset = nullptr;  // last rx_reset (recorded on the compute stream)
  bool reset_pending = false;
  cudaStream_t last_cs = nullptr;  // stream of the last push (input arrival events)
  bool copy_dirty = false;         // ingests queued since ev_copy was last recorded
  long long pushed = 0;       // samples per pol written to the ring
  long long n_total = -1;     // samples per pol in the stream (after end)
  bool ended = false;
  long long f_next = 0;       // next frame to launch
  long long f_waited = 0;     // frames whose CD pass the copy stream has waited for
  long long decided = 0;      // symbols decided by launched work
  long long bits_done = 0;    // bits of completed frames
  long long bits_pulled = 0;
  long long dec_done = 0;
  bool synced = false;
  bool tail_launched = false;
  long long w_next = 0;       // next BER slip window to finalise
  int n_win_ring = 0;
  int la = 0;                 // lookahead samples beyond a frame
  int tail = 0;               // symbols excluded from BER at the stream end
  std::vector<cudaEvent_t> cd_done;   // per frame slot (ring of 64)
  std::deque<rxrt::PendingFrame> pend;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<double> lat_ms;
  double gpu_ms = 0.0;
  long long frames_done = 0;
  void* stage[rxrt::kStageSlots] = {};              // device staging for host pushes
  cudaEvent_t ev_stage_in[rxrt::kStageSlots] = {};   // H2D copy into the slot done (copy stream)
  cudaEvent_t ev_stage_free[rxrt::kStageSlots] = {}; // ingest of the slot done (pushing stream)
  long long stage_i = 0;
  size_t stage_bytes = 0;
  std::deque<rxrt::StageEv> ingest_ev;
  long long gen = 0;
  rx::StreamState st_init{};             // initial device state (host copy for resets)
  double stage_ms[RX_NSTAGES] = {0};
  long long stage_n[RX_NSTAGES] = {0};   // kernel launches per stage
  size_t dev_bytes = 0;                  // device memory held by the handle
  bool own_work = false;                 // frames launched on the handle's own streams since its last batched push
  cudaEvent_t batch_done = nullptr;      // end of the last batched push that carried this stream (the batch's event)
};

namespace rxrt {

cudaEvent_t get_event(rx_handle* h);
// Harvest completed frames (in order): latency, device time, bits.
void harvest(rx_handle* h);
// Waits for everything the library has queued.
cudaError_t sync_all(rx_handle* h);
// Records ev_copy after the ingests queued so far (on the last push stream).
cudaError_t mark_copy(rx_handle* h);

// The BER work of a decision pass (host state advanced as it is planned):
// the sync search once the sync window has been decided, then the
// reference bits and the count of every newly decided symbol.
struct BerPlan {
  bool sync = false;       // reference of the sync window + the sync search
  long long sync_sym0 = 0;
  int sync_nbits = 0;
  bool ref = false;        // reference of the counted range
  long long ref_sym0 = 0;
  int ref_nbits = 0;
  bool count = false;      // the count pass (launch_ber; it may find nothing to do)
  long long ka = 0, kb = 0, w_from = 0, w_to = 0, k_lim = 0;
  int launches = 0;        // kernels the plain path launches for it
};

BerPlan plan_ber(rx_handle* h, const FrameArgs& fa, bool final_);
FrameArgs frame_args(const rx_handle* h, long long f, bool final_);
// The timing-acquisition CD pass before the first frame.
FrameArgs est_pass_args(const FrameArgs& fa);
// Device state with frame f's slot.
RxDev slot_dev(const rx_handle* h, long long f);
RxDev decide_dev(const RxDev& base, long long pass);
// The decide-only pass at the stream end.
FrameArgs tail_args(const rx_handle* h);

}  // namespace rxrt
