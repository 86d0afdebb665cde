/*
 * rx.h -- C ABI of the GB300 dual-polarisation coherent receiver.
 *
 * One handle = one receiver stream.  The handle owns device memory on one
 * CUDA device and CUDA streams of its own; every step of the chain runs
 * in hand-written CUDA kernels (sm_103a) behind these calls.
 *
 * The chain (per stream, both polarisations jointly), with the passage of
 * arXiv 2108.07001 each step follows where the paper has one:
 *   ingest    pushed samples are appended to a device ring so that the stream
 *             stays contiguous across pushes (Sec. II: a kernel handles the
 *             overlap with the last block of the previous buffer);
 *   CD        overlap-save FFT -> x H -> IFFT with
 *             H = exp(+j beta2 L w^2/2) * RRC matched filter * exp(+j w tau)
 *             (Sec. II: 100 % overlap-save frequency-domain processing and
 *             frequency-domain static equalisation that compensates CD);
 *   timing    Godard band-edge spectral correlation, fed back per frame;
 *   FO        4th-power periodogram peak per frame, phase-continuous removal;
 *   MIMO      2x2 butterfly FIR, T taps at T/2 spacing, block-LMS adaptation
 *             (CMA acquisition, then decision-directed LMS: Sec. II uses a
 *             DD-LMS time-domain equaliser);
 *   BPS       blind phase search over B test angles, pi/2 unwrap;
 *   decide    hard decisions and Gray demapping (Sec. II);
 *   BER       against the known PRBS-31 payload, Q from BER (Sec. III).
 * The paper describes a single-polarisation Kramers-Kronig receiver; the
 * polarisation demultiplexing, CMA, FO/timing recovery and blind phase
 * search follow their textbook definitions.
 *
 * Error behaviour: every call returns RX_OK (0) or a negative RX_E* code;
 * rx_last_error() gives a message for the last failing call of the calling
 * thread.  No call aborts the process.
 */
#ifndef GB300_RX_H
#define GB300_RX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  RX_OK = 0,
  RX_EINVAL = -1,     /* bad argument or configuration */
  RX_ENOMEM = -2,     /* device or host allocation failed */
  RX_EAGAIN = -3,     /* no room: pull bits first (backpressure, not a failure) */
  RX_ETIMEDOUT = -4,  /* a wait ran out */
  RX_EDEVICE = -5,    /* CUDA error; see rx_last_error() */
  RX_ESTATE = -6      /* call not valid in this state (e.g. push after end of stream) */
};

enum { RX_QPSK = 2, RX_QAM16 = 4 };          /* bits per symbol per polarisation */
enum { RX_C128 = 0, RX_C64 = 1, RX_C16 = 2 }; /* complex double / float / half */

/* Receiver configuration.  Fill with rx_config_default() and override.
 * Sizes are in symbols per polarisation unless stated; sps is fixed at 2. */
typedef struct rx_config {
  double baud_hz;          /* symbol rate Rs; sample rate is 2 Rs */
  int modulation;          /* RX_QPSK or RX_QAM16 */
  double fiber_len_m;      /* fibre length L */
  double D_ps_nm_km;       /* dispersion parameter D */
  double lambda_m;         /* carrier wavelength (1550e-9) */
  double rrc_rolloff;      /* RRC matched filter roll-off folded into H; < 0: none */
  int fft_n;               /* OLS FFT size (power of two, 1024..32768); 0: auto */
  int cd_halo;             /* OLS overlap M-1 in samples (even); 0: 1.1 x CD memory */
  int mimo_taps;           /* T, odd, 3..31 */
  int bps_angles;          /* B: 32 or 64 */
  int bps_half_window;     /* W: window is 2W+1 symbols, 8/12/16/24/32 */
  int bps_coarse_stride;   /* S: 1 = search all B angles; B/16 (QPSK) or B/8
                              (16QAM) = two-stage search: the window costs
                              of the B/S angles b = S j, then the fine index
                              at the vertex of the parabola through the
                              coarse minimum and its two neighbours */
  int sub_block_syms;      /* K: symbols per tap update (64) */
  int seg_syms;            /* S: symbols per adaptive segment (multiple of K) */
  int frame_syms;          /* F: symbols per processing frame (multiple of S) */
  int cma_syms;            /* CMA portion of the acquisition */
  int acq_syms;            /* acquisition length (<= frame_syms) */
  float mu_cma, mu_dd;     /* LMS step sizes */
  float timing_gain;       /* feedback gain of the per-frame timing update */
  int storage_dtype;       /* device ring storage: RX_C64 or RX_C16 */
  uint64_t prbs_seed;      /* payload PRBS seed for BER counting; 0: no BER */
  int ber_skip_syms;       /* first symbol of the BER sync window */
  int sync_syms;           /* sync window length */
  int sync_max_delay;      /* delay search range +- */
  int slip_window;         /* cycle-slip window (symbols) */
  size_t max_block_samples;/* largest n_per_pol accepted by one push */
  int64_t history_syms;    /* keep equalised symbols, BPS angles and unwrap
                              counters of the first history_syms symbols on
                              the device for inspection; 0: off */
  int profile;             /* 1: time every stage with CUDA events */
  int device;              /* CUDA device ordinal */
  /* Launch tiles (results do not depend on them; rx_autotune_tiles picks
   * them on the GPU at hand): */
  int mimo_block_warps;    /* equaliser segment chains (one warp each) per block: 1, 2, 4 or 8; 0: 4 */
  int bps_block_runs;      /* full-search BPS runs of 256 symbols (one warp each) per block: 4 or 8; 0: 8 */
} rx_config;

/* Stages reported by rx_stage_times, in this order. */
enum { RX_STAGE_INGEST = 0, RX_STAGE_CD, RX_STAGE_EST, RX_STAGE_ACQUIRE, RX_STAGE_MIMO,
       RX_STAGE_BPS, RX_STAGE_DEMAP, RX_STAGE_BER, RX_NSTAGES };

/* Counters and the latest estimates.  All counts cover symbols processed
 * by completed frames. */
typedef struct rx_stats_t {
  uint64_t samples_in;     /* samples per polarisation pushed */
  uint64_t symbols_out;    /* symbols per polarisation decided */
  uint64_t frames;         /* frames completed */
  uint64_t bits;           /* payload bits compared (both polarisations) */
  uint64_t bit_errors;
  double ber;
  double q_db;             /* 20 log10(sqrt(2) erfcinv(2 BER)); 0 if no BER */
  double evm;              /* error power / reference power over counted symbols */
  uint64_t cycle_slips;
  int synced;              /* BER sync done */
  int sync_delay, sync_perm, sync_quadrant_x, sync_quadrant_y;
  int cma_reinit;          /* singularity re-initialisation happened */
  double fo_hz;            /* last frame's frequency offset estimate */
  double tau_s;            /* timing correction applied to the last frame */
  double latency_p50_ms, latency_p99_ms; /* push-to-decided latency of frames */
  double gpu_ms_total;     /* device time of completed frames */
} rx_stats_t;

typedef struct rx_handle rx_handle;

/* Defaults: QPSK at 28 GBd over 1,000 km of D = 17 ps/(nm km) at 1550 nm,
 * RRC 0.1, T = 15, B = 64, W = 16, K = 64, S = 512, F = 65536,
 * CMA 16384 of 20480 acquisition symbols, BER sync from symbol 16384 (the
 * CMA -> DD switch), mu_cma 3e-2, mu_dd 5e-3, timing
 * gain 0.5, complex64 storage, no BER, 2^17-sample pushes, no history,
 * device 0. */
void rx_config_default(rx_config* cfg);

/* Validates cfg, computes the CD filter in FP64 on the host and allocates
 * all device state on cfg->device.  *out receives the handle (caller frees
 * it with rx_destroy).  Returns RX_EINVAL (message says which field),
 * RX_ENOMEM or RX_EDEVICE. */
int rx_create(const rx_config* cfg, rx_handle** out);

/* Appends n_per_pol samples of both polarisations.  Layout: planar
 * [pol][n_per_pol], each sample re/im interleaved, element type dtype
 * (RX_C128 / RX_C64 / RX_C16).  on_device: 1 = samples is a device
 * pointer; 0 = a host pointer, copied before the call returns; 2 = a
 * pointer to page-locked host memory, copied to the device by a copy
 * engine in stream order without a host wait; 3 = a pointer to
 * page-locked host memory that the ingest kernel reads itself through the
 * device mapping (no copy engine, no staging buffer).  With 2 and 3 the
 * caller keeps the buffer unchanged until the work on cuda_stream has
 * passed it (RX_EINVAL if the memory is not page-locked and mapped).  The
 * call is asynchronous: the copy into the
 * library's ring is a kernel launched on cuda_stream (a cudaStream_t, NULL =
 * legacy default stream), so it follows the work already queued there and
 * later work on cuda_stream follows it; the caller may reuse a device
 * buffer in stream order.
 * When the ring is full, cuda_stream is made to wait for the frames that
 * still read the overwritten slots.
 * Complete frames are processed on the library's own stream.
 * samples == NULL with n_per_pol == 0 marks the end of the stream: the
 * remaining samples are processed with zeros beyond the end.
 * Returns RX_EINVAL (size > max_block_samples, bad dtype or on_device), RX_ESTATE (after
 * end of stream), RX_EAGAIN (decided bits not pulled and the output ring
 * is full) or RX_EDEVICE. */
int rx_push_block(rx_handle* h, const void* samples, size_t n_per_pol, int dtype,
                  int on_device, void* cuda_stream);

/* Copies up to cap_bytes*8 decided bits to the host buffer out (caller
 * owned) and removes them from the library.  Bit order: symbol-major,
 * polarisation x then y, per symbol the I bits then the Q bits, MSB first;
 * bit i of the stream is bit (7 - i%8) of out[i/8].  Only whole bytes are
 * returned; *n_bits receives the count.  Waits up to timeout_ms for queued
 * frames to finish (0: no wait, < 0: wait for all queued work).  Returns
 * RX_ETIMEDOUT if the wait ran out (bits decided so far are still
 * returned), RX_EDEVICE on a CUDA error. */
int rx_pull_bits(rx_handle* h, uint8_t* out, size_t cap_bytes, size_t* n_bits, int timeout_ms);

/* Waits for all queued work, then fills *out.  RX_EDEVICE on CUDA error. */
int rx_stats(rx_handle* h, rx_stats_t* out);

/* Many streams pushed in one call, one launch per stage (Sec. II: large
 * buffers keep many threads busy and cut per-launch overhead; here the
 * blocks of many streams fill each launch instead).  rx_batch_push
 * ingests every stream's block with one launch and then runs the frames
 * the blocks complete by ordinal: the i-th frame of every stream that
 * completes at least i + 1 frames goes through each stage (CD + timing/FO
 * statistics, estimators, acquisition, MIMO, BPS, demap, BER) in one
 * launch; streams whose FFT size and storage type, tap count or BPS form
 * differ get a launch of their own for that stage.
 * The ingest runs on cuda_stream; the stages run on the batch's own four
 * streams (front: CD and estimators, mid: acquisition and MIMO, back: BPS,
 * then demap and BER), pipelined over ordinals and calls with the buffer-reuse
 * waits of the plain path, so every stream gets what the same blocks
 * pushed with rx_push_block give: the same frames, sync and slips, soft
 * values equal to FP32 rounding (the batched kernels are compiled
 * separately), and so the same bits except where a decision lies within
 * that rounding of a threshold.  The arguments of a call are one page-locked table copied to
 * the device once (four tables rotate: a call waits on the host for the
 * call four back to finish).
 *
 * rx_batch_create: n_streams (1..RX_BATCH_MAX) distinct handles of one
 * device; the batch keeps the pointers (the caller keeps the handles alive
 * and destroys the batch first).  RX_EINVAL, RX_EDEVICE.
 * rx_batch_push: samples[c], n_per_pol[c] as rx_push_block for stream c
 * (n_per_pol[c] = 0 with samples[c] != NULL: nothing for c; samples[c] =
 * NULL with n_per_pol[c] = 0: end of stream c); on_device 1 (device
 * pointers) or 2 and 3 alike (page-locked host memory mapped for the
 * device, read by the ingest kernel in stream order: the caller keeps it
 * unchanged until the work on cuda_stream has passed it).  A refused call changes nothing:
 * RX_EINVAL (bad argument, size > max_block_samples), RX_ESTATE (a stream
 * has ended), RX_EAGAIN (a stream's output ring is full: pull its bits),
 * RX_EDEVICE.  Streams of a batch may also be pushed, pulled, reset and
 * ended through their own calls; work is ordered across the two paths.
 * Bits and statistics are read per stream (rx_pull_bits, rx_stats).
 * rx_batch_info: calls, kernel launches and frames of the batch so far, and
 * the host time its calls spent waiting for a table (ms; NULL pointers
 * skipped).
 * rx_batch_destroy: waits for the batch's streams, frees the batch (not
 * the streams).
 * rx_batch_set_graph: on = 1, before the batch's first push, switches it to
 * graph replay.  One CUDA graph is built here, node by node (no stream
 * capture, so other threads' CUDA calls are unaffected): every stage
 * launch of up to the batch's largest ordinal count per call, one kernel
 * node per ordinal and launch group, with the same stage-to-stage and
 * buffer-reuse edges as the stream mode.  Every later call replays it with one launch
 * on the batch's last stage stream after the call's ingest; on the host a
 * call only sets the grid of each node whose block count changed and
 * disables the nodes with no work (ordinals beyond the call's, groups with
 * no frame at an ordinal).  The graph reads the call's per-ordinal tables
 * from one fixed device table, so a call's table copy waits (on the
 * device) for the previous call's graph: consecutive calls do not overlap
 * their stages as in the stream mode.  Results equal the stream mode's.
 * on = 0 before the first push returns to the stream mode.  RX_EINVAL
 * (null batch), RX_ESTATE (the batch has pushed), RX_EDEVICE (building or
 * instantiating the graph failed; the batch stays in the stream mode).
 * rx_batch_graph_info: replays of the graph so far and kernel nodes in it
 * (both 0 in the stream mode); NULL pointers skipped. */
#define RX_BATCH_MAX 256
typedef struct rx_batch rx_batch;
int rx_batch_create(rx_handle* const* streams, int n_streams, rx_batch** out);
int rx_batch_push(rx_batch* b, const void* const* samples, const size_t* n_per_pol, int dtype, int on_device,
                  void* cuda_stream);
int rx_batch_info(const rx_batch* b, int64_t* calls, int64_t* launches, int64_t* frames, double* wait_ms);
void rx_batch_destroy(rx_batch* b);
int rx_batch_set_graph(rx_batch* b, int on);
int rx_batch_graph_info(const rx_batch* b, int64_t* replays, int64_t* nodes);

/* Waits for queued work and frees everything the handle owns. */
int rx_destroy(rx_handle* h);

/* Starts a new stream on the handle: the device state is re-initialised
 * in stream order after all queued work (no host wait), the host counters
 * restart, allocations and the CD filter are kept.  Bits of the previous
 * stream that were not pulled are dropped.  Stage timings are kept. */
int rx_reset(rx_handle* h);

/* Makes later work queued on cuda_stream (a cudaStream_t) wait for all
 * work the library has queued so far (stream-ordered completion; no host
 * wait).  Returns RX_EDEVICE on a CUDA error. */
int rx_join(rx_handle* h, void* cuda_stream);

/* Per-stage kernel launch counts since rx_create and, with
 * cfg.profile = 1, per-stage device time in ms (event pairs around each
 * stage on the library's streams); arrays of RX_NSTAGES entries indexed by
 * RX_STAGE_*.  Waits for queued work. */
int rx_stage_times(rx_handle* h, double* ms, int64_t* launches);

/* Message of the last failing call in this thread ("" if none). */
const char* rx_last_error(void);

/* ---- inspection (tests and tools) -------------------------------------
 * Per-frame estimates of the last completed frames, oldest first:
 * out[4*i + 0] = tau (s) applied, out[4*i+1] = FO estimate (Hz),
 * out[4*i+2] = AGC gain, out[4*i+3] = FO phase at the frame start (rad).
 * Returns the number of frames written (<= cap_frames) or a negative code.
 * The first 4096 frames of the stream are kept. */
int rx_frame_trace(rx_handle* h, double* out, int cap_frames);

/* Copies the 2x2xT complex taps [p][q][t] of the acquisition result
 * (which = -1) or of adaptive chain `which` (0 <= which < F/S) as float
 * re/im pairs into out (capacity 8*T floats).  Waits for queued work. */
int rx_get_taps(rx_handle* h, int which, float* out);

/* Copies equalised symbols y (MIMO output before carrier recovery) of
 * symbols [first, first + n) from the inspection history into host out as
 * complex float [pol][n] (re/im interleaved).  Waits for queued work.
 * RX_EINVAL if the range is outside [0, history_syms). */
int rx_get_equalised(rx_handle* h, int64_t first, int64_t n, float* out);

/* Copies the BPS angle index b (uint8, [pol][n]) and the unwrap counter m
 * (int32, [pol][n]) of symbols [first, first + n) from the inspection
 * history.  Waits for queued work.  RX_EINVAL outside the history. */
int rx_get_phase(rx_handle* h, int64_t first, int64_t n, uint8_t* bhat, int32_t* m);

/* ---- allocation-free block decisions ----------------------------------
 * The paper has no counterpart to this call; it exists for callers that
 * must not enter the CUDA allocator: for example a capture thread with a
 * hard deadline, where cudaMalloc's latency and implicit synchronisation
 * are not acceptable, or a process whose device memory is already held by
 * another pool allocator, so a cudaMalloc would fail.
 *
 * Blind phase search, unwrap, decisions and Gray demapping of one block of
 * n equalised symbols y (device, complex float, planar [2][n], re/im
 * interleaved), exactly as the streaming receiver decides a stream that
 * consists of this one block (window truncated at both ends, unwrap
 * counter starting at 0).  Decided bits go to the device buffer bits
 * (caller owned, at least ceil(n * 2 * modulation / 8) bytes) in the
 * rx_pull_bits order.  Work is queued on cuda_stream; nothing is allocated:
 * all working memory is one static device array of about 1.4 MB that every
 * device which loads the library holds until the process exits.
 *   n                 1 .. RX_NOALLOC_MAX_SYMS, else RX_EINVAL
 *   y                 8-byte aligned (a complex float), else RX_EINVAL
 *   modulation        RX_QPSK or RX_QAM16; bps_angles 32 or 64;
 *   bps_half_window   8, 12, 16, 24 or 32
 * The first call on a device (the device current at the call) looks up
 * that array's device address and sets kernel attributes; make that first
 * call before any stream capture.  All calls share the one array and it
 * keeps the last call's contents: calls whose work overlaps on the GPU
 * (different streams, or several host threads) race and must be ordered
 * by the caller.  Returns RX_OK, RX_EINVAL or RX_EDEVICE (message via
 * rx_last_error()). */
#define RX_NOALLOC_MAX_SYMS 65536
int rx_decide_block_noalloc(const void* y, int64_t n, int modulation, int bps_angles,
                            int bps_half_window, uint8_t* bits, void* cuda_stream);

/* ---- autotuner ----------------------------------------------------------
 * Picks the overlap-save FFT size for cfg on this GPU.  A larger N wastes a
 * smaller halo fraction h / N but costs more per output sample; the paper
 * fixes its block geometry for its own GPU (Sec. II).  Every admissible N
 * (a power of two in [1024, 32768] with N - halo >= 256) runs cfg's whole
 * chain on a zero stream (BER off): two frames untimed (the first, with the
 * acquisition, completes), then `frames` frames (1..64) timed; the fastest goes to *fft_n and its
 * time per 2^20 samples per polarisation to *ms_per_msample (may be NULL).  Creates and frees one
 * receiver per candidate; errors as rx_create, RX_EINVAL on bad arguments
 * or when no N is admissible. */
int rx_autotune_fft(const rx_config* cfg, int frames, int* fft_n, double* ms_per_msample);

/* Picks the FFT size and the launch tiles for cfg on this GPU: first the
 * FFT size as rx_autotune_fft (tiles 4 and 8), then the equaliser's
 * segment chains per block (1, 2, 4, 8), then the full blind phase
 * search's runs per block (4, 8; not for the two-stage search), each timed
 * with the others at their best so far and kept only if more than 1 %
 * faster.  The tiles change no result (rx_config.mimo_block_warps,
 * bps_block_runs); the paper picks its buffer and block sizes for its GPU
 * (Sec. II), this picks them for the GPU at hand.  Results in *fft_n,
 * *mimo_block_warps, *bps_block_runs and the time per 2^20 samples per
 * polarisation in *ms_per_msample (may be NULL).  Errors as
 * rx_autotune_fft. */
int rx_autotune_tiles(const rx_config* cfg, int frames, int* fft_n, int* mimo_block_warps, int* bps_block_runs,
                      double* ms_per_msample);

/* FP32 arithmetic peak of device, measured (the denominator of the ALU
 * rooflines): every SM filled with 2048 threads running eight independent
 * FMA chains, best of six timed launches, in TFLOP/s for the scalar form
 * (fma.rn.f32) in *tflops_fma and the packed-pair form (fma.rn.f32x2, two
 * FMAs per instruction) in *tflops_fma2.  RX_EINVAL (null pointer),
 * RX_EDEVICE. */
int rx_fp32_peak(int device, double* tflops_fma, double* tflops_fma2);

/* ---- serving: many channel streams on one GPU ---------------------------
 * The paper runs several CUDA streams so that buffers are processed
 * concurrently (Sec. II); a server extends this to many independent channel
 * streams.  It owns one receiver per channel stream, each with its state
 * (ring, equaliser taps, phase, timing, BER counters) resident on the
 * device between blocks, and worker threads that admit submitted capture
 * blocks in arrival order, round-robin over streams, as soon as the
 * stream's receiver can take them (its output ring has room), so blocks of
 * different streams are on the GPU at the same time and their work
 * overlaps.  Results of a stream do not depend on the other streams.
 *
 * Streams are admitted by device memory: rx_server_open creates the
 * stream's receiver and keeps it only if the device memory it holds fits
 * in what is left of the server's budget; otherwise it frees it again and
 * returns RX_EAGAIN (retry after closing a stream).
 *
 * Latency of a frame = time from the submission of the block that
 * completed the frame's input (its look-ahead included) to the frame's
 * bits being ready, host clock, queueing inside the server included.
 *
 * Batched rounds (batch = 1 or 2; max_streams <= RX_BATCH_MAX, one worker): the
 * worker keeps one rx_batch over the open streams and, each round, takes
 * the first queued block of every stream and pushes the device blocks of
 * one input type (dtype and on_device of the first such block) and the
 * ends of stream in one rx_batch_push, so each stage of every stream's
 * completed frames runs in one launch; the other blocks of the round
 * (pageable host blocks, other input types, or all of them when a
 * stream's output ring is full) go through their stream's rx_push_block.
 * A stream's results are the same alone and in any mix, and equal to the
 * same blocks pushed through an rx_batch of its own.  When streams open
 * or close, the worker builds the new batch at its next round and frees
 * the old one once its work is complete, without waiting for it
 * (rx_server_close returns once the stream is out of the batch and the
 * batch is freed).  batch = 2 switches each batch to graph replay
 * (rx_batch_set_graph) when it is built.
 *
 * Each receiver runs four CUDA streams; set CUDA_DEVICE_MAX_CONNECTIONS=32
 * in the environment before the process creates its CUDA context, or the
 * default 8 hardware queues serialise the streams' kernels (64 streams:
 * 4.0 vs 11.4 Gsamples/s on a GB300).
 */
typedef struct rx_server rx_server;

typedef struct rx_server_config {
  int64_t mem_budget_bytes; /* device memory for streams; <= 0: free memory at create minus 1 GiB */
  int max_streams;          /* 1 .. 1024 */
  int device;               /* CUDA device of every stream (their rx_config.device must match) */
  int64_t bits_cap_bytes;   /* per-stream host buffer of decided bits not yet pulled (>= 4096);
                               when full the stream's blocks wait (backpressure) */
  int workers;              /* worker threads, 1..64; worker k serves the streams with id % workers == k */
  int batch;                /* 0: every block through its stream's rx_push_block; 1: batched rounds (below);
                               2: batched rounds replaying one CUDA graph per round (rx_batch_set_graph) */
} rx_server_config;

typedef struct rx_server_stats_t {
  int64_t blocks_submitted, blocks_pushed, blocks_queued;
  int64_t samples_pushed;    /* samples per polarisation, all streams */
  int64_t frames_done;
  double latency_p50_ms, latency_p99_ms, latency_max_ms;
  int64_t latency_samples;
  int64_t mem_in_use_bytes, mem_budget_bytes;
  int streams_open;
  int worker_error;          /* first error of the worker (RX_* code), 0 if none */
  int64_t batch_calls;       /* batched mode: rx_batch_push calls made so far */
  double worker_round_ms;    /* host time the workers spent in passes / rounds */
  double worker_push_ms;     /* of which in rx_push_block / rx_batch_push calls */
  double worker_poll_ms;     /* of which polling frame completion and moving bits to the host */
} rx_server_stats_t;

void rx_server_config_default(rx_server_config* cfg);

/* Starts the worker thread.  RX_EINVAL on a bad config, RX_EDEVICE if the
 * device does not exist. */
int rx_server_create(const rx_server_config* cfg, rx_server** out);

/* Opens a channel stream with receiver configuration cfg (as rx_create);
 * *stream_id receives its id.  RX_EAGAIN when the stream does not fit in
 * the remaining memory budget or max_streams are open. */
int rx_server_open(rx_server* s, const rx_config* cfg, int* stream_id);

/* Queues one capture block of stream_id: planar [2][n_per_pol] samples of
 * dtype (as rx_push_block).  A host block is copied before the call
 * returns.  A device block (on_device) must hold its data when submitted
 * (it is read on the server's own CUDA streams, unordered with the
 * caller's) and stay valid and unchanged until rx_server_sync(s,
 * stream_id) returns.  Returns the block's sequence number (>= 0) or an
 * RX_* error (RX_EINVAL: bad stream, null or empty block, bad dtype;
 * RX_ESTATE: after rx_server_end). */
int64_t rx_server_submit(rx_server* s, int stream_id, const void* samples, size_t n_per_pol, int dtype,
                         int on_device);

/* Marks the end of stream_id's input: its remaining frames are processed
 * after its queued blocks. */
int rx_server_end(rx_server* s, int stream_id);

/* Waits until every block of stream_id submitted so far has been pushed
 * and all launched frames are done (and, after rx_server_end, the stream
 * is flushed).  timeout_ms < 0 waits without limit; RX_ETIMEDOUT when the
 * limit passes first.  Returns the worker's error if it stopped. */
int rx_server_sync(rx_server* s, int stream_id, int timeout_ms);

/* Moves up to cap_bytes of stream_id's decided bits (rx_pull_bits order)
 * out of the server's host buffer; *n_bits receives the count. */
int rx_server_pull_bits(rx_server* s, int stream_id, uint8_t* out, size_t cap_bytes, size_t* n_bits);

/* Statistics of stream_id's receiver (as rx_stats; waits for its queued
 * device work). */
int rx_server_stream_stats(rx_server* s, int stream_id, rx_stats_t* out);

/* The receiver of stream_id, for inspection calls (rx_get_equalised,
 * rx_frame_trace, ...) after rx_server_sync; NULL for a bad id. */
rx_handle* rx_server_handle(rx_server* s, int stream_id);

/* Waits for stream_id's queued work, frees its receiver and its budget. */
int rx_server_close(rx_server* s, int stream_id);

int rx_server_stats(rx_server* s, rx_server_stats_t* out);

/* Stops the worker, closes every stream and frees the server. */
int rx_server_destroy(rx_server* s);

/* ---- Kramers-Kronig front end (paper Sec. II) ------------------------------
 *
 * The paper's own receiver detects a single-polarisation minimum-phase
 * signal (a carrier tone plus QAM on one side of it) with one photodiode
 * and a 12-bit ADC, and recovers the optical field with the Kramers-Kronig
 * relations.  Per sample t of the stream:
 *
 *   I_t = adc_gain (code_t - adc_offset)             (12-bit fixed point to float)
 *   u_t = ln(max(I_t, adc_gain / 2)) / 2              (log amplitude)
 *   phi = Hilbert transform of u in 100 % overlap-save blocks of N = fft_n
 *         samples: segment b holds outputs [b N/2, (b+1) N/2) and is taken
 *         from samples N/4 .. 3N/4 - 1 of the block over [b N/2 - N/4,
 *         b N/2 + 3N/4) (u = 0 outside the stream), whose DFT is multiplied
 *         by -j sgn(k) (0 at k = 0 and N/2)
 *   E_t = exp(u_t + j phi_t) exp(-j 2 pi (f_shift_hz / fs_hz) t)   (field, downshifted)
 *
 * Output: complex64 field samples (re, im interleaved) in device memory, in
 * stream order.  A segment is written once the input reaches the end of its
 * block, so the output lags the input by N/4 to 3N/4 - 1 samples until
 * rx_kk_end writes the rest. */
typedef struct rx_kk_config {
  double fs_hz;            /* ADC sample rate */
  double f_shift_hz;       /* downshift frequency: signal centre above the carrier */
  double adc_gain;         /* intensity per ADC code (> 0) */
  double adc_offset;       /* ADC code of zero intensity */
  int fft_n;               /* N: 1024 (the paper's), 2048 or 4096 */
  size_t max_block_samples;/* largest n accepted by one rx_kk_push */
  int device;              /* CUDA device ordinal */
} rx_kk_config;

typedef struct rx_kk rx_kk;

/* Defaults: 4 GS/s, shift 0.516 GHz, gain 1, offset 0, N = 1024, 2^22-sample
 * pushes (the paper's buffer), device 0. */
void rx_kk_config_default(rx_kk_config* cfg);

/* Validates cfg (RX_EINVAL naming the field), allocates the device state
 * (carry of the previous block's samples, staging for host pushes, FFT
 * twiddles) on cfg->device.  *out receives the handle; free with
 * rx_kk_destroy. */
int rx_kk_create(const rx_kk_config* cfg, rx_kk** out);

/* Appends n ADC codes (int16, the 12-bit values).  on_device: 1 = codes is
 * a device pointer read in stream order; 0 = host memory copied in stream
 * order (page-locked memory is copied without a host wait and must stay
 * unchanged until the stream passes the copy; pageable memory is staged
 * before the call returns).  Writes the field of every newly complete
 * segment to out (device, complex64), *n_out samples, in stream order on
 * cuda_stream (NULL: the legacy default stream).  RX_EINVAL if n exceeds
 * max_block_samples or out_cap (complex samples) is smaller than *n_out
 * would be (at most n + fft_n/2 - 1); RX_ESTATE after rx_kk_end. */
int rx_kk_push(rx_kk* h, const int16_t* codes, size_t n, int on_device, float* out, size_t out_cap,
               size_t* n_out, void* cuda_stream);

/* End of stream: writes the field of the remaining samples (at most
 * 3 fft_n/4 - 1) to out, *n_out of them; input past the end counts as
 * absent. */
int rx_kk_end(rx_kk* h, float* out, size_t out_cap, size_t* n_out, void* cuda_stream);

/* Starts a new stream on the same handle (stream order: call after the
 * previous stream's work, or on the same CUDA stream). */
int rx_kk_reset(rx_kk* h);

/* Samples pushed and field samples written so far. */
int rx_kk_position(const rx_kk* h, int64_t* samples_in, int64_t* samples_out);

void rx_kk_destroy(rx_kk* h);

/* Many front ends in one launch: rx_kk_batch_push plans a push of every
 * channel, writes the plans to a table and replays a CUDA graph of the
 * table's copy, one field kernel over every channel's segment pairs
 * (channels' pushes may differ in length; a block finds its channel from
 * the prefix sums of their pair counts) and one carry kernel.  Each
 * channel's results are those of rx_kk_push with the same codes.  The
 * channels must share fft_n and device and must not be pushed otherwise
 * while the batch is in use; rx_kk_batch_destroy does not free them. */
typedef struct rx_kk_batch rx_kk_batch;

/* n_channels in 1..256 distinct handles; builds the graphs. */
int rx_kk_batch_create(rx_kk* const* channels, int n_channels, rx_kk_batch** out);

/* For every channel c: n[c] codes at the device pointer codes[c] (0: none
 * this time), field out to out[c] (device, capacity out_cap[c] complex
 * samples), n_out[c] written, in stream order on cuda_stream.  Checks
 * every channel before launching anything (RX_EINVAL / RX_ESTATE as
 * rx_kk_push). */
int rx_kk_batch_push(rx_kk_batch* b, const int16_t* const* codes, const size_t* n, float* const* out,
                     const size_t* out_cap, size_t* n_out, void* cuda_stream);

void rx_kk_batch_destroy(rx_kk_batch* b);

/* ---- KK receiver chain (paper Sec. II) -------------------------------------
 *
 * The rest of the paper's single-polarisation receiver after the KK front
 * end: the downshifted field at 4 samples per symbol goes through
 *
 *   a static equaliser with resampling to 2 samples per symbol: 100 %
 *     overlap-save blocks of eq_fft_n samples (N4) advancing by N4/2; each
 *     block's DFT is cut to the 2-sps band (bins -N4/4 .. N4/4 - 1) and
 *     multiplied by the CD compensation exp(+j beta2 L w^2 / 2), w = 2 pi
 *     (f + f_shift) (the dispersion acted with the carrier at DC), times the
 *     RRC matched filter; an N4/2-point inverse DFT gives 2-sps outputs
 *     [b N4/4, (b+1) N4/4) from its samples N4/8 .. 3N4/8 - 1;
 *   a widely-linear DD-LMS equaliser with 4 taps at 2 samples per symbol,
 *     y_k = sum_t h1[t] x[2k+t-1] + h2[t] conj(x[2k+t-1]): block-LMS over
 *     sub-blocks of 64 symbols (e = y - dec(y), h1 -= mu mean(e conj x),
 *     h2 -= mu mean(e x)); one sequential acquisition chain over the first
 *     acq_syms symbols from h1 = unit tap at offset 0, h2 = 0, then frames
 *     of frame_syms symbols cut into segments of seg_syms, each continuing
 *     its own taps from the previous frame;
 *   hard decisions and Gray demapping to packed bits (symbol-major, I bits
 *     then Q bits, MSB first; QPSK - -> 1, + -> 0; 16QAM -3, -1, 1, 3 ->
 *     00, 01, 11, 10 at unit symbol energy). */
typedef struct rx_kkrx_config {
  rx_kk_config fe;         /* the front end; fe.fs_hz must be 4 x baud_hz */
  double baud_hz;          /* symbol rate */
  int modulation;          /* RX_QPSK or RX_QAM16 */
  double fiber_len_m;      /* L for the CD compensation */
  double D_ps_nm_km;       /* dispersion parameter */
  double lambda_m;         /* carrier wavelength */
  double rrc_rolloff;      /* matched filter roll-off (paper: 0.01) */
  int eq_fft_n;            /* N4: 1024 or 2048 */
  float mu;                /* DD-LMS step size */
  int seg_syms;            /* S: multiple of 64 */
  int frame_syms;          /* F: multiple of S, at most 2^24 */
  int acq_syms;            /* acquisition chain length, multiple of 64, <= F */
  int64_t history_syms;    /* keep the equalised symbols of the first history_syms
                              symbols for rx_kkrx_equalised; 0: off */
} rx_kkrx_config;

typedef struct rx_kkrx rx_kkrx;

/* Defaults: the front end's defaults, 1 GBd QPSK, no fibre, D = 17 at
 * 1550 nm, roll-off 0.01, N4 = 1024, mu 5e-3, S = 512, F = 2^20 (one 2^22-
 * sample ADC buffer per frame), acquisition 8192 symbols, no history. */
void rx_kkrx_config_default(rx_kkrx_config* cfg);

/* Validates cfg (RX_EINVAL naming the field) and allocates the chain on
 * cfg->fe.device; free with rx_kkrx_destroy. */
int rx_kkrx_create(const rx_kkrx_config* cfg, rx_kkrx** out);

/* Appends n ADC codes (as rx_kk_push: on_device 1 = device pointer, 0 =
 * host memory).  The bits of every frame this push completes, *n_bits of
 * them (a whole number of frames), are written to bits (device memory,
 * packed); a frame completes once the 2-sps samples reach 2(f+1)F + 1.
 * The front end runs in stream order on cuda_stream, the equaliser and the
 * DD-LMS on the handle's own stream, so successive pushes overlap: the bits
 * are in place (and the codes' device memory free) in cuda_stream's order
 * after rx_kkrx_end, or after cudaDeviceSynchronize.  RX_EINVAL if
 * bits_cap_bytes is too small. */
int rx_kkrx_push(rx_kkrx* h, const int16_t* codes, size_t n, int on_device, uint8_t* bits,
                 size_t bits_cap_bytes, size_t* n_bits, void* cuda_stream);

/* End of stream: the remaining frames (the last one may be short; symbols
 * = codes / 4) and their bits; samples past the end count as zero.  Joins
 * the handle's stream onto cuda_stream: all of the stream's bits are in
 * place in cuda_stream's order. */
int rx_kkrx_end(rx_kkrx* h, uint8_t* bits, size_t bits_cap_bytes, size_t* n_bits, void* cuda_stream);

/* Equalised symbols [first, first + n) (within history_syms) as complex
 * float pairs, copied to host memory after the device is idle. */
int rx_kkrx_equalised(rx_kkrx* h, int64_t first, int64_t n, float* out);

/* Starts a new stream (waits for the handle's own stream first). */
int rx_kkrx_reset(rx_kkrx* h);

/* Many receivers in one launch per stage: rx_kkrx_batch_push runs every
 * channel's front end in one rx_kk_batch graph replay, every channel's
 * new equaliser segments in one more graph replay (uneven counts; a block
 * finds its channel from their prefix sums) and the DD-LMS of each frame
 * that completed, all in stream order on cuda_stream.  Each channel's bits
 * are those of rx_kkrx_push with the same codes.  The channels must share
 * fe.fft_n, eq_fft_n, frame_syms, seg_syms, acq_syms, modulation and device,
 * and are not pushed otherwise while the batch is in use; their streams
 * end with rx_kkrx_end.  rx_kkrx_batch_destroy does not free them. */
typedef struct rx_kkrx_batch rx_kkrx_batch;

/* n_channels in 1..256 distinct handles (waits for their own streams). */
int rx_kkrx_batch_create(rx_kkrx* const* channels, int n_channels, rx_kkrx_batch** out);

/* For every channel c: n[c] codes at the device pointer codes[c] (0: none),
 * the bits of the frames it completes to bits[c] (device, capacity
 * bits_cap_bytes[c]), n_bits[c] of them.  Checks every channel before
 * launching anything. */
int rx_kkrx_batch_push(rx_kkrx_batch* b, const int16_t* const* codes, const size_t* n, uint8_t* const* bits,
                       const size_t* bits_cap_bytes, size_t* n_bits, void* cuda_stream);

void rx_kkrx_batch_destroy(rx_kkrx_batch* b);

void rx_kkrx_destroy(rx_kkrx* h);

#ifdef __cplusplus
}
#endif
#endif /* GB300_RX_H */
