"""ctypes binding of the receiver's C ABI (include/rx.h).

Argument marshalling only: every step of the chain runs in the CUDA
kernels of librx.so.  Loading fails loudly when the library is missing;
there is no fallback.  Device buffers come from PyTorch (``data_ptr()``)
and streams from ``torch.cuda.current_stream().cuda_stream``; numpy arrays
are pushed from host memory.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librx.so")

RX_OK, RX_EINVAL, RX_ENOMEM, RX_EAGAIN, RX_ETIMEDOUT, RX_EDEVICE, RX_ESTATE = 0, -1, -2, -3, -4, -5, -6
RX_QPSK, RX_QAM16 = 2, 4
RX_C128, RX_C64, RX_C16 = 0, 1, 2

# Each receiver drives four CUDA streams and a server many receivers; with
# the default 8 hardware work queues their kernels serialise.  The count is
# read when the process creates its CUDA context, so this only takes effect
# if the binding is imported before CUDA is initialised.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
STAGES = ["ingest", "cd", "est", "acquire", "mimo", "bps", "demap", "ber"]

# every function declared in include/rx.h
EXPORTS = ["rx_config_default", "rx_create", "rx_push_block", "rx_pull_bits", "rx_stats",
           "rx_destroy", "rx_reset", "rx_join", "rx_stage_times", "rx_last_error",
           "rx_frame_trace", "rx_get_taps", "rx_get_equalised", "rx_get_phase",
           "rx_decide_block_noalloc", "rx_batch_create", "rx_batch_push", "rx_batch_info", "rx_batch_destroy",
           "rx_batch_set_graph", "rx_batch_graph_info",
           "rx_server_config_default", "rx_server_create", "rx_server_open", "rx_server_submit",
           "rx_server_end", "rx_server_sync", "rx_server_pull_bits", "rx_server_stream_stats",
           "rx_server_handle", "rx_server_close", "rx_server_stats", "rx_server_destroy",
           "rx_autotune_fft", "rx_autotune_tiles", "rx_fp32_peak",
           "rx_kk_config_default", "rx_kk_create", "rx_kk_push", "rx_kk_end", "rx_kk_reset",
           "rx_kk_position", "rx_kk_destroy", "rx_kk_batch_create", "rx_kk_batch_push", "rx_kk_batch_destroy",
           "rx_kkrx_config_default", "rx_kkrx_create", "rx_kkrx_push", "rx_kkrx_end", "rx_kkrx_equalised",
           "rx_kkrx_reset", "rx_kkrx_destroy", "rx_kkrx_batch_create", "rx_kkrx_batch_push",
           "rx_kkrx_batch_destroy"]


class RxConfig(ctypes.Structure):
    _fields_ = [
        ("baud_hz", ctypes.c_double),
        ("modulation", ctypes.c_int),
        ("fiber_len_m", ctypes.c_double),
        ("D_ps_nm_km", ctypes.c_double),
        ("lambda_m", ctypes.c_double),
        ("rrc_rolloff", ctypes.c_double),
        ("fft_n", ctypes.c_int),
        ("cd_halo", ctypes.c_int),
        ("mimo_taps", ctypes.c_int),
        ("bps_angles", ctypes.c_int),
        ("bps_half_window", ctypes.c_int),
        ("bps_coarse_stride", ctypes.c_int),
        ("sub_block_syms", ctypes.c_int),
        ("seg_syms", ctypes.c_int),
        ("frame_syms", ctypes.c_int),
        ("cma_syms", ctypes.c_int),
        ("acq_syms", ctypes.c_int),
        ("mu_cma", ctypes.c_float),
        ("mu_dd", ctypes.c_float),
        ("timing_gain", ctypes.c_float),
        ("storage_dtype", ctypes.c_int),
        ("prbs_seed", ctypes.c_uint64),
        ("ber_skip_syms", ctypes.c_int),
        ("sync_syms", ctypes.c_int),
        ("sync_max_delay", ctypes.c_int),
        ("slip_window", ctypes.c_int),
        ("max_block_samples", ctypes.c_size_t),
        ("history_syms", ctypes.c_int64),
        ("profile", ctypes.c_int),
        ("device", ctypes.c_int),
        ("mimo_block_warps", ctypes.c_int),
        ("bps_block_runs", ctypes.c_int),
    ]


class KKConfig(ctypes.Structure):
    """rx_kk_config: the Kramers-Kronig front end."""
    _fields_ = [
        ("fs_hz", ctypes.c_double),
        ("f_shift_hz", ctypes.c_double),
        ("adc_gain", ctypes.c_double),
        ("adc_offset", ctypes.c_double),
        ("fft_n", ctypes.c_int),
        ("max_block_samples", ctypes.c_size_t),
        ("device", ctypes.c_int),
    ]


class KKRxConfig(ctypes.Structure):
    """rx_kkrx_config: the KK receiver chain."""
    _fields_ = [
        ("fe", KKConfig),
        ("baud_hz", ctypes.c_double),
        ("modulation", ctypes.c_int),
        ("fiber_len_m", ctypes.c_double),
        ("D_ps_nm_km", ctypes.c_double),
        ("lambda_m", ctypes.c_double),
        ("rrc_rolloff", ctypes.c_double),
        ("eq_fft_n", ctypes.c_int),
        ("mu", ctypes.c_float),
        ("seg_syms", ctypes.c_int),
        ("frame_syms", ctypes.c_int),
        ("acq_syms", ctypes.c_int),
        ("history_syms", ctypes.c_int64),
    ]


class RxStats(ctypes.Structure):
    _fields_ = [
        ("samples_in", ctypes.c_uint64),
        ("symbols_out", ctypes.c_uint64),
        ("frames", ctypes.c_uint64),
        ("bits", ctypes.c_uint64),
        ("bit_errors", ctypes.c_uint64),
        ("ber", ctypes.c_double),
        ("q_db", ctypes.c_double),
        ("evm", ctypes.c_double),
        ("cycle_slips", ctypes.c_uint64),
        ("synced", ctypes.c_int),
        ("sync_delay", ctypes.c_int),
        ("sync_perm", ctypes.c_int),
        ("sync_quadrant_x", ctypes.c_int),
        ("sync_quadrant_y", ctypes.c_int),
        ("cma_reinit", ctypes.c_int),
        ("fo_hz", ctypes.c_double),
        ("tau_s", ctypes.c_double),
        ("latency_p50_ms", ctypes.c_double),
        ("latency_p99_ms", ctypes.c_double),
        ("gpu_ms_total", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerConfig(ctypes.Structure):
    _fields_ = [
        ("mem_budget_bytes", ctypes.c_int64),
        ("max_streams", ctypes.c_int),
        ("device", ctypes.c_int),
        ("bits_cap_bytes", ctypes.c_int64),
        ("workers", ctypes.c_int),
        ("batch", ctypes.c_int),
    ]


class ServerStats(ctypes.Structure):
    _fields_ = [
        ("blocks_submitted", ctypes.c_int64),
        ("blocks_pushed", ctypes.c_int64),
        ("blocks_queued", ctypes.c_int64),
        ("samples_pushed", ctypes.c_int64),
        ("frames_done", ctypes.c_int64),
        ("latency_p50_ms", ctypes.c_double),
        ("latency_p99_ms", ctypes.c_double),
        ("latency_max_ms", ctypes.c_double),
        ("latency_samples", ctypes.c_int64),
        ("mem_in_use_bytes", ctypes.c_int64),
        ("mem_budget_bytes", ctypes.c_int64),
        ("streams_open", ctypes.c_int),
        ("worker_error", ctypes.c_int),
        ("batch_calls", ctypes.c_int64),
        ("worker_round_ms", ctypes.c_double),
        ("worker_push_ms", ctypes.c_double),
        ("worker_poll_ms", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load librx.so and declare the signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"receiver library not built: {path} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P, I, SZ, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_int64
    lib.rx_config_default.argtypes = [ctypes.POINTER(RxConfig)]
    lib.rx_config_default.restype = None
    lib.rx_create.argtypes = [ctypes.POINTER(RxConfig), ctypes.POINTER(P)]
    lib.rx_push_block.argtypes = [P, P, SZ, I, I, P]
    lib.rx_pull_bits.argtypes = [P, P, SZ, ctypes.POINTER(SZ), I]
    lib.rx_stats.argtypes = [P, ctypes.POINTER(RxStats)]
    lib.rx_destroy.argtypes = [P]
    lib.rx_reset.argtypes = [P]
    lib.rx_join.argtypes = [P, P]
    lib.rx_stage_times.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64)]
    lib.rx_last_error.argtypes = []
    lib.rx_last_error.restype = ctypes.c_char_p
    lib.rx_frame_trace.argtypes = [P, ctypes.POINTER(ctypes.c_double), I]
    lib.rx_get_taps.argtypes = [P, I, ctypes.POINTER(ctypes.c_float)]
    lib.rx_get_equalised.argtypes = [P, I64, I64, ctypes.POINTER(ctypes.c_float)]
    lib.rx_get_phase.argtypes = [P, I64, I64, ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ctypes.c_int32)]
    lib.rx_decide_block_noalloc.argtypes = [P, I64, I, I, I, P, P]
    lib.rx_server_config_default.argtypes = [ctypes.POINTER(ServerConfig)]
    lib.rx_server_config_default.restype = None
    lib.rx_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(P)]
    lib.rx_server_open.argtypes = [P, ctypes.POINTER(RxConfig), ctypes.POINTER(I)]
    lib.rx_server_submit.argtypes = [P, I, P, SZ, I, I]
    lib.rx_server_submit.restype = I64
    lib.rx_server_end.argtypes = [P, I]
    lib.rx_server_sync.argtypes = [P, I, I]
    lib.rx_server_pull_bits.argtypes = [P, I, P, SZ, ctypes.POINTER(SZ)]
    lib.rx_server_stream_stats.argtypes = [P, I, ctypes.POINTER(RxStats)]
    lib.rx_server_handle.argtypes = [P, I]
    lib.rx_server_handle.restype = P
    lib.rx_server_close.argtypes = [P, I]
    lib.rx_server_stats.argtypes = [P, ctypes.POINTER(ServerStats)]
    lib.rx_server_destroy.argtypes = [P]
    lib.rx_autotune_fft.argtypes = [ctypes.POINTER(RxConfig), I, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_double)]
    lib.rx_autotune_tiles.argtypes = [ctypes.POINTER(RxConfig), I, ctypes.POINTER(I), ctypes.POINTER(I),
                                      ctypes.POINTER(I), ctypes.POINTER(ctypes.c_double)]
    lib.rx_kk_config_default.argtypes = [ctypes.POINTER(KKConfig)]
    lib.rx_kk_config_default.restype = None
    lib.rx_kk_create.argtypes = [ctypes.POINTER(KKConfig), ctypes.POINTER(P)]
    lib.rx_kk_push.argtypes = [P, P, SZ, I, P, SZ, ctypes.POINTER(SZ), P]
    lib.rx_kk_end.argtypes = [P, P, SZ, ctypes.POINTER(SZ), P]
    lib.rx_kk_reset.argtypes = [P]
    lib.rx_kk_position.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64)]
    lib.rx_kk_destroy.argtypes = [P]
    lib.rx_kk_destroy.restype = None
    lib.rx_kk_batch_create.argtypes = [ctypes.POINTER(P), I, ctypes.POINTER(P)]
    lib.rx_kk_batch_push.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(SZ), ctypes.POINTER(P), ctypes.POINTER(SZ),
                                     ctypes.POINTER(SZ), P]
    lib.rx_kk_batch_destroy.argtypes = [P]
    lib.rx_kk_batch_destroy.restype = None
    lib.rx_kkrx_config_default.argtypes = [ctypes.POINTER(KKRxConfig)]
    lib.rx_kkrx_config_default.restype = None
    lib.rx_kkrx_create.argtypes = [ctypes.POINTER(KKRxConfig), ctypes.POINTER(P)]
    lib.rx_kkrx_push.argtypes = [P, P, SZ, I, P, SZ, ctypes.POINTER(SZ), P]
    lib.rx_kkrx_end.argtypes = [P, P, SZ, ctypes.POINTER(SZ), P]
    lib.rx_kkrx_equalised.argtypes = [P, I64, I64, ctypes.POINTER(ctypes.c_float)]
    lib.rx_kkrx_reset.argtypes = [P]
    lib.rx_kkrx_destroy.argtypes = [P]
    lib.rx_kkrx_destroy.restype = None
    lib.rx_kkrx_batch_create.argtypes = [ctypes.POINTER(P), I, ctypes.POINTER(P)]
    lib.rx_kkrx_batch_push.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(SZ), ctypes.POINTER(P), ctypes.POINTER(SZ),
                                       ctypes.POINTER(SZ), P]
    lib.rx_kkrx_batch_destroy.argtypes = [P]
    lib.rx_kkrx_batch_destroy.restype = None
    lib.rx_fp32_peak.argtypes = [I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.rx_batch_create.argtypes = [ctypes.POINTER(P), I, ctypes.POINTER(P)]
    lib.rx_batch_push.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(SZ), I, I, P]
    lib.rx_batch_info.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64),
                                  ctypes.POINTER(ctypes.c_double)]
    lib.rx_batch_destroy.argtypes = [P]
    lib.rx_batch_destroy.restype = None
    lib.rx_batch_set_graph.argtypes = [P, I]
    lib.rx_batch_graph_info.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64)]
    for name in ["rx_create", "rx_push_block", "rx_pull_bits", "rx_stats", "rx_destroy", "rx_reset",
                 "rx_join", "rx_stage_times", "rx_frame_trace", "rx_get_taps", "rx_get_equalised",
                 "rx_get_phase", "rx_decide_block_noalloc", "rx_server_create", "rx_server_open",
                 "rx_server_end", "rx_server_sync", "rx_server_pull_bits", "rx_server_stream_stats",
                 "rx_server_close", "rx_server_stats", "rx_server_destroy", "rx_autotune_fft",
                 "rx_kk_create", "rx_kk_push", "rx_kk_end", "rx_kk_reset", "rx_kk_position",
                 "rx_kk_batch_create", "rx_kk_batch_push",
                 "rx_kkrx_create", "rx_kkrx_push", "rx_kkrx_end", "rx_kkrx_equalised", "rx_kkrx_reset",
                 "rx_kkrx_batch_create", "rx_kkrx_batch_push", "rx_batch_create", "rx_batch_push",
                 "rx_batch_info", "rx_batch_set_graph", "rx_batch_graph_info", "rx_fp32_peak", "rx_autotune_tiles"]:
        getattr(lib, name).restype = I
    _lib = lib
    return lib


class RxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rx error {code}: {msg}")
        self.code = code


def _check(rc: int) -> int:
    if rc < 0:
        raise RxError(rc, load().rx_last_error().decode())
    return rc


def default_config(**overrides) -> RxConfig:
    cfg = RxConfig()
    load().rx_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


_DT = {np.dtype(np.complex128): RX_C128, np.dtype(np.complex64): RX_C64}


class Receiver:
    """One receiver stream (rx_create ... rx_destroy)."""

    def __init__(self, cfg: RxConfig | None = None, **overrides):
        self.lib = load()
        self.cfg = cfg if cfg is not None else default_config(**overrides)
        h = ctypes.c_void_p()
        _check(self.lib.rx_create(ctypes.byref(self.cfg), ctypes.byref(h)))
        self.h = h

    # -- pushing --
    def push_device(self, ptr: int, n_per_pol: int, dtype: int, stream: int = 0) -> None:
        """Push n_per_pol samples from device memory at ptr (planar [2][n])."""
        _check(self.lib.rx_push_block(self.h, ctypes.c_void_p(ptr), n_per_pol, dtype, 1, ctypes.c_void_p(stream)))

    def push_pinned(self, ptr: int, n_per_pol: int, dtype: int, stream: int = 0) -> None:
        """Push from page-locked host memory at ptr, copied to the device in
        stream order without a host wait (keep it unchanged until the stream
        has passed it)."""
        _check(self.lib.rx_push_block(self.h, ctypes.c_void_p(ptr), n_per_pol, dtype, 2, ctypes.c_void_p(stream)))

    def push_mapped(self, ptr: int, n_per_pol: int, dtype: int, stream: int = 0) -> None:
        """Push from page-locked host memory at ptr, read by the ingest
        kernel through the device mapping in stream order (no copy engine;
        keep it unchanged until the stream has passed it)."""
        _check(self.lib.rx_push_block(self.h, ctypes.c_void_p(ptr), n_per_pol, dtype, 3, ctypes.c_void_p(stream)))

    def push_host(self, x: np.ndarray, stream: int = 0) -> None:
        """Push a host array: complex [2, n] (c128/c64) or float16 [2, n, 2] (c16)."""
        if x.dtype == np.float16:
            dt = RX_C16
            n = x.shape[1]
        else:
            dt = _DT[x.dtype]
            n = x.shape[1]
        x = np.ascontiguousarray(x)
        _check(self.lib.rx_push_block(self.h, x.ctypes.data_as(ctypes.c_void_p), n, dt, 0, ctypes.c_void_p(stream)))

    def push_tensor(self, t, stream: int | None = None) -> None:
        """Push a CUDA tensor: complex [2, n] (complex128/complex64) or
        float16 [2, n, 2]."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        if t.dtype == torch.float16:
            dt, n = RX_C16, t.shape[1]
        elif t.dtype == torch.complex128:
            dt, n = RX_C128, t.shape[1]
        elif t.dtype == torch.complex64:
            dt, n = RX_C64, t.shape[1]
        else:
            raise TypeError(t.dtype)
        assert t.is_cuda and t.is_contiguous()
        self.push_device(t.data_ptr(), n, dt, stream)

    def end(self) -> None:
        _check(self.lib.rx_push_block(self.h, None, 0, RX_C64, 0, None))

    # -- results --
    def pull_bits(self, cap_bytes: int, timeout_ms: int = -1) -> np.ndarray:
        """Returns the decided bits as a uint8 array of 0/1 values."""
        buf = np.empty(max(cap_bytes, 1), dtype=np.uint8)
        nb = ctypes.c_size_t(0)
        rc = self.lib.rx_pull_bits(self.h, buf.ctypes.data_as(ctypes.c_void_p), cap_bytes, ctypes.byref(nb), timeout_ms)
        if rc not in (RX_OK, RX_ETIMEDOUT):
            _check(rc)
        n = nb.value
        return np.unpackbits(buf[:(n + 7) // 8])[:n]

    def pull_bytes(self, out: np.ndarray, timeout_ms: int = -1) -> int:
        nb = ctypes.c_size_t(0)
        rc = self.lib.rx_pull_bits(self.h, out.ctypes.data_as(ctypes.c_void_p), out.nbytes, ctypes.byref(nb), timeout_ms)
        if rc not in (RX_OK, RX_ETIMEDOUT):
            _check(rc)
        return nb.value

    def stats(self) -> dict:
        s = RxStats()
        _check(self.lib.rx_stats(self.h, ctypes.byref(s)))
        return s.as_dict()

    def stage_times(self) -> dict:
        ms = (ctypes.c_double * len(STAGES))()
        n = (ctypes.c_int64 * len(STAGES))()
        _check(self.lib.rx_stage_times(self.h, ms, n))
        return {STAGES[i]: (ms[i], n[i]) for i in range(len(STAGES))}

    def frame_trace(self, cap: int = 4096) -> np.ndarray:
        out = np.zeros(4 * cap, dtype=np.float64)
        n = _check(self.lib.rx_frame_trace(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), cap))
        return out[:4 * n].reshape(n, 4)

    def taps(self, which: int = -1) -> np.ndarray:
        T = self.cfg.mimo_taps
        out = np.zeros(8 * T, dtype=np.float32)
        _check(self.lib.rx_get_taps(self.h, which, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out.view(np.complex64).reshape(2, 2, T)

    def equalised(self, first: int, n: int) -> np.ndarray:
        out = np.zeros(4 * n, dtype=np.float32)
        _check(self.lib.rx_get_equalised(self.h, first, n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out.view(np.complex64).reshape(2, n)

    def phase(self, first: int, n: int):
        b = np.zeros(2 * n, dtype=np.uint8)
        m = np.zeros(2 * n, dtype=np.int32)
        _check(self.lib.rx_get_phase(self.h, first, n, b.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                     m.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        return b.reshape(2, n), m.reshape(2, n)

    def reset(self) -> None:
        _check(self.lib.rx_reset(self.h))

    def join(self, stream: int) -> None:
        _check(self.lib.rx_join(self.h, ctypes.c_void_p(stream)))

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.rx_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def default_server_config(**overrides) -> ServerConfig:
    cfg = ServerConfig()
    load().rx_server_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


class _Borrowed(Receiver):
    """A receiver owned by a server (inspection calls only; never destroyed here)."""

    def __init__(self, lib, h, cfg):
        self.lib, self.h, self.cfg = lib, h, cfg

    def close(self) -> None:
        self.h = None


class Batch:
    """Several receiver streams pushed together (rx_batch_*): one launch per
    stage and frame ordinal over every stream's frames; graph=True replays
    one captured CUDA graph per call instead (rx_batch_set_graph)."""

    def __init__(self, receivers: list, graph: bool = False):
        self.lib = load()
        self.receivers = list(receivers)
        n = len(self.receivers)
        arr = (ctypes.c_void_p * n)(*[r.h.value for r in self.receivers])
        b = ctypes.c_void_p()
        _check(self.lib.rx_batch_create(arr, n, ctypes.byref(b)))
        self.b = b
        if graph:
            try:
                _check(self.lib.rx_batch_set_graph(self.b, 1))
            except Exception:
                self.close()
                raise
        self._ptr = (ctypes.c_void_p * n)()
        self._n = (ctypes.c_size_t * n)()

    def push(self, ptrs, ns, dtype: int, stream: int = 0, on_device: int = 1) -> None:
        """Pointers (planar [2][n] each) and samples per polarisation per
        stream; n = 0 pushes nothing to that stream, ptr None with n = 0
        ends it."""
        for i in range(len(self.receivers)):
            self._ptr[i] = ptrs[i]
            self._n[i] = ns[i]
        _check(self.lib.rx_batch_push(self.b, self._ptr, self._n, dtype, on_device, ctypes.c_void_p(stream)))

    def end(self, stream: int = 0) -> None:
        """Ends every stream of the batch in one call."""
        self.push([None] * len(self.receivers), [0] * len(self.receivers), RX_C64, stream)

    def info(self) -> dict:
        c, l, f, w = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        _check(self.lib.rx_batch_info(self.b, ctypes.byref(c), ctypes.byref(l), ctypes.byref(f), ctypes.byref(w)))
        return {"calls": c.value, "launches": l.value, "frames": f.value, "wait_ms": w.value}

    def graph_info(self) -> dict:
        r, n = ctypes.c_int64(), ctypes.c_int64()
        _check(self.lib.rx_batch_graph_info(self.b, ctypes.byref(r), ctypes.byref(n)))
        return {"replays": r.value, "nodes": n.value}

    def close(self) -> None:
        if getattr(self, "b", None):
            self.lib.rx_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Many channel streams on one GPU (rx_server_*): a worker thread admits
    submitted capture blocks as each stream's receiver can take them."""

    def __init__(self, cfg: ServerConfig | None = None, **overrides):
        self.lib = load()
        self.cfg = cfg if cfg is not None else default_server_config(**overrides)
        s = ctypes.c_void_p()
        _check(self.lib.rx_server_create(ctypes.byref(self.cfg), ctypes.byref(s)))
        self.s = s
        self._cfgs = {}

    def open(self, cfg: RxConfig | None = None, **overrides) -> int:
        """Opens a stream; raises RxError (code RX_EAGAIN) when it does not fit."""
        cfg = cfg if cfg is not None else default_config(**overrides)
        sid = ctypes.c_int()
        _check(self.lib.rx_server_open(self.s, ctypes.byref(cfg), ctypes.byref(sid)))
        self._cfgs[sid.value] = cfg
        return sid.value

    def submit_device(self, sid: int, ptr: int, n_per_pol: int, dtype: int) -> int:
        return _check(self.lib.rx_server_submit(self.s, sid, ctypes.c_void_p(ptr), n_per_pol, dtype, 1))

    def submit_host(self, sid: int, x: np.ndarray) -> int:
        x = np.ascontiguousarray(x)
        dt = RX_C16 if x.dtype == np.float16 else _DT[x.dtype]
        return _check(self.lib.rx_server_submit(self.s, sid, x.ctypes.data_as(ctypes.c_void_p), x.shape[1], dt, 0))

    def end(self, sid: int) -> None:
        _check(self.lib.rx_server_end(self.s, sid))

    def sync(self, sid: int, timeout_ms: int = -1) -> None:
        _check(self.lib.rx_server_sync(self.s, sid, timeout_ms))

    def pull_bytes(self, sid: int, cap_bytes: int = 1 << 26) -> tuple[np.ndarray, int]:
        out = np.empty(cap_bytes, dtype=np.uint8)
        nb = ctypes.c_size_t()
        _check(self.lib.rx_server_pull_bits(self.s, sid, out.ctypes.data_as(ctypes.c_void_p), cap_bytes,
                                            ctypes.byref(nb)))
        return out[:(nb.value + 7) // 8].copy(), nb.value

    def stream_stats(self, sid: int) -> dict:
        st = RxStats()
        _check(self.lib.rx_server_stream_stats(self.s, sid, ctypes.byref(st)))
        return st.as_dict()

    def receiver(self, sid: int) -> Receiver:
        h = self.lib.rx_server_handle(self.s, sid)
        if not h:
            raise RxError(RX_EINVAL, "no such stream")
        return _Borrowed(self.lib, ctypes.c_void_p(h), self._cfgs[sid])

    def close_stream(self, sid: int) -> None:
        _check(self.lib.rx_server_close(self.s, sid))
        self._cfgs.pop(sid, None)

    def stats(self) -> dict:
        st = ServerStats()
        _check(self.lib.rx_server_stats(self.s, ctypes.byref(st)))
        return st.as_dict()

    def close(self) -> None:
        if getattr(self, "s", None):
            self.lib.rx_server_destroy(self.s)
            self.s = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fp32_peak(device: int = 0) -> tuple[float, float]:
    """Measured FP32 peak of the device in TFLOP/s: (fma.rn.f32 form,
    fma.rn.f32x2 form)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().rx_fp32_peak(device, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def autotune_fft(cfg: RxConfig | None = None, frames: int = 3, **overrides) -> tuple[int, float]:
    """The fastest overlap-save FFT size for cfg on this GPU and its time
    per 2^20 samples per polarisation (rx_autotune_fft)."""
    cfg = cfg if cfg is not None else default_config(**overrides)
    n = ctypes.c_int()
    ms = ctypes.c_double()
    _check(load().rx_autotune_fft(ctypes.byref(cfg), frames, ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def autotune_tiles(cfg: RxConfig | None = None, frames: int = 3, **overrides) -> dict:
    """FFT size and launch tiles for cfg on this GPU (rx_autotune_tiles)."""
    cfg = cfg if cfg is not None else default_config(**overrides)
    n, mw, br = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ms = ctypes.c_double()
    _check(load().rx_autotune_tiles(ctypes.byref(cfg), frames, ctypes.byref(n), ctypes.byref(mw), ctypes.byref(br),
                                    ctypes.byref(ms)))
    return {"fft_n": n.value, "mimo_block_warps": mw.value, "bps_block_runs": br.value, "ms_per_msample": ms.value}


def default_kk_config(**overrides) -> KKConfig:
    cfg = KKConfig()
    load().rx_kk_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


class KKFrontEnd:
    """Kramers-Kronig front end (rx_kk_create ... rx_kk_destroy): int16 ADC
    codes in, the downshifted complex64 field out, both in device memory."""

    def __init__(self, cfg: KKConfig | None = None, **overrides):
        self.lib = load()
        self.cfg = cfg if cfg is not None else default_kk_config(**overrides)
        h = ctypes.c_void_p()
        _check(self.lib.rx_kk_create(ctypes.byref(self.cfg), ctypes.byref(h)))
        self.h = h

    def push_device(self, codes_ptr: int, n: int, out_ptr: int, out_cap: int, stream: int = 0) -> int:
        """Codes at a device pointer; returns the field samples written at out_ptr."""
        n_out = ctypes.c_size_t()
        _check(self.lib.rx_kk_push(self.h, ctypes.c_void_p(codes_ptr), n, 1, ctypes.c_void_p(out_ptr), out_cap,
                                   ctypes.byref(n_out), ctypes.c_void_p(stream)))
        return n_out.value

    def push_host(self, codes: np.ndarray, out_ptr: int, out_cap: int, stream: int = 0) -> int:
        """Codes from a host int16 array (copied in stream order)."""
        codes = np.ascontiguousarray(codes, dtype=np.int16)
        n_out = ctypes.c_size_t()
        _check(self.lib.rx_kk_push(self.h, codes.ctypes.data_as(ctypes.c_void_p), codes.size, 0,
                                   ctypes.c_void_p(out_ptr), out_cap, ctypes.byref(n_out), ctypes.c_void_p(stream)))
        return n_out.value

    def push_tensor(self, codes, out, stream: int | None = None) -> int:
        """codes: int16 CUDA tensor; out: complex64 CUDA tensor with room for the
        samples this push completes.  Returns how many were written to out[:n]."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        assert codes.is_cuda and codes.dtype == torch.int16 and codes.is_contiguous()
        assert out.is_cuda and out.dtype == torch.complex64 and out.is_contiguous()
        return self.push_device(codes.data_ptr(), codes.numel(), out.data_ptr(), out.numel(), stream)

    def end_tensor(self, out, stream: int | None = None) -> int:
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        assert out.is_cuda and out.dtype == torch.complex64 and out.is_contiguous()
        return self.end(out.data_ptr(), out.numel(), stream)

    def end(self, out_ptr: int, out_cap: int, stream: int = 0) -> int:
        n_out = ctypes.c_size_t()
        _check(self.lib.rx_kk_end(self.h, ctypes.c_void_p(out_ptr), out_cap, ctypes.byref(n_out),
                                  ctypes.c_void_p(stream)))
        return n_out.value

    def reset(self) -> None:
        _check(self.lib.rx_kk_reset(self.h))

    def position(self) -> tuple[int, int]:
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(self.lib.rx_kk_position(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.rx_kk_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class KKBatch:
    """Several KK front ends pushed together (rx_kk_batch_*): one graph
    replay per batch push, whatever the channels' push lengths."""

    def __init__(self, channels: list):
        self.lib = load()
        self.channels = list(channels)
        n = len(self.channels)
        arr = (ctypes.c_void_p * n)(*[c.h.value for c in self.channels])
        b = ctypes.c_void_p()
        _check(self.lib.rx_kk_batch_create(arr, n, ctypes.byref(b)))
        self.b = b
        self._codes = (ctypes.c_void_p * n)()
        self._n = (ctypes.c_size_t * n)()
        self._out = (ctypes.c_void_p * n)()
        self._cap = (ctypes.c_size_t * n)()
        self._nout = (ctypes.c_size_t * n)()

    def push(self, codes_ptrs, ns, out_ptrs, out_caps, stream: int = 0) -> list[int]:
        """Device pointers and lengths per channel (n = 0: nothing for that
        channel); returns the field samples written per channel."""
        for i in range(len(self.channels)):
            self._codes[i] = codes_ptrs[i]
            self._n[i] = ns[i]
            self._out[i] = out_ptrs[i]
            self._cap[i] = out_caps[i]
        _check(self.lib.rx_kk_batch_push(self.b, self._codes, self._n, self._out, self._cap, self._nout,
                                         ctypes.c_void_p(stream)))
        return list(self._nout)

    def close(self) -> None:
        if getattr(self, "b", None):
            self.lib.rx_kk_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def default_kkrx_config(fe: dict | None = None, **overrides) -> KKRxConfig:
    """Chain defaults with overrides; fe holds front-end fields (fs_hz, ...)."""
    cfg = KKRxConfig()
    load().rx_kkrx_config_default(ctypes.byref(cfg))
    for k, v in (fe or {}).items():
        if not hasattr(cfg.fe, k):
            raise KeyError(k)
        setattr(cfg.fe, k, v)
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


class KKReceiver:
    """The paper's KK receiver chain (rx_kkrx_*): int16 ADC codes in, packed
    decided bits out, both in device memory."""

    def __init__(self, cfg: KKRxConfig | None = None, fe: dict | None = None, **overrides):
        self.lib = load()
        self.cfg = cfg if cfg is not None else default_kkrx_config(fe, **overrides)
        h = ctypes.c_void_p()
        _check(self.lib.rx_kkrx_create(ctypes.byref(self.cfg), ctypes.byref(h)))
        self.h = h

    def push_device(self, codes_ptr: int, n: int, bits_ptr: int, bits_cap: int, stream: int = 0) -> int:
        """Returns the number of bits written at bits_ptr."""
        nb = ctypes.c_size_t()
        _check(self.lib.rx_kkrx_push(self.h, ctypes.c_void_p(codes_ptr), n, 1, ctypes.c_void_p(bits_ptr), bits_cap,
                                     ctypes.byref(nb), ctypes.c_void_p(stream)))
        return nb.value

    def push_host(self, codes: np.ndarray, bits_ptr: int, bits_cap: int, stream: int = 0) -> int:
        codes = np.ascontiguousarray(codes, dtype=np.int16)
        nb = ctypes.c_size_t()
        _check(self.lib.rx_kkrx_push(self.h, codes.ctypes.data_as(ctypes.c_void_p), codes.size, 0,
                                     ctypes.c_void_p(bits_ptr), bits_cap, ctypes.byref(nb), ctypes.c_void_p(stream)))
        return nb.value

    def end(self, bits_ptr: int, bits_cap: int, stream: int = 0) -> int:
        nb = ctypes.c_size_t()
        _check(self.lib.rx_kkrx_end(self.h, ctypes.c_void_p(bits_ptr), bits_cap, ctypes.byref(nb),
                                    ctypes.c_void_p(stream)))
        return nb.value

    def equalised(self, first: int, n: int) -> np.ndarray:
        out = np.zeros(2 * n, dtype=np.float32)
        _check(self.lib.rx_kkrx_equalised(self.h, first, n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out.view(np.complex64)

    def reset(self) -> None:
        _check(self.lib.rx_kkrx_reset(self.h))

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.rx_kkrx_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class KKReceiverBatch:
    """Several KK receivers pushed together (rx_kkrx_batch_*); their streams
    end with each receiver's own end()."""

    def __init__(self, receivers: list):
        self.lib = load()
        self.receivers = list(receivers)
        n = len(self.receivers)
        arr = (ctypes.c_void_p * n)(*[r.h.value for r in self.receivers])
        b = ctypes.c_void_p()
        _check(self.lib.rx_kkrx_batch_create(arr, n, ctypes.byref(b)))
        self.b = b
        self._codes = (ctypes.c_void_p * n)()
        self._n = (ctypes.c_size_t * n)()
        self._bits = (ctypes.c_void_p * n)()
        self._cap = (ctypes.c_size_t * n)()
        self._nb = (ctypes.c_size_t * n)()

    def push(self, codes_ptrs, ns, bits_ptrs, bits_caps, stream: int = 0) -> list[int]:
        """Device pointers and lengths per channel; returns the bits written per channel."""
        for i in range(len(self.receivers)):
            self._codes[i] = codes_ptrs[i]
            self._n[i] = ns[i]
            self._bits[i] = bits_ptrs[i]
            self._cap[i] = bits_caps[i]
        _check(self.lib.rx_kkrx_batch_push(self.b, self._codes, self._n, self._bits, self._cap, self._nb,
                                           ctypes.c_void_p(stream)))
        return list(self._nb)

    def close(self) -> None:
        if getattr(self, "b", None):
            self.lib.rx_kkrx_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
