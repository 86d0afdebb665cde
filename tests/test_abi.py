"""The C-ABI library: builds, loads, exports every declared entry point,
struct layouts agree between C and the binding, and argument checks work
without a GPU (no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rx.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2108_07001_gb300 import build, rx
    build.build()
    return rx.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rx_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2108_07001_gb300 import rx
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(rx.EXPORTS) == names


def test_struct_layout_matches_c(tmp_path, lib):
    from paper_2108_07001_gb300 import rx
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "rx.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(rx_config), sizeof(rx_stats_t),"
        " offsetof(rx_config, prbs_seed), offsetof(rx_config, device), offsetof(rx_stats_t, fo_hz),"
        " offsetof(rx_config, history_syms)); return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == [ctypes.sizeof(rx.RxConfig), ctypes.sizeof(rx.RxStats), rx.RxConfig.prbs_seed.offset,
                    rx.RxConfig.device.offset, rx.RxStats.fo_hz.offset, rx.RxConfig.history_syms.offset]


def test_defaults(lib):
    from paper_2108_07001_gb300 import rx
    c = rx.default_config()
    assert c.baud_hz == 28e9 and c.modulation == rx.RX_QPSK and c.mimo_taps == 15
    assert c.bps_angles == 64 and c.bps_half_window == 16 and c.sub_block_syms == 64
    assert c.bps_coarse_stride == 1
    assert c.frame_syms == 65536 and c.seg_syms == 512 and c.storage_dtype == rx.RX_C64


@pytest.mark.parametrize("field,value,msg", [
    ("mimo_taps", 16, "mimo_taps"),
    ("mimo_taps", 33, "mimo_taps"),
    ("bps_angles", 48, "bps_angles"),
    ("bps_half_window", 5, "bps_half_window"),
    ("bps_coarse_stride", 2, "bps_coarse_stride"),   # QPSK with 64 angles: 1 or 4
    ("bps_coarse_stride", 8, "bps_coarse_stride"),
    ("sub_block_syms", 32, "sub_block_syms"),
    ("seg_syms", 100, "seg_syms"),
    ("frame_syms", 1000, "frame_syms"),
    ("acq_syms", 1 << 20, "acq_syms"),
    ("storage_dtype", 0, "storage_dtype"),
    ("modulation", 3, "modulation"),
    ("baud_hz", 0.0, "baud_hz"),
    ("fft_n", 3000, "fft_n"),
    ("fft_n", 1024, "halo"),
    ("mimo_block_warps", 3, "mimo_block_warps"),
    ("bps_block_runs", 2, "bps_block_runs"),
])
def test_invalid_config_is_rejected(lib, field, value, msg):
    from paper_2108_07001_gb300 import rx
    kw = {field: value}
    if msg == "halo":
        kw["fiber_len_m"] = 10000e3
    c = rx.default_config(**kw)
    h = ctypes.c_void_p()
    rc = lib.rx_create(ctypes.byref(c), ctypes.byref(h))
    assert rc == rx.RX_EINVAL
    assert msg in lib.rx_last_error().decode()
    assert not h.value


def test_ber_frame_rule(lib):
    from paper_2108_07001_gb300 import rx
    c = rx.default_config(prbs_seed=5, frame_syms=4096, acq_syms=2048, cma_syms=1024)
    h = ctypes.c_void_p()
    assert lib.rx_create(ctypes.byref(c), ctypes.byref(h)) == rx.RX_EINVAL
    assert "sync" in lib.rx_last_error().decode()


def test_null_arguments(lib):
    from paper_2108_07001_gb300 import rx
    assert lib.rx_create(None, None) == rx.RX_EINVAL
    assert lib.rx_push_block(None, None, 0, 1, 0, None) == rx.RX_EINVAL
    assert lib.rx_stats(None, None) == rx.RX_EINVAL
    assert lib.rx_destroy(None) == rx.RX_OK


def test_valid_config_without_device(lib):
    import torch
    from paper_2108_07001_gb300 import rx
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    c = rx.default_config()
    h = ctypes.c_void_p()
    assert lib.rx_create(ctypes.byref(c), ctypes.byref(h)) == rx.RX_EDEVICE


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2108_07001_gb300 import rx
    old = rx._lib
    rx._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            rx.load(str(tmp_path / "missing.so"))
    finally:
        rx._lib = old


def test_server_struct_layout_matches_c(tmp_path, lib):
    from paper_2108_07001_gb300 import rx
    src = tmp_path / "slayout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "rx.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu\\n\", sizeof(rx_server_config), sizeof(rx_server_stats_t),"
        " offsetof(rx_server_config, workers), offsetof(rx_server_stats_t, latency_p99_ms),"
        " offsetof(rx_server_stats_t, worker_error)); return 0;}\n")
    exe = tmp_path / "slayout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == [ctypes.sizeof(rx.ServerConfig), ctypes.sizeof(rx.ServerStats), rx.ServerConfig.workers.offset,
                    rx.ServerStats.latency_p99_ms.offset, rx.ServerStats.worker_error.offset]


def test_server_config_checks_without_device(lib):
    from paper_2108_07001_gb300 import rx
    c = rx.default_server_config()
    assert c.max_streams == 64 and c.bits_cap_bytes == 64 << 20 and c.mem_budget_bytes == 0 and c.workers == 4
    s = ctypes.c_void_p()
    bad = rx.default_server_config(max_streams=0)
    assert lib.rx_server_create(ctypes.byref(bad), ctypes.byref(s)) == rx.RX_EINVAL
    assert b"max_streams" in lib.rx_last_error()
    bad = rx.default_server_config(bits_cap_bytes=100)
    assert lib.rx_server_create(ctypes.byref(bad), ctypes.byref(s)) == rx.RX_EINVAL
    bad = rx.default_server_config(workers=0)
    assert lib.rx_server_create(ctypes.byref(bad), ctypes.byref(s)) == rx.RX_EINVAL
    for b in (-1, 3):
        bad = rx.default_server_config(batch=b)
        assert lib.rx_server_create(ctypes.byref(bad), ctypes.byref(s)) == rx.RX_EINVAL
        assert b"batch" in lib.rx_last_error()
    bad = rx.default_server_config(batch=2, max_streams=257)
    assert lib.rx_server_create(ctypes.byref(bad), ctypes.byref(s)) == rx.RX_EINVAL
    # no GPU in this container: a valid config stops at the device check
    rc = lib.rx_server_create(ctypes.byref(rx.default_server_config()), ctypes.byref(s))
    assert rc in (rx.RX_OK, rx.RX_EDEVICE)
    if rc == rx.RX_OK:
        lib.rx_server_destroy(s)
    assert lib.rx_server_submit(None, 0, None, 0, rx.RX_C64, 1) == rx.RX_EINVAL
    assert lib.rx_server_stats(None, None) == rx.RX_EINVAL


def test_autotune_argument_checks_without_device(lib):
    from paper_2108_07001_gb300 import rx
    n, ms = ctypes.c_int(), ctypes.c_double()
    cfg = rx.default_config()
    assert lib.rx_autotune_fft(None, 3, ctypes.byref(n), None) == rx.RX_EINVAL
    assert lib.rx_autotune_fft(ctypes.byref(cfg), 0, ctypes.byref(n), None) == rx.RX_EINVAL
    far = rx.default_config(fiber_len_m=200000e3)  # halo (~50k samples) longer than any FFT size
    assert lib.rx_autotune_fft(ctypes.byref(far), 3, ctypes.byref(n), None) == rx.RX_EINVAL
    assert b"halo" in lib.rx_last_error()
    mw, br = ctypes.c_int(), ctypes.c_int()
    assert lib.rx_autotune_tiles(ctypes.byref(cfg), 3, ctypes.byref(n), None, ctypes.byref(br), None) == rx.RX_EINVAL
    assert lib.rx_autotune_tiles(ctypes.byref(cfg), 65, ctypes.byref(n), ctypes.byref(mw), ctypes.byref(br),
                                 None) == rx.RX_EINVAL
    assert lib.rx_autotune_tiles(ctypes.byref(far), 3, ctypes.byref(n), ctypes.byref(mw), ctypes.byref(br),
                                 None) == rx.RX_EINVAL


def test_kk_struct_layout_matches_c(tmp_path, lib):
    from paper_2108_07001_gb300 import rx
    src = tmp_path / "klayout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "rx.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu\\n\", sizeof(rx_kk_config), offsetof(rx_kk_config, fft_n),"
        " offsetof(rx_kk_config, max_block_samples), offsetof(rx_kk_config, device)); return 0;}\n")
    exe = tmp_path / "klayout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == [ctypes.sizeof(rx.KKConfig), rx.KKConfig.fft_n.offset, rx.KKConfig.max_block_samples.offset,
                    rx.KKConfig.device.offset]


@pytest.mark.parametrize("field,value,msg", [
    ("fft_n", 512, "fft_n"),
    ("fft_n", 3000, "fft_n"),
    ("fs_hz", 0.0, "fs_hz"),
    ("adc_gain", -1.0, "adc_gain"),
    ("max_block_samples", 0, "max_block_samples"),
])
def test_kk_config_checks_without_device(lib, field, value, msg):
    from paper_2108_07001_gb300 import rx
    c = rx.default_kk_config()
    assert (c.fs_hz, c.f_shift_hz, c.fft_n, c.max_block_samples) == (4e9, 0.516e9, 1024, 1 << 22)
    bad = rx.default_kk_config(**{field: value})
    h = ctypes.c_void_p()
    assert lib.rx_kk_create(ctypes.byref(bad), ctypes.byref(h)) == rx.RX_EINVAL
    assert msg in lib.rx_last_error().decode()
    assert not h.value
    n = ctypes.c_size_t()
    assert lib.rx_kk_push(None, None, 0, 1, None, 0, ctypes.byref(n), None) == rx.RX_EINVAL
    assert lib.rx_kk_end(None, None, 0, ctypes.byref(n), None) == rx.RX_EINVAL


def test_kkrx_struct_layout_matches_c(tmp_path, lib):
    from paper_2108_07001_gb300 import rx
    src = tmp_path / "krlayout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "rx.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu\\n\", sizeof(rx_kkrx_config), offsetof(rx_kkrx_config, baud_hz),"
        " offsetof(rx_kkrx_config, mu), offsetof(rx_kkrx_config, acq_syms), offsetof(rx_kkrx_config, history_syms));"
        " return 0;}\n")
    exe = tmp_path / "krlayout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == [ctypes.sizeof(rx.KKRxConfig), rx.KKRxConfig.baud_hz.offset, rx.KKRxConfig.mu.offset,
                    rx.KKRxConfig.acq_syms.offset, rx.KKRxConfig.history_syms.offset]


@pytest.mark.parametrize("fe,kw,msg", [
    ({"fs_hz": 3e9}, {}, "fs_hz"),
    ({}, {"modulation": 3}, "modulation"),
    ({}, {"eq_fft_n": 4096}, "eq_fft_n"),
    ({}, {"seg_syms": 100}, "seg_syms"),
    ({}, {"frame_syms": 1000}, "frame_syms"),
    ({}, {"acq_syms": 1 << 21}, "acq_syms"),
    ({}, {"mu": 0.0}, "mu"),
    ({"fft_n": 512}, {}, "fft_n"),
])
def test_kkrx_config_checks_without_device(lib, fe, kw, msg):
    from paper_2108_07001_gb300 import rx
    c = rx.default_kkrx_config()
    assert (c.baud_hz, c.fe.fs_hz, c.frame_syms, c.seg_syms, c.eq_fft_n) == (1e9, 4e9, 1 << 20, 512, 1024)
    bad = rx.default_kkrx_config(fe, **kw)
    h = ctypes.c_void_p()
    assert lib.rx_kkrx_create(ctypes.byref(bad), ctypes.byref(h)) == rx.RX_EINVAL
    assert msg in lib.rx_last_error().decode()
    assert not h.value


def test_smoke_configuration_is_valid(lib):
    """The receiver settings smoke() runs pass validation (on a machine
    without a GPU rx_create then stops at the device)."""
    import importlib.util
    import torch
    from paper_2108_07001_gb300 import rx
    spec = importlib.util.spec_from_file_location("graft_entry", os.path.join(ROOT, "__graft_entry__.py"))
    ge = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(ge)
    c = rx.default_config(**ge.SMOKE_RX, history_syms=1 << 14)
    h = ctypes.c_void_p()
    rc = lib.rx_create(ctypes.byref(c), ctypes.byref(h))
    if torch.cuda.is_available():
        assert rc == rx.RX_OK, lib.rx_last_error()
        lib.rx_destroy(h)
    else:
        assert rc == rx.RX_EDEVICE, lib.rx_last_error()


def test_kk_batch_argument_checks_without_device(lib):
    from paper_2108_07001_gb300 import rx
    b = ctypes.c_void_p()
    assert lib.rx_kk_batch_create(None, 1, ctypes.byref(b)) == rx.RX_EINVAL
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.rx_kk_batch_create(arr, 0, ctypes.byref(b)) == rx.RX_EINVAL
    assert lib.rx_kk_batch_create(arr, 1, ctypes.byref(b)) == rx.RX_EINVAL  # null channel
    assert lib.rx_kk_batch_create(arr, 257, ctypes.byref(b)) == rx.RX_EINVAL
    assert lib.rx_kk_batch_push(None, None, None, None, None, None, None) == rx.RX_EINVAL


def test_kkrx_batch_argument_checks_without_device(lib):
    from paper_2108_07001_gb300 import rx
    b = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.rx_kkrx_batch_create(None, 1, ctypes.byref(b)) == rx.RX_EINVAL
    assert lib.rx_kkrx_batch_create(arr, 0, ctypes.byref(b)) == rx.RX_EINVAL
    assert lib.rx_kkrx_batch_create(arr, 1, ctypes.byref(b)) == rx.RX_EINVAL
    assert lib.rx_kkrx_batch_create(arr, 257, ctypes.byref(b)) == rx.RX_EINVAL
    assert lib.rx_kkrx_batch_push(None, None, None, None, None, None, None) == rx.RX_EINVAL


def test_batch_argument_checks_without_device(lib):
    from paper_2108_07001_gb300 import rx
    b = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.rx_batch_create(None, 1, ctypes.byref(b)) == rx.RX_EINVAL
    assert lib.rx_batch_create(arr, 0, ctypes.byref(b)) == rx.RX_EINVAL
    assert lib.rx_batch_create(arr, 1, ctypes.byref(b)) == rx.RX_EINVAL  # null stream
    assert lib.rx_batch_create(arr, 257, ctypes.byref(b)) == rx.RX_EINVAL
    assert lib.rx_batch_push(None, None, None, rx.RX_C64, 1, None) == rx.RX_EINVAL
    assert lib.rx_batch_info(None, None, None, None, None) == rx.RX_EINVAL
    assert lib.rx_batch_set_graph(None, 1) == rx.RX_EINVAL
    assert lib.rx_batch_graph_info(None, None, None) == rx.RX_EINVAL
    lib.rx_batch_destroy(None)  # no-op


def test_fp32_peak_argument_checks_without_device(lib):
    from paper_2108_07001_gb300 import rx
    assert lib.rx_fp32_peak(0, None, None) == rx.RX_EINVAL
