"""The C ABI without a GPU: the library builds and loads, exports every
symbol include/lem.h declares, the binding covers them, and host-side
argument checks answer before any device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    with open(os.path.join(ROOT, "include", header)) as f:
        src = f.read()
    return sorted(set(re.findall(r"^LEM_API\s+[\w\s\*]+?\b(lem_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1803_02977_gb300 import lem
    return lem.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared("lem.h")
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_1803_02977_gb300 import lem
    bound = sorted(n for n, _, _ in lem.SIGNATURES)
    assert bound == _declared("lem.h")


def test_status_strings(lib):
    from paper_1803_02977_gb300 import lem
    for code in (lem.LEM_OK, lem.LEM_EINVAL, lem.LEM_ENOMEM, lem.LEM_ECUDA, lem.LEM_ETIMEOUT,
                 lem.LEM_ESTATE, lem.LEM_EOVERFLOW, lem.LEM_EBOUNDS):
        s = lib.lem_status_string(code).decode()
        assert s and s != "unknown status"


@pytest.mark.parametrize("nx,ny,dx,K,dt,want", [
    (2, 10, 100.0, 1e-5, 1000.0, -1),          # too narrow
    (10, 2, 100.0, 1e-5, 1000.0, -1),
    (10, 10, 0.0, 1e-5, 1000.0, -1),           # dx <= 0
    (10, 10, 100.0, -1.0, 1000.0, -1),         # K < 0
    (10, 10, 100.0, 1e-5, 0.0, -1),            # dt <= 0
    (10, 10, float("nan"), 1e-5, 1000.0, -1),
    (65536, 65536, 100.0, 1e-5, 1000.0, -6),   # 2^32 cells: 32-bit addresses overflow
])
def test_create_rejects_bad_arguments_on_host(lib, nx, ny, dx, K, dt, want):
    h = ctypes.c_void_p(1)
    rc = lib.lem_create(ctypes.byref(h), nx, ny, dx, K, 0.5, 1e-3, dt)
    assert rc == want
    assert h.value is None


def test_null_context_calls_are_rejected(lib):
    assert lib.lem_step(None, 1) == -1
    assert lib.lem_receivers(None, None) == -1
    assert lib.lem_sync(None) == -1
    lib.lem_destroy(None)


def test_algorithmic_bytes_match_the_roofline_table():
    import bench
    assert sum(bench.algo_bytes(8, 4).values()) == 66   # FP64 elevations, int32 counts
    assert sum(bench.algo_bytes(4, 4).values()) == 50   # FP32, int32
    assert sum(bench.algo_bytes(4, 8).values()) == 62   # FP32, int64


def test_new_entry_points_reject_null_context_without_device_work(lib):
    # answered on the host: no context, so no device memory is touched
    from paper_1803_02977_gb300 import lem
    c_d, c_i, c_vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
    assert lib.lem_set_slope_exponent(None, c_d(2.0), c_d(1e-12), c_i(10)) == lem.LEM_EINVAL
    assert lib.lem_fill(None) == lem.LEM_EINVAL
    assert lib.lem_set_fill(None, c_i(1)) == lem.LEM_EINVAL
    stats = (ctypes.c_int64 * 4)()
    assert lib.lem_fill_stats(None, stats) == lem.LEM_EINVAL
    assert lib.lem_accumulate_mfd(None, c_d(1.0), None, c_vp(0), None) == lem.LEM_EINVAL


def test_graph_state_and_jump_entry_points_reject_null_context(lib):
    from paper_1803_02977_gb300 import lem
    n = ctypes.c_int64(0)
    stats = (ctypes.c_int64 * 2)()
    assert lib.lem_last_graph(None, None, None) == lem.LEM_EINVAL
    assert lib.lem_state_size(None, ctypes.byref(n)) == lem.LEM_EINVAL
    assert lib.lem_get_state(None, ctypes.c_void_p(0), ctypes.c_int64(0)) == lem.LEM_EINVAL
    assert lib.lem_set_state(None, ctypes.c_void_p(0), ctypes.c_int64(0)) == lem.LEM_EINVAL
    assert lib.lem_jump_stats(None, stats) == lem.LEM_EINVAL


def test_debug_library_builds_and_exports_the_same_symbols():
    from paper_1803_02977_gb300 import build, lem
    path = build.build(debug=True)
    L = ctypes.CDLL(path)
    for n in _declared("lem.h"):
        assert hasattr(L, n), n
    assert L.lem_step(None, 1) == lem.LEM_EINVAL
