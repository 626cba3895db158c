"""ctypes binding of liblem.so (include/lem.h), one function per C entry point.

Argument marshalling only: torch tensors supply device memory and the CUDA
stream, every computation runs in the library's CUDA kernels.  There is no
CPU fallback: if the compiled library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

LEM_OK, LEM_EINVAL, LEM_ENOMEM, LEM_ECUDA, LEM_ETIMEOUT, LEM_ESTATE, LEM_EOVERFLOW = \
    0, -1, -2, -3, -4, -5, -6
LEM_EBOUNDS = -7
LEM_F64, LEM_F32 = 0, 1

_lib = None


class _nvtx:
    """An NVTX range around a host call, so that a profiler's timeline names
    each stage and step; a no-op where NVTX is unavailable (markers only: a
    call never fails over them)."""

    def __init__(self, name):
        self.name = name
        self.pushed = False

    def __enter__(self):
        try:
            torch.cuda.nvtx.range_push(self.name)
            self.pushed = True
        except Exception:  # noqa: BLE001
            pass
        return self

    def __exit__(self, *exc):
        if self.pushed:
            try:
                torch.cuda.nvtx.range_pop()
            except Exception:  # noqa: BLE001
                pass
        return False


class LemError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = lib().lem_status_string(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")


class lem_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("dx", ctypes.c_double),
                ("K", ctypes.c_double), ("m", ctypes.c_double), ("U", ctypes.c_double),
                ("dt", ctypes.c_double), ("area_scale", ctypes.c_double),
                ("dtype", ctypes.c_int), ("count_bits", ctypes.c_int)]


# (name, restype, argtypes) of every entry point declared in include/lem.h
_VP, _I, _D, _I64P = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int64)
SIGNATURES = [
    ("lem_create", _I, [ctypes.POINTER(_VP), _I, _I, _D, _D, _D, _D, _D]),
    ("lem_create_ex", _I, [ctypes.POINTER(_VP), ctypes.POINTER(lem_params)]),
    ("lem_destroy", None, [_VP]),
    ("lem_set_stream", _I, [_VP, _VP]),
    ("lem_bind_elevation", _I, [_VP, _VP, _I]),
    ("lem_set_uplift_field", _I, [_VP, _VP]),
    ("lem_receivers", _I, [_VP, _VP]),
    ("lem_donors", _I, [_VP, _VP, _VP]),
    ("lem_levels", _I, [_VP, _I64P, _VP, _VP, _VP]),
    ("lem_accumulate", _I, [_VP, _VP]),
    ("lem_erode", _I, [_VP]),
    ("lem_step", _I, [_VP, _I]),
    ("lem_set_slope_exponent", _I, [_VP, _D, _D, _I]),
    ("lem_accumulate_mfd", _I, [_VP, _D, _VP, _VP, _I64P]),
    ("lem_fill", _I, [_VP]),
    ("lem_set_fill", _I, [_VP, _I]),
    ("lem_fill_stats", _I, [_VP, _I64P]),
    ("lem_set_receivers", _I, [_VP, _VP]),
    ("lem_last_graph", _I, [_VP, _VP, _VP]),
    ("lem_state_size", _I, [_VP, _I64P]),
    ("lem_get_state", _I, [_VP, _VP, ctypes.c_int64]),
    ("lem_set_state", _I, [_VP, _VP, ctypes.c_int64]),
    ("lem_sync", _I, [_VP]),
    ("lem_set_wait_limit", _I, [_VP, _D]),
    ("lem_selftest_wait", _I, [_VP]),
    ("lem_set_step_mode", _I, [_VP, _I]),
    ("lem_set_tiling", _I, [_VP, _I, _I]),
    ("lem_get_tiling", _I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    ("lem_step_stats", _I, [_VP, _I64P, _I64P]),
    ("lem_tier_stats", _I, [_VP, _I64P]),
    ("lem_jump_stats", _I, [_VP, _I64P]),
    ("lem_trace_enable", _I, [_VP, _I]),
    ("lem_trace_read", _I, [_VP, _VP, _VP, _I, ctypes.POINTER(_I)]),
    ("lem_adjoint", _I, [_VP, _VP, _VP, _I, _I, _VP, ctypes.POINTER(_D), _VP]),
    ("lem_batch_create", _I, [ctypes.POINTER(_VP), _I, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _I]),
    ("lem_batch_destroy", None, [_VP]),
    ("lem_batch_offsets", _I, [_VP, _VP]),
    ("lem_batch_set_stream", _I, [_VP, _VP]),
    ("lem_batch_bind_elevation", _I, [_VP, _VP]),
    ("lem_batch_set_config", _I, [_VP, _I, _I]),
    ("lem_batch_step", _I, [_VP, _I]),
    ("lem_batch_sync", _I, [_VP]),
    ("lem_step_noalloc", _I, [_I, _I, _VP, _D, _D, _D, _D, _D, _I, _VP]),
    ("lem_status_string", ctypes.c_char_p, [_I]),
]

LEM_NOALLOC_MAX_CELLS = 1 << 18

TRACE_PHASES = {1: "start", 2: "receivers", 3: "level0", 4: "bfs_wide", 5: "bfs_narrow",
                6: "acc_wide", 7: "acc_narrow", 8: "uplift", 9: "erode_wide",
                10: "erode_narrow", 11: "private_levels", 12: "private_accumulate",
                13: "private_erode", 14: "step_end", 15: "block0_done", 16: "tiles_end",
                17: "jump_tour", 18: "jump_rank", 19: "jump_init", 20: "jump_erode",
                21: "block_end"}


def _load(path):
    L = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def lib(build_if_missing: bool = True):
    """Load liblem.so (building it in-tree first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.LIB_PATH
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise ImportError(f"liblem.so is not built ({path}); run __graft_entry__.build()")
        _lib = _load(path)
    return _lib


class use_debug_library:
    """Within this context every call of the binding goes to liblem_debug.so,
    the build whose kernels check their indices (LEM_EBOUNDS on a failed
    check, never a trap); contexts must be created and used inside it."""

    def __enter__(self):
        global _lib
        path = _build.build(debug=True)
        self.saved = _lib
        _lib = _load(path)
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _check(status, where):
    if status != LEM_OK:
        raise LemError(status, where)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


# ---- one Python function per C entry point --------------------------------

def lem_create(nx, ny, dx, K, m, U, dt):
    h = _VP()
    _check(lib().lem_create(ctypes.byref(h), nx, ny, dx, K, m, U, dt), "lem_create")
    return h


def lem_create_ex(nx, ny, dx, K, m, U, dt, area_scale=0.0, dtype=LEM_F64, count_bits=32):
    p = lem_params(nx, ny, dx, K, m, U, dt, area_scale, dtype, count_bits)
    h = _VP()
    _check(lib().lem_create_ex(ctypes.byref(h), ctypes.byref(p)), "lem_create_ex")
    return h


def lem_destroy(ctx):
    lib().lem_destroy(ctx)


def lem_set_stream(ctx, stream=None):
    s = (stream or torch.cuda.current_stream()).cuda_stream
    _check(lib().lem_set_stream(ctx, ctypes.c_void_p(s)), "lem_set_stream")


def lem_bind_elevation(ctx, h, dtype):
    _check(lib().lem_bind_elevation(ctx, _ptr(h), dtype), "lem_bind_elevation")


def lem_set_uplift_field(ctx, U):
    _check(lib().lem_set_uplift_field(ctx, _ptr(U)), "lem_set_uplift_field")


def lem_receivers(ctx, rec=None):
    _check(lib().lem_receivers(ctx, _ptr(rec)), "lem_receivers")


def lem_donors(ctx, dnum=None, donor=None):
    _check(lib().lem_donors(ctx, _ptr(dnum), _ptr(donor)), "lem_donors")


def lem_levels(ctx, queue=None, levels=None, depth=None):
    L = ctypes.c_int64(0)
    _check(lib().lem_levels(ctx, ctypes.byref(L), _ptr(queue), _ptr(levels), _ptr(depth)),
           "lem_levels")
    return L.value


def lem_accumulate(ctx, counts=None):
    _check(lib().lem_accumulate(ctx, _ptr(counts)), "lem_accumulate")


def lem_erode(ctx):
    _check(lib().lem_erode(ctx), "lem_erode")


def lem_step(ctx, nsteps):
    _check(lib().lem_step(ctx, nsteps), "lem_step")


def lem_set_slope_exponent(ctx, n, eps=1e-12, max_iter=100):
    _check(lib().lem_set_slope_exponent(ctx, n, eps, max_iter), "lem_set_slope_exponent")


def lem_accumulate_mfd(ctx, A, p=1.0, w=None):
    """Eq. 2 with multiple flow directions into the float64 tensor A;
    returns the number of levels."""
    L = ctypes.c_int64(0)
    _check(lib().lem_accumulate_mfd(ctx, p, _ptr(w), _ptr(A), ctypes.byref(L)),
           "lem_accumulate_mfd")
    return L.value


def lem_fill(ctx):
    _check(lib().lem_fill(ctx), "lem_fill")


def lem_set_fill(ctx, on):
    _check(lib().lem_set_fill(ctx, 1 if on else 0), "lem_set_fill")


def lem_fill_stats(ctx):
    """(rounds, tile visits, relaxation passes, unsettled visits) of the last flood."""
    v = (ctypes.c_int64 * 4)()
    _check(lib().lem_fill_stats(ctx, v), "lem_fill_stats")
    return tuple(int(x) for x in v)


def lem_set_receivers(ctx, rec):
    _check(lib().lem_set_receivers(ctx, _ptr(rec)), "lem_set_receivers")


def lem_last_graph(ctx, rec=None, mask=None):
    _check(lib().lem_last_graph(ctx, _ptr(rec), _ptr(mask)), "lem_last_graph")


def lem_state_size(ctx):
    n = ctypes.c_int64(0)
    _check(lib().lem_state_size(ctx, ctypes.byref(n)), "lem_state_size")
    return n.value


def lem_get_state(ctx):
    """The context's state as a host numpy uint8 array (lem_get_state)."""
    import numpy as np
    buf = np.empty(lem_state_size(ctx), np.uint8)
    _check(lib().lem_get_state(ctx, buf.ctypes.data_as(_VP), buf.size), "lem_get_state")
    return buf


def lem_set_state(ctx, buf):
    import numpy as np
    b = np.ascontiguousarray(buf, np.uint8)
    _check(lib().lem_set_state(ctx, b.ctypes.data_as(_VP), b.size), "lem_set_state")


def lem_sync(ctx):
    _check(lib().lem_sync(ctx), "lem_sync")


def lem_set_wait_limit(ctx, seconds):
    _check(lib().lem_set_wait_limit(ctx, seconds), "lem_set_wait_limit")


def lem_selftest_wait(ctx):
    """Returns the raw status (LEM_ETIMEOUT expected)."""
    return lib().lem_selftest_wait(ctx)


def lem_set_step_mode(ctx, mode):
    _check(lib().lem_set_step_mode(ctx, mode), "lem_set_step_mode")


def lem_set_tiling(ctx, strip_rows=0, half_tiles=0):
    _check(lib().lem_set_tiling(ctx, strip_rows, half_tiles), "lem_set_tiling")


def lem_get_tiling(ctx):
    """(rows per strip of the codes pass, half-height warp tiles) in use."""
    k, h = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().lem_get_tiling(ctx, ctypes.byref(k), ctypes.byref(h)), "lem_get_tiling")
    return k.value, h.value


def lem_step_stats(ctx):
    """(steps without device-wide levels, steps with them)."""
    p, g = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib().lem_step_stats(ctx, ctypes.byref(p), ctypes.byref(g)), "lem_step_stats")
    return p.value, g.value


def lem_tier_stats(ctx):
    """Cells handled by (warp tiles, block queues, device-wide levels)."""
    v = (ctypes.c_int64 * 3)()
    _check(lib().lem_tier_stats(ctx, v), "lem_tier_stats")
    return tuple(int(x) for x in v)


def lem_jump_stats(ctx):
    """(steps whose device tier used pointer jumping, erosion rounds of the latest)."""
    v = (ctypes.c_int64 * 2)()
    _check(lib().lem_jump_stats(ctx, v), "lem_jump_stats")
    return int(v[0]), int(v[1])


def lem_adjoint(ctx, h0, lambda_T, nsteps, ckpt_every, dLdU, lambda_0=None):
    """Fills dLdU (and lambda_0 if given); returns dL/dK."""
    k = ctypes.c_double(0.0)
    _check(lib().lem_adjoint(ctx, _ptr(h0), _ptr(lambda_T), nsteps, ckpt_every, _ptr(dLdU),
                             ctypes.byref(k), _ptr(lambda_0)), "lem_adjoint")
    return k.value


def _host(arr, ctype):
    import numpy as np
    a = np.ascontiguousarray(arr, dtype=ctype)
    return a, a.ctypes.data_as(_VP)


def lem_batch_create(nx, ny, dx, K, m, U, dt, dtype=LEM_F32):
    import numpy as np
    R = len(nx)
    keep = [_host(nx, np.int32), _host(ny, np.int32)] + [_host(v, np.float64)
                                                        for v in (dx, K, m, U, dt)]
    b = _VP()
    _check(lib().lem_batch_create(ctypes.byref(b), R, *[p for _, p in keep], dtype),
           "lem_batch_create")
    return b


def lem_batch_destroy(b):
    lib().lem_batch_destroy(b)


def lem_batch_offsets(b, R):
    import numpy as np
    off = np.zeros(R + 1, np.int64)
    _check(lib().lem_batch_offsets(b, off.ctypes.data_as(_VP)), "lem_batch_offsets")
    return off


def lem_batch_set_stream(b, stream=None):
    s = (stream or torch.cuda.current_stream()).cuda_stream
    _check(lib().lem_batch_set_stream(b, ctypes.c_void_p(s)), "lem_batch_set_stream")


def lem_batch_bind_elevation(b, h):
    _check(lib().lem_batch_bind_elevation(b, _ptr(h)), "lem_batch_bind_elevation")


def lem_batch_set_config(b, block_threads, items_per_thread):
    _check(lib().lem_batch_set_config(b, block_threads, items_per_thread),
           "lem_batch_set_config")


def lem_batch_step(b, nsteps):
    _check(lib().lem_batch_step(b, nsteps), "lem_batch_step")


def lem_batch_sync(b):
    _check(lib().lem_batch_sync(b), "lem_batch_sync")


BATCH_CONFIGS = [(256, 4), (256, 8), (512, 4), (512, 8), (1024, 4), (1024, 8)]


class Batch:
    """R independent FP32 grids advanced together (packed elevations)."""

    def __init__(self, surfaces, dx, K, m, U, dt, stream=None):
        import numpy as np
        R = len(surfaces)
        bc = lambda v: list(v) if hasattr(v, "__len__") else [v] * R  # noqa: E731
        self.shapes = [s.shape for s in surfaces]
        self.b = lem_batch_create([s.shape[1] for s in surfaces], [s.shape[0] for s in surfaces],
                                  bc(dx), bc(K), bc(m), bc(U), bc(dt))
        self.R = R
        self.offsets = lem_batch_offsets(self.b, R)
        flat = np.concatenate([np.asarray(s, np.float32).ravel() for s in surfaces])
        self.h = torch.tensor(flat, device="cuda")
        lem_batch_set_stream(self.b, stream)
        lem_batch_bind_elevation(self.b, self.h)

    def surface(self, r):
        ny, nx = self.shapes[r]
        return self.h[self.offsets[r]:self.offsets[r + 1]].view(ny, nx)

    def set_config(self, block_threads, items_per_thread):
        lem_batch_set_config(self.b, block_threads, items_per_thread)

    def step(self, nsteps=1):
        with _nvtx("lem.batch_step"):
            lem_batch_step(self.b, nsteps)

    def sync(self):
        lem_batch_sync(self.b)

    def close(self):
        if self.b:
            lem_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lem_step_noalloc(h, dx, K, m, U, dt, nsteps, stream=None):
    """Allocation-free steps on a (ny, nx) float64 CUDA tensor; returns the raw
    status (the library allocates nothing: see include/lem.h)."""
    if h.dtype != torch.float64:
        raise ValueError("lem_step_noalloc takes float64 elevations")
    ny, nx = h.shape
    # the library launches on the current device: make it h's
    with torch.cuda.device(h.device):
        s = (stream or torch.cuda.current_stream(h.device)).cuda_stream
        return lib().lem_step_noalloc(nx, ny, _ptr(h), dx, K, m, U, dt, nsteps,
                                      ctypes.c_void_p(s))


def lem_trace_enable(ctx, capacity):
    _check(lib().lem_trace_enable(ctx, capacity), "lem_trace_enable")


def lem_trace_read(ctx, cap=4096):
    """Returns a list of (ns, phase name, level) recorded since the last read."""
    import numpy as np
    ns = np.zeros(cap, np.int64)
    tags = np.zeros(cap, np.int32)
    n = ctypes.c_int(0)
    _check(lib().lem_trace_read(ctx, ns.ctypes.data_as(_VP), tags.ctypes.data_as(_VP), cap,
                                ctypes.byref(n)), "lem_trace_read")
    m = min(n.value, cap)
    return [(int(ns[i]), TRACE_PHASES.get(int(tags[i]) >> 16, "?"), int(tags[i]) & 0xFFFF)
            for i in range(m)]


# ---- convenience wrapper ------------------------------------------------------

class Model:
    """One grid: a context plus the bound elevation tensor (ny, nx) on cuda."""

    def __init__(self, h, dx=100.0, K=1e-5, m=0.5, U=1e-3, dt=1000.0, area_scale=0.0,
                 count_bits=32, stream=None):
        if h.dtype == torch.float64:
            self.dtype = LEM_F64
        elif h.dtype == torch.float32:
            self.dtype = LEM_F32
        else:
            raise ValueError("elevations must be float64 or float32")
        self.h = h.contiguous()
        self.ny, self.nx = self.h.shape
        self.count_bits = count_bits
        self.ctx = lem_create_ex(self.nx, self.ny, dx, K, m, U, dt, area_scale, self.dtype,
                                 count_bits)
        lem_set_stream(self.ctx, stream)
        lem_bind_elevation(self.ctx, self.h, self.dtype)
        self._Uf = None

    @property
    def N(self):
        return self.nx * self.ny

    def close(self):
        if self.ctx:
            lem_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_uplift_field(self, Uf):
        self._Uf = None if Uf is None else Uf.to(torch.float64).contiguous()
        lem_set_uplift_field(self.ctx, self._Uf)

    def receivers(self):
        rec = torch.empty(self.N, dtype=torch.int32, device=self.h.device)
        with _nvtx("lem.receivers"):
            lem_receivers(self.ctx, rec)
        return rec

    def donors(self):
        dnum = torch.empty(self.N, dtype=torch.int32, device=self.h.device)
        donor = torch.empty(self.N * 8, dtype=torch.int32, device=self.h.device)
        with _nvtx("lem.donors"):
            lem_donors(self.ctx, dnum, donor)
        return dnum, donor.view(self.N, 8)

    def levels(self, want_depth=True):
        q = torch.empty(self.N, dtype=torch.int32, device=self.h.device)
        lev = torch.empty(self.N + 1, dtype=torch.int64, device=self.h.device)
        depth = torch.empty(self.N, dtype=torch.int32, device=self.h.device) if want_depth else None
        with _nvtx("lem.levels"):
            L = lem_levels(self.ctx, q, lev, depth)
        return q, lev[:L + 1], depth

    def accumulate(self):
        dt = torch.int64 if self.count_bits == 64 else torch.int32
        cnt = torch.empty(self.N, dtype=dt, device=self.h.device)
        with _nvtx("lem.accumulate"):
            lem_accumulate(self.ctx, cnt)
        return cnt

    def erode(self):
        with _nvtx("lem.erode"):
            lem_erode(self.ctx)

    def step(self, nsteps=1):
        with _nvtx("lem.step"):
            lem_step(self.ctx, nsteps)

    def last_graph(self):
        """(rec int32[N], donor mask uint8[N]) of the last step's receiver graph."""
        rec = torch.empty(self.N, dtype=torch.int32, device=self.h.device)
        msk = torch.empty(self.N, dtype=torch.uint8, device=self.h.device)
        lem_last_graph(self.ctx, rec, msk)
        return rec, msk

    def set_receivers(self, rec):
        lem_set_receivers(self.ctx, rec)

    def set_slope_exponent(self, n, eps=1e-12, max_iter=100):
        lem_set_slope_exponent(self.ctx, n, eps, max_iter)

    def fill(self):
        with _nvtx("lem.fill"):
            lem_fill(self.ctx)

    def accumulate_mfd(self, p=1.0, w=None):
        """(A, number of levels) of Eq. 2 with multiple flow directions."""
        A = torch.empty(self.ny, self.nx, dtype=torch.float64, device=self.h.device)
        wt = None if w is None else w.to(torch.float64).contiguous()
        with _nvtx("lem.accumulate_mfd"):
            L = lem_accumulate_mfd(self.ctx, A, p, wt)
        return A, L

    def set_fill(self, on):
        lem_set_fill(self.ctx, on)

    def sync(self):
        lem_sync(self.ctx)
