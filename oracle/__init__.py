"""Serial FP64 oracle of the landscape-evolution time step (test infrastructure).

This package is the plain, slow, obviously correct CPU restatement of
Barnes, "Accelerating a Landscape Evolution Model with Parallelism"
(arXiv:1803.02977), Algorithms 1-6, written in C (``lem_oracle.c``) and driven
from numpy through ctypes.  Only the test suite, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline leg may import it.  It shares no code with
the CUDA library.

Functions and their pins are documented in ``lem_oracle.h``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lem_oracle.c")
_HDR = os.path.join(_HERE, "lem_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liblem_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no contraction, no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or max(
        os.path.getmtime(_SRC), os.path.getmtime(_HDR)) > os.path.getmtime(_LIB_PATH)
    if not (force or stale):
        return _LIB_PATH
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_OUT_DIR)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [("dx", ctypes.c_double), ("K", ctypes.c_double), ("m", ctypes.c_double),
                ("U", ctypes.c_double), ("dt", ctypes.c_double),
                ("area_scale", ctypes.c_double), ("Ufield", ctypes.c_void_p)]


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        pp = ctypes.POINTER(Params)
        L.orc_receivers.argtypes = [i32, i32, vp, vp]
        L.orc_receivers_f32.argtypes = [i32, i32, vp, vp]
        L.orc_donors_grid.argtypes = [i32, i32, vp, vp, vp]
        L.orc_donors_graph.argtypes = [i32, vp, i32, vp, vp]
        L.orc_donors_graph.restype = i32
        L.orc_queue.argtypes = [i64, vp, i32, vp, vp, vp, vp, vp]
        L.orc_queue.restype = i64
        L.orc_accumulate.argtypes = [i64, vp, vp, i64, i32, vp, vp, vp]
        L.orc_uplift.argtypes = [i32, i32, vp, pp]
        L.orc_erode.argtypes = [i32, i32, vp, vp, vp, vp, i64, vp, pp]
        L.orc_erode_newton.argtypes = [i32, i32, vp, vp, vp, vp, i64, vp, pp, dbl, dbl, i32]
        L.orc_accumulate_mfd.argtypes = [i32, i32, vp, vp, dbl, vp, vp]
        L.orc_accumulate_mfd.restype = i64
        L.orc_fill_eps.argtypes = [i32, i32, vp, vp]
        L.orc_fill_eps.restype = i32
        L.orc_fill_eps_f32.argtypes = [i32, i32, vp, vp]
        L.orc_fill_eps_f32.restype = i32
        L.orc_run.argtypes = [i32, i32, vp, i32, pp, vp, vp]
        L.orc_run.restype = i32
        L.orc_adjoint_step.argtypes = [i32, i32, vp, vp, vp, vp, i64, vp, pp, vp, vp, vp,
                                       ctypes.POINTER(dbl)]
        L.orc_tangent_step.argtypes = [i32, i32, vp, vp, vp, vp, i64, vp, pp, vp, vp, dbl, vp]
        _lib = L
    return _lib


def params(dx=100.0, K=1e-5, m=0.5, U=1e-3, dt=1000.0, area_scale=None, Ufield=None):
    """Build a Params struct; area_scale defaults to dx*dx (Alg 4's init)."""
    if area_scale is None:
        area_scale = dx * dx
    p = Params(dx, K, m, U, dt, area_scale, None)
    if Ufield is not None:
        Ufield = np.ascontiguousarray(Ufield, dtype=np.float64)
        p.Ufield = Ufield.ctypes.data
        p._keep = Ufield  # keep alive
    return p


# ---- stage wrappers (numpy in, numpy out) ---------------------------------

def receivers(h):
    """Alg 1 on a (ny, nx) float64 or float32 array -> int32 rec (flat, self = NoFlow)."""
    ny, nx = h.shape
    rec = np.empty(nx * ny, np.int32)
    if h.dtype == np.float32:
        hh = np.ascontiguousarray(h)
        lib().orc_receivers_f32(nx, ny, _p(hh), _p(rec))
    else:
        hh = np.ascontiguousarray(h, dtype=np.float64)
        lib().orc_receivers(nx, ny, _p(hh), _p(rec))
    return rec


def donors_grid(nx, ny, rec):
    """Alg 2 on the grid -> (dnum int32[N], donor int32[N, 8])."""
    rec = np.ascontiguousarray(rec, dtype=np.int32)
    n = nx * ny
    dnum = np.zeros(n, np.int32)
    donor = np.full((n, 8), -1, np.int32)
    lib().orc_donors_grid(nx, ny, _p(rec), _p(dnum), _p(donor))
    return dnum, donor


def donors_graph(rec, dmax):
    rec = np.ascontiguousarray(rec, dtype=np.int32)
    n = rec.size
    dnum = np.zeros(n, np.int32)
    donor = np.full((n, dmax), -1, np.int32)
    rc = lib().orc_donors_graph(n, _p(rec), dmax, _p(dnum), _p(donor))
    if rc != 0:
        raise ValueError("a node has more than dmax donors")
    return dnum, donor


def queue(rec, dnum, donor):
    """Alg 3 -> (Queue int32[N], Levels int64[L+1], depth int32[N])."""
    rec = np.ascontiguousarray(rec, dtype=np.int32)
    n = rec.size
    dmax = donor.shape[1]
    q = np.full(n, -1, np.int32)
    lev = np.zeros(n + 1, np.int64)
    depth = np.empty(n, np.int32)
    donor = np.ascontiguousarray(donor, dtype=np.int32)
    dnum = np.ascontiguousarray(dnum, dtype=np.int32)
    L = lib().orc_queue(n, _p(rec), dmax, _p(dnum), _p(donor), _p(q), _p(lev), _p(depth))
    return q, lev[:L + 1].copy(), depth


def accumulate(queue_, levels, dnum, donor):
    """Alg 4 with w = 1 -> int64 cell counts."""
    n = dnum.size
    cnt = np.zeros(n, np.int64)
    levels = np.ascontiguousarray(levels, dtype=np.int64)
    lib().orc_accumulate(n, _p(np.ascontiguousarray(queue_, np.int32)), _p(levels),
                         levels.size - 1, donor.shape[1],
                         _p(np.ascontiguousarray(dnum, np.int32)),
                         _p(np.ascontiguousarray(donor, np.int32)), _p(cnt))
    return cnt


def uplift(h, p):
    """Alg 5 in place on a (ny, nx) float64 array."""
    ny, nx = h.shape
    lib().orc_uplift(nx, ny, _p(h), ctypes.byref(p))


def erode(h, rec, queue_, levels, cnt, p):
    """Alg 6 (n = 1) in place on a (ny, nx) float64 array already uplifted."""
    ny, nx = h.shape
    levels = np.ascontiguousarray(levels, dtype=np.int64)
    lib().orc_erode(nx, ny, _p(h), _p(np.ascontiguousarray(rec, np.int32)),
                    _p(np.ascontiguousarray(queue_, np.int32)), _p(levels), levels.size - 1,
                    _p(np.ascontiguousarray(cnt, np.int64)), ctypes.byref(p))


def erode_newton(h, rec, queue_, levels, cnt, p, n_exp, eps=1e-12, max_iter=100):
    """Alg 6 for general n-hat (Newton-Raphson from h0) in place on a (ny, nx)
    float64 array already uplifted."""
    ny, nx = h.shape
    levels = np.ascontiguousarray(levels, dtype=np.int64)
    lib().orc_erode_newton(nx, ny, _p(h), _p(np.ascontiguousarray(rec, np.int32)),
                           _p(np.ascontiguousarray(queue_, np.int32)), _p(levels),
                           levels.size - 1, _p(np.ascontiguousarray(cnt, np.int64)),
                           ctypes.byref(p), float(n_exp), float(eps), int(max_iter))


class StepGraph:
    """Everything one step computes from its input elevations."""

    def __init__(self, h, frozen_rec=None):
        ny, nx = h.shape
        self.nx, self.ny = nx, ny
        self.rec = receivers(h) if frozen_rec is None else np.ascontiguousarray(
            frozen_rec, np.int32).copy()
        self.dnum, self.donor = donors_grid(nx, ny, self.rec)
        self.queue, self.levels, self.depth = queue(self.rec, self.dnum, self.donor)
        self.cnt = accumulate(self.queue, self.levels, self.dnum, self.donor)

    @property
    def nlevels(self):
        return self.levels.size - 1


def step(h, p, frozen_rec=None):
    """One full step; returns (h_next, StepGraph)."""
    g = StepGraph(h, frozen_rec)
    hn = np.array(h, dtype=np.float64, copy=True)
    uplift(hn, p)
    erode(hn, g.rec, g.queue, g.levels, g.cnt, p)
    return hn, g


def accumulate_mfd(h, p=1.0, w=None):
    """Eq. 2 with multiple flow directions on a (ny, nx) float64 array:
    returns (A float64 (ny, nx), level int32 (ny, nx), number of levels)."""
    ny, nx = h.shape
    src = np.ascontiguousarray(h, np.float64)
    wt = None if w is None else np.ascontiguousarray(w, np.float64).ravel()
    A = np.zeros(nx * ny, np.float64)
    lev = np.full(nx * ny, -1, np.int32)
    L = lib().orc_accumulate_mfd(nx, ny, _p(src), _p(wt), float(p), _p(A), _p(lev))
    if L < 0:
        raise MemoryError("oracle allocation failed")
    return A.reshape(ny, nx), lev.reshape(ny, nx), int(L)


def fill(h):
    """Depression filling with epsilon increments (Priority-Flood) of a
    (ny, nx) float64 or float32 array; returns the filled array (same dtype)."""
    ny, nx = h.shape
    if h.dtype == np.float32:
        src = np.ascontiguousarray(h, np.float32)
        out = np.empty_like(src)
        rc = lib().orc_fill_eps_f32(nx, ny, _p(src), _p(out))
    else:
        src = np.ascontiguousarray(h, np.float64)
        out = np.empty_like(src)
        rc = lib().orc_fill_eps(nx, ny, _p(src), _p(out))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return out


def step_newton(h, p, n_exp, eps=1e-12, max_iter=100, frozen_rec=None):
    """One full step with Alg 6's Newton iteration for a general n-hat;
    returns (h_next, StepGraph)."""
    g = StepGraph(h, frozen_rec)
    hn = np.array(h, dtype=np.float64, copy=True)
    uplift(hn, p)
    erode_newton(hn, g.rec, g.queue, g.levels, g.cnt, p, n_exp, eps, max_iter)
    return hn, g


def run(h, p, nsteps, frozen_rec=None, want_levels=False):
    """nsteps steps on a copy of h (float64); optionally the per-step level count."""
    ny, nx = h.shape
    hh = np.array(h, dtype=np.float64, copy=True, order="C")
    lv = np.zeros(max(nsteps, 1), np.int64)
    fr = None if frozen_rec is None else np.ascontiguousarray(frozen_rec, np.int32)
    rc = lib().orc_run(nx, ny, _p(hh), nsteps, ctypes.byref(p), _p(fr), _p(lv))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return (hh, lv[:nsteps]) if want_levels else hh


def tangent_step(h_next, g, p, dh, dU, dK):
    ny, nx = h_next.shape
    out = np.zeros(nx * ny, np.float64)
    lib().orc_tangent_step(nx, ny, _p(np.ascontiguousarray(h_next, np.float64)), _p(g.rec),
                           _p(g.queue), _p(g.levels), g.nlevels, _p(g.cnt), ctypes.byref(p),
                           _p(np.ascontiguousarray(dh, np.float64).ravel()),
                           _p(np.ascontiguousarray(dU, np.float64).ravel()), float(dK), _p(out))
    return out.reshape(ny, nx)


def adjoint_step(h_next, g, p, lam, dLdU, dLdK=0.0):
    """Returns (lam_prev, dLdU (updated in place), dLdK)."""
    ny, nx = h_next.shape
    lam_prev = np.zeros(nx * ny, np.float64)
    k = ctypes.c_double(dLdK)
    lib().orc_adjoint_step(nx, ny, _p(np.ascontiguousarray(h_next, np.float64)), _p(g.rec),
                           _p(g.queue), _p(g.levels), g.nlevels, _p(g.cnt), ctypes.byref(p),
                           _p(np.ascontiguousarray(lam, np.float64).ravel()), _p(lam_prev),
                           _p(dLdU), ctypes.byref(k))
    return lam_prev.reshape(ny, nx), dLdU, k.value


def loss_and_grad(h0, p, nsteps, h_obs):
    """L = sum((h_T - h_obs)^2) and (dL/dU field, dL/dK) by the step adjoint.

    Stores every step's input (no checkpointing: the oracle favours plainness).
    The uplift must be given as a per-cell field in p (p.Ufield)."""
    ny, nx = h0.shape
    hs = [np.array(h0, np.float64)]
    graphs = []
    for _ in range(nsteps):
        hn, g = step(hs[-1], p)
        hs.append(hn)
        graphs.append(g)
    hT = hs[-1]
    loss = float(np.sum((hT - h_obs) ** 2))
    lam = 2.0 * (hT - h_obs)
    dLdU = np.zeros(nx * ny, np.float64)
    dLdK = 0.0
    for t in range(nsteps - 1, -1, -1):
        lam, dLdU, dLdK = adjoint_step(hs[t + 1], graphs[t], p, lam, dLdU, dLdK)
    return loss, dLdU.reshape(ny, nx), dLdK
