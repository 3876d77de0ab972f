"""FP64 CPU oracle (ctypes binding of ivv_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the library.  It shares no code with
the CUDA path; both consume the seeded inputs of
``paper_1404_3363_gb300.scenes``.

Functions follow the paper (Fuchs & Hjelmervik, TVCG 2015):
  eval           Eq. 1 (Cox-de Boor), first partials, scalar per mode
                 (control points, det J, Eq. 23, von Mises of §6.2 Eq. 24)
  hits / pairs   §4.1 intersections, §4.2 Alg. 2 pairing
  invert         §5.1 Newton (RF) with QR, clamping and line search
  composite      §3.2.1 Alg. 1 with supersampling
  render         the whole per-pixel path, per-sample RF (method 0),
                 RKF45 on the pulled-back ODE of §5.2 (method 1) or one step
                 per sample interval of the fixed-step RK family of §5.2-5.3
                 (FIXED_* methods) or of implicit Euler (IMPLICIT_EULER)
  table1         §5.3 Table 1 harness (fixed-step RK family / RF / implicit
                 Euler)
  eval2          second partials (the Hessian used by implicit Euler)
Cutting and near-clip planes (§5.5) act on the depth-sorted intersections
before compositing (render with params.near_clip / params.cut_planes).
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

_LIB = None

# render methods: per-sample root finding, RKF45 with error control, and the
# fixed-step explicit RK family of §5.2-5.3 (one step per sample interval)
METHOD_RF = 0
METHOD_RKF45 = 1
FIXED_EULER, FIXED_MIDPOINT, FIXED_KUTTA3, FIXED_RK4, FIXED_RK4_38, FIXED_FEHLBERG5 = 11, 12, 13, 14, 15, 16
FIXED_ORDER = {11: 1, 12: 2, 13: 3, 14: 4, 15: 4, 16: 5}
# implicit Euler of §5.2 (one step per sample interval, Newton with the exact
# Jacobian of G)
IMPLICIT_EULER = 17

c_double_p = C.POINTER(C.c_double)


class _Block(C.Structure):
    _fields_ = [("degree", C.c_int * 3), ("n_cp", C.c_int * 3),
                ("knots", c_double_p * 3), ("geom_cp", c_double_p),
                ("scalar_cp", c_double_p), ("disp_cp", c_double_p)]


class _Camera(C.Structure):
    _fields_ = [("ortho", C.c_int), ("eye", C.c_double * 3), ("target", C.c_double * 3),
                ("up", C.c_double * 3), ("fovy_deg", C.c_double), ("ortho_height", C.c_double)]


class _TF(C.Structure):
    _fields_ = [("n_knots", C.c_int), ("r", c_double_p), ("rgba", c_double_p),
                ("sigma", C.c_double), ("lo", C.c_double), ("hi", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("ds", C.c_double), ("supersample_k", C.c_int), ("c", C.c_double),
                ("early_alpha", C.c_double), ("method", C.c_int),
                ("newton_tol", C.c_double), ("rk_tol", C.c_double),
                ("near_clip", C.c_double), ("n_cut", C.c_int), ("cut", (C.c_double * 4) * 4)]


class Hit(C.Structure):
    _fields_ = [("t", C.c_double), ("p", C.c_double * 3), ("block", C.c_int),
                ("face", C.c_int), ("front", C.c_int)]


class Pair(C.Structure):
    _fields_ = [("block", C.c_int), ("t_in", C.c_double), ("t_out", C.c_double),
                ("p_in", C.c_double * 3), ("p_out", C.c_double * 3)]


class PixelStats(C.Structure):
    _fields_ = [("npairs", C.c_int), ("unmatched", C.c_int), ("newton_fail", C.c_int),
                ("nsamples", C.c_int), ("rk_steps", C.c_int), ("shrunk", C.c_int)]


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_volume_create.restype = C.c_void_p
        L.orc_volume_create.argtypes = [C.POINTER(_Block), C.c_int, C.c_int, C.c_char_p, C.c_int]
        L.orc_volume_destroy.argtypes = [C.c_void_p]
        L.orc_volume_diag.restype = C.c_double
        L.orc_volume_diag.argtypes = [C.c_void_p]
        L.orc_volume_npieces.argtypes = [C.c_void_p]
        L.orc_eval.argtypes = [C.c_void_p, C.c_int, C.c_int, c_double_p, c_double_p, c_double_p, c_double_p]
        L.orc_basis.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, c_double_p, c_double_p, c_double_p]
        L.orc_scalar_range.argtypes = [C.c_void_p, C.c_int, c_double_p, c_double_p]
        L.orc_ray.argtypes = [C.POINTER(_Camera), C.c_int, C.c_int, C.c_double, C.c_double, c_double_p, c_double_p]
        L.orc_hits.argtypes = [C.c_void_p, c_double_p, c_double_p, C.c_int, C.POINTER(Hit)]
        L.orc_pair_hits.argtypes = [C.POINTER(Hit), C.c_int, C.c_int, C.POINTER(Pair), C.POINTER(C.c_int)]
        L.orc_pixel_pairs.argtypes = [C.c_void_p, C.POINTER(_Camera), C.c_int, C.c_int, C.c_int, C.c_int,
                                      C.c_int, C.POINTER(Pair), C.POINTER(C.c_int)]
        L.orc_invert.argtypes = [C.c_void_p, C.c_int, c_double_p, c_double_p, C.c_double, C.c_int, c_double_p]
        L.orc_composite.argtypes = [C.POINTER(_TF), C.c_int, C.c_double, C.c_int, c_double_p, c_double_p, c_double_p]
        L.orc_trace_pair.argtypes = [C.c_void_p, C.POINTER(_TF), C.POINTER(_Params), c_double_p, c_double_p,
                                     C.POINTER(Pair), C.c_int, c_double_p]
        L.orc_render.argtypes = [C.c_void_p, C.POINTER(_TF), C.POINTER(_Camera), C.POINTER(_Params),
                                 C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                 c_double_p, C.POINTER(PixelStats)]
        L.orc_table1.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, c_double_p]
        L.orc_table1_ex.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, c_double_p, C.POINTER(C.c_long)]
        L.orc_eval2.argtypes = [C.c_void_p, C.c_int, C.c_int, c_double_p, c_double_p, c_double_p, c_double_p]
        L.orc_window_pairs.argtypes = [C.c_void_p, C.POINTER(_Camera), C.c_int, C.c_int, C.c_int, C.c_int,
                                       C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), c_double_p,
                                       C.POINTER(C.c_int)]
        L.orc_walk_into_block.argtypes = [C.c_void_p, C.c_int, c_double_p, c_double_p, C.c_double, C.c_double,
                                          c_double_p, c_double_p, c_double_p, c_double_p]
        L.orc_t1_irk1_step.argtypes = [c_double_p, C.c_double, C.c_double, C.c_double, C.c_int, c_double_p]
        _LIB = L
    return _LIB


def _dp(a):
    return a.ctypes.data_as(c_double_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def camera_struct(cam):
    c = _Camera()
    c.ortho = int(cam.ortho)
    for i in range(3):
        c.eye[i], c.target[i], c.up[i] = cam.eye[i], cam.target[i], cam.up[i]
    c.fovy_deg = cam.fovy_deg
    c.ortho_height = cam.ortho_height
    return c


class OracleVolume:
    """Oracle copy of a multi-block volume (scalar mode CP / DETJ / QUALITY /
    VONMISES, the last from the blocks' displacement control points, §6.2)."""

    def __init__(self, blocks, scalar_mode):
        L = lib()
        self._keep = []
        arr = (_Block * len(blocks))()
        for bi, b in enumerate(blocks):
            kn = [_f64(k) for k in b.knots]
            g = _f64(b.geom_cp)
            s = _f64(b.scalar_cp) if b.scalar_cp is not None else None
            u = _f64(b.disp_cp) if getattr(b, "disp_cp", None) is not None else None
            self._keep += kn + [g] + [x for x in (s, u) if x is not None]
            nu, nv, nw = b.n_cp
            for d in range(3):
                arr[bi].degree[d] = int(b.degree[d])
                arr[bi].knots[d] = _dp(kn[d])
            arr[bi].n_cp[0], arr[bi].n_cp[1], arr[bi].n_cp[2] = nu, nv, nw
            arr[bi].geom_cp = _dp(g)
            arr[bi].scalar_cp = _dp(s) if s is not None else c_double_p()
            arr[bi].disp_cp = _dp(u) if u is not None else c_double_p()
        err = C.create_string_buffer(256)
        h = L.orc_volume_create(arr, len(blocks), int(scalar_mode), err, 256)
        if not h:
            raise ValueError("oracle: " + err.value.decode())
        self.h = h
        self.n_blocks = len(blocks)
        self.mode = scalar_mode

    def __del__(self):
        if getattr(self, "h", None) and _LIB is not None:
            _LIB.orc_volume_destroy(self.h)
            self.h = None

    @property
    def diag(self):
        return lib().orc_volume_diag(self.h)

    @property
    def n_pieces(self):
        return lib().orc_volume_npieces(self.h)

    def eval(self, block, p):
        p = _f64(np.atleast_2d(p))
        n = p.shape[0]
        phi = np.zeros((n, 3))
        J = np.zeros((n, 3, 3))
        rho = np.zeros(n)
        lib().orc_eval(self.h, block, n, _dp(p), _dp(phi), _dp(J), _dp(rho))
        return phi, J, rho

    def eval2(self, block, p):
        """phi, J and the Hessian H[n][r][a][b] = d^2 phi_r / dp_a dp_b."""
        p = _f64(np.atleast_2d(p))
        n = p.shape[0]
        phi = np.zeros((n, 3))
        J = np.zeros((n, 3, 3))
        H = np.zeros((n, 3, 3, 3))
        lib().orc_eval2(self.h, block, n, _dp(p), _dp(phi), _dp(J), _dp(H))
        return phi, J, H

    def basis(self, block, direction, x, n_cp):
        x = _f64(np.atleast_1d(x))
        N = np.zeros((len(x), n_cp))
        dN = np.zeros((len(x), n_cp))
        lib().orc_basis(self.h, block, direction, len(x), _dp(x), _dp(N), _dp(dN))
        return N, dN

    def scalar_range(self, n=64):
        cache = self.__dict__.setdefault("_range_cache", {})
        if n not in cache:
            lo, hi = C.c_double(), C.c_double()
            lib().orc_scalar_range(self.h, n, C.byref(lo), C.byref(hi))
            cache[n] = (lo.value, hi.value)
        return cache[n]

    def hits(self, o, d, cap=256):
        out = (Hit * cap)()
        o, d = _f64(o), _f64(d)
        n = lib().orc_hits(self.h, _dp(o), _dp(d), cap, out)
        return [out[i] for i in range(min(n, cap))]

    def pixel_pairs(self, cam, W, H, x, y, cap=64):
        out = (Pair * cap)()
        um = C.c_int()
        c = camera_struct(cam)
        n = lib().orc_pixel_pairs(self.h, C.byref(c), W, H, x, y, cap, out, C.byref(um))
        return [out[i] for i in range(min(n, cap))], um.value

    def window_pairs(self, cam, W, H, window=None, cap=16, n_threads=None):
        """Entry/exit pairs of every pixel of a window (x0, x1, y0, y1) of a
        W x H image: (count [h*w], pairs [cap][h*w][8] as (p_in, t_in, p_out,
        t_out), block [cap][h*w]), the layout of the library's pair export."""
        x0, x1, y0, y1 = window if window is not None else (0, W, 0, H)
        npx = (x1 - x0) * (y1 - y0)
        cnt = np.zeros(npx, np.int32)
        pairs = np.full((cap, npx, 8), np.nan)
        blk = np.full((cap, npx), -1, np.int32)
        c = camera_struct(cam)
        nt = n_threads if n_threads is not None else (os.cpu_count() or 1)
        lib().orc_window_pairs(self.h, C.byref(c), W, H, x0, x1, y0, y1, nt, cap,
                               cnt.ctypes.data_as(C.POINTER(C.c_int)), _dp(pairs),
                               blk.ctypes.data_as(C.POINTER(C.c_int)))
        return cnt, pairs, blk

    def walk_into_block(self, block, o, d, t0, t1, p0, p1):
        """First point of the ray segment [t0, t1] inside the block (§5.4's
        walk along the ray): (t, p) or None."""
        o, d, p0, p1 = _f64(o), _f64(d), _f64(p0), _f64(p1)
        t = C.c_double()
        p = np.zeros(3)
        ok = lib().orc_walk_into_block(self.h, block, _dp(o), _dp(d), float(t0), float(t1), _dp(p0), _dp(p1),
                                       C.byref(t), _dp(p))
        return (t.value, p) if ok else None

    def invert(self, block, g, p0, tol=1e-13, maxit=50):
        g, p0 = _f64(g), _f64(p0)
        p = np.zeros(3)
        it = lib().orc_invert(self.h, block, _dp(g), _dp(p0), tol * self.diag, maxit, _dp(p))
        return p, it


def pair_hits(hits):
    n = len(hits)
    arr = (Hit * max(n, 1))(*hits)
    out = (Pair * max(n, 1))()
    um = C.c_int()
    k = lib().orc_pair_hits(arr, n, max(n, 1), out, C.byref(um))
    return [out[i] for i in range(k)], um.value


def ray(cam, W, H, x, y):
    o = np.zeros(3)
    d = np.zeros(3)
    c = camera_struct(cam)
    lib().orc_ray(C.byref(c), W, H, float(x), float(y), _dp(o), _dp(d))
    return o, d


def tf_struct(tf, lo, hi):
    r = _f64(tf.r)
    rgba = _f64(tf.rgba)
    t = _TF()
    t.n_knots = len(r)
    t.r = _dp(r)
    t.rgba = _dp(rgba)
    t.sigma = float(tf.sigma)
    t.lo = float(lo)
    t.hi = float(hi)
    return t, (r, rgba)


def composite(tf, s, rho, K=4, early=1 - 1e-4, lo=0.0, hi=1.0):
    t, keep = tf_struct(tf, lo, hi)
    s, rho = _f64(s), _f64(rho)
    out = np.zeros(4)
    lib().orc_composite(C.byref(t), K, early, len(s), _dp(s), _dp(rho), _dp(out))
    return out


def params_struct(p, diag, method=0, newton_tol=1e-13, rk_tol=1e-12):
    q = _Params()
    q.ds = p.ds if p.ds > 0 else diag / 128.0
    q.supersample_k = p.supersample_k
    q.c = p.c
    q.early_alpha = p.early_alpha
    q.method = method
    q.newton_tol = newton_tol
    q.rk_tol = rk_tol
    q.near_clip = getattr(p, "near_clip", 0.0)
    planes = list(getattr(p, "cut_planes", ()))
    assert len(planes) <= 4
    q.n_cut = len(planes)
    for k, pl in enumerate(planes):
        for c in range(4):
            q.cut[k][c] = float(pl[c])
    return q


def resolve_range(vol: OracleVolume, tf):
    lo, hi = tf.lo, tf.hi
    if not (math.isfinite(lo) and math.isfinite(hi) and hi > lo):
        lo, hi = vol.scalar_range(64)
        if not hi > lo:
            hi = lo + 1.0
    return lo, hi


def trace_pair(vol, scene, o, d, pair, method=0, cap=100000):
    lo, hi = resolve_range(vol, scene.tf)
    t, keep = tf_struct(scene.tf, lo, hi)
    prm = params_struct(scene.params, vol.diag, method)
    rows = np.zeros((cap, 5))
    o, d = _f64(o), _f64(d)
    n = lib().orc_trace_pair(vol.h, C.byref(t), C.byref(prm), _dp(o), _dp(d), C.byref(pair), cap, _dp(rows))
    return rows[:min(n, cap)]


def render(scene, vol=None, method=0, window=None, n_threads=None, stats=False,
           newton_tol=1e-13, rk_tol=1e-12):
    """FP64 image of a scene (or of a window (x0, x1, y0, y1) of it).

    Returns float64 [h][w][4] (and per-pixel stats if asked)."""
    if vol is None:
        vol = OracleVolume(scene.blocks, scene.scalar_mode)
    W, H = scene.width, scene.height
    x0, x1, y0, y1 = window if window is not None else (0, W, 0, H)
    lo, hi = resolve_range(vol, scene.tf)
    t, keep = tf_struct(scene.tf, lo, hi)
    prm = params_struct(scene.params, vol.diag, method, newton_tol, rk_tol)
    c = camera_struct(scene.camera)
    out = np.zeros((y1 - y0, x1 - x0, 4))
    st = (PixelStats * ((y1 - y0) * (x1 - x0)))() if stats else None
    nt = n_threads if n_threads is not None else (os.cpu_count() or 1)
    lib().orc_render(vol.h, C.byref(t), C.byref(c), C.byref(prm), W, H, x0, x1, y0, y1, nt,
                     _dp(out), st)
    if stats:
        arr = np.array([[s.npairs, s.unmatched, s.newton_fail, s.nsamples, s.rk_steps, s.shrunk] for s in st],
                       dtype=np.int64).reshape(y1 - y0, x1 - x0, 6)
        return out, arr
    return out


def table1(method, ds, c=1.0, rf_tol=1e-14):
    e = C.c_double()
    lib().orc_table1(int(method), float(ds), float(c), float(rf_tol), C.byref(e))
    return e.value


def t1_irk1_step(p, h, c=100.0, tol=1e-13, max_it=50):
    """One implicit Euler step on the Table 1 harness's analytic map:
    (new point, Newton iterations or -1 for the boundary step of §5.4)."""
    p = _f64(p)
    pn = np.zeros(3)
    it = lib().orc_t1_irk1_step(_dp(p), float(h), float(c), float(tol), int(max_it), _dp(pn))
    return pn, it


def table1_irk1(ds, c=100.0):
    """Table 1's implicit Euler row: (error, steps, Newton iterations)."""
    e, it = C.c_double(), C.c_long()
    steps = lib().orc_table1_ex(8, float(ds), float(c), 1e-14, C.byref(e), C.byref(it))
    return e.value, steps, it.value
