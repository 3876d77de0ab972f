"""Thin Python binding of libivv.so (include/ivv.h): argument marshalling only.

Every step of the render runs in the library's CUDA kernels; PyTorch provides
device memory (tensors) and streams.  There is no CPU fallback: if the library
is missing or no GPU is present, these calls raise.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libivv.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ivv.h")

IVV_OK = 0
STATUS_NAMES = {0: "IVV_OK", 1: "IVV_ERR_INVALID_ARG", 2: "IVV_ERR_CUDA", 3: "IVV_ERR_OOM",
                4: "IVV_ERR_ABUF_OVERFLOW", 5: "IVV_ERR_NONCONVERGED", 6: "IVV_ERR_DEGENERATE",
                7: "IVV_ERR_UNSUPPORTED", 8: "IVV_ERR_WORKSPACE"}
FLAG_STATS = 1
FLAG_TIMING = 2
GUESS_PARAMS = 4611
# ODE integrators (rk_method): error-controlled BS3(2), the explicit fixed-step
# family and implicit Euler
RK_BS32, RK_EULER, RK_MIDPOINT, RK_KUTTA3, RK_RK4, RK_RK4_38, RK_FEHLBERG5, RK_IMPLICIT_EULER = range(8)
STAGES = ("project", "intersect", "pair", "integrate")

c_double_p = C.POINTER(C.c_double)
c_float_p = C.POINTER(C.c_float)


class IvvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class BlockDesc(C.Structure):
    _fields_ = [("degree", C.c_int * 3), ("n_cp", C.c_int * 3), ("knots", c_double_p * 3),
                ("geom_cp", c_double_p), ("scalar_cp", c_double_p), ("disp_cp", c_double_p)]


class Camera(C.Structure):
    _fields_ = [("ortho", C.c_int), ("eye", C.c_double * 3), ("target", C.c_double * 3),
                ("up", C.c_double * 3), ("fovy_deg", C.c_double), ("ortho_height", C.c_double)]


METHOD_ODE, METHOD_RF = 0, 1
GUESS_CENTER, GUESS_MLP, GUESS_CHORD = 0, 1, 2


class RenderParams(C.Structure):
    _fields_ = [("rk_tol", C.c_double), ("ds", C.c_double), ("supersample_k", C.c_int),
                ("c", C.c_double), ("early_alpha", C.c_double), ("use_mlp_guess", C.c_int),
                ("precision", C.c_int), ("flags", C.c_int), ("x0", C.c_int), ("y0", C.c_int),
                ("full_width", C.c_int), ("full_height", C.c_int), ("method", C.c_int), ("rf_tol", C.c_double),
                ("rk_method", C.c_int), ("near_clip", C.c_double), ("n_cut_planes", C.c_int),
                ("cut_planes", (C.c_double * 4) * 4)]


class Limits(C.Structure):
    _fields_ = [("max_frags", C.c_int), ("max_pairs", C.c_int), ("items_per_pixel", C.c_int),
                ("max_rk_steps", C.c_int), ("max_newton", C.c_int)]


class GuessTrainParams(C.Structure):
    _fields_ = [("samples_per_block", C.c_int), ("epochs", C.c_int), ("batch", C.c_int), ("lr", C.c_float),
                ("seed", C.c_ulonglong)]


class Request(C.Structure):
    _fields_ = [("volume", C.c_void_p), ("camera", Camera), ("width", C.c_int), ("height", C.c_int),
                ("tf_n", C.c_int), ("tf_r", c_float_p), ("tf_rgba", c_float_p), ("tf_sigma", C.c_float),
                ("scalar_lo", C.c_double), ("scalar_hi", C.c_double), ("out_rgba", C.c_void_p)]


class BatchTuning(C.Structure):
    _fields_ = [("tile_w", C.c_int), ("tile_h", C.c_int), ("k5_ctas_per_sm", C.c_int), ("step_samples", C.c_int)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [(n, C.c_ulonglong) for n in (
        "rays", "pairs", "fragments", "samples", "rk_steps", "rk_rejects", "rhs_evals", "isect_newton",
        "isect_tests", "fp64_solves", "abuf_overflow", "pair_overflow", "unmatched", "step_cap",
        "rf_newton_iters", "rf_unconverged", "isect_items", "isect_split", "rho_evals", "entry_shrinks",
        "entry_newton", "async_timeouts")] + \
        [("max_delta_p", C.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_LIB = None


def header_functions():
    """Names of the functions include/ivv.h declares."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ivv_[a-z_0-9]+)\s*\(", src)))


def load(path: str = LIB_PATH):
    """Load libivv.so (built by paper_1404_3363_gb300.build)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise IvvError(-1, "libivv.so not built (%s); run __graft_entry__.build()" % path)
    L = C.CDLL(path)
    vp = C.c_void_p
    L.ivv_last_error.restype = C.c_char_p
    L.ivv_create_volume.argtypes = [C.POINTER(BlockDesc), C.c_int, C.c_int, vp, C.POINTER(vp)]
    L.ivv_set_transfer_function.argtypes = [vp, C.c_int, c_float_p, c_float_p, C.c_float, C.c_float, C.c_float]
    L.ivv_get_scalar_range.argtypes = [vp, c_double_p, c_double_p]
    L.ivv_workspace_size.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_size_t)]
    L.ivv_render.argtypes = [vp, C.POINTER(Camera), C.POINTER(RenderParams), C.c_int, C.c_int, vp, vp,
                             C.c_size_t, vp]
    L.ivv_render_to_host.argtypes = [vp, C.POINTER(Camera), C.POINTER(RenderParams), C.c_int, C.c_int, vp, vp]
    L.ivv_render_to_host_async.argtypes = [vp, C.POINTER(Camera), C.POINTER(RenderParams), C.c_int, C.c_int, vp,
                                           vp]
    L.ivv_render_to_host_wait.argtypes = [vp]
    L.ivv_render_noalloc.argtypes = [vp, C.POINTER(Camera), C.POINTER(RenderParams), C.c_int, C.c_int, vp, vp]
    L.ivv_render_pairs.argtypes = [vp, C.POINTER(Camera), C.POINTER(RenderParams), C.c_int, C.c_int, C.c_int,
                                   vp, vp, vp, vp, C.c_size_t, vp]
    L.ivv_eval_points.argtypes = [vp, C.c_int, C.c_int, vp, vp, vp, vp, vp]
    L.ivv_host_eval.argtypes = [C.POINTER(BlockDesc), C.c_int, C.c_int, C.c_int, C.c_int, c_double_p, c_double_p,
                                c_double_p, c_double_p]
    L.ivv_get_stage_times.argtypes = [vp, c_float_p]
    L.ivv_host_render_pairs.argtypes = [C.POINTER(BlockDesc), C.c_int, C.c_int, C.POINTER(Camera),
                                        C.POINTER(RenderParams), C.c_int, C.c_int, C.c_int, vp, vp, vp]
    L.ivv_train_guess.argtypes = [vp, C.POINTER(GuessTrainParams), c_float_p, vp]
    L.ivv_guess_points.argtypes = [vp, C.c_int, vp, vp, vp, vp]
    L.ivv_invert_points.argtypes = [vp, C.c_int, vp, vp, C.c_int, C.c_float, vp, vp, vp]
    L.ivv_guess_loss_grad.argtypes = [vp, C.c_int, C.c_int, vp, vp, c_float_p, c_float_p, vp]
    L.ivv_get_guess_weights.argtypes = [vp, C.c_int, c_float_p, c_float_p, c_float_p]
    L.ivv_set_guess_weights.argtypes = [vp, C.c_int, c_float_p]
    L.ivv_get_stats.argtypes = [vp, C.POINTER(Stats)]
    L.ivv_reset_stats.argtypes = [vp]
    L.ivv_set_limits.argtypes = [vp, C.POINTER(Limits)]
    L.ivv_get_limits.argtypes = [vp, C.POINTER(Limits)]
    L.ivv_check_frame.argtypes = [vp]
    L.ivv_volume_info.argtypes = [vp] + [C.POINTER(C.c_int)] * 4
    L.ivv_destroy_volume.argtypes = [vp]
    L.ivv_destroy_volume.restype = None
    L.ivv_batch_create.argtypes = [C.POINTER(Request), C.c_int, C.POINTER(RenderParams), vp, C.POINTER(vp)]
    L.ivv_batch_render.argtypes = [vp, C.c_int, vp]
    L.ivv_batch_set_camera.argtypes = [vp, C.c_int, C.POINTER(Camera), vp]
    L.ivv_batch_set_tuning.argtypes = [vp, C.POINTER(BatchTuning)]
    L.ivv_batch_get_tuning.argtypes = [vp, C.POINTER(BatchTuning)]
    L.ivv_batch_autotune.argtypes = [vp, C.c_int, C.POINTER(BatchTuning), c_float_p, vp]
    L.ivv_batch_get_stats.argtypes = [vp, C.POINTER(Stats)]
    L.ivv_batch_reset_stats.argtypes = [vp]
    L.ivv_batch_get_stage_times.argtypes = [vp, c_float_p]
    L.ivv_batch_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_longlong), C.POINTER(C.c_size_t),
                                 C.POINTER(C.c_int)]
    L.ivv_batch_destroy.argtypes = [vp]
    L.ivv_batch_destroy.restype = None
    _LIB = L
    return L


def _check(status):
    if status != IVV_OK:
        raise IvvError(status, load().ivv_last_error().decode(errors="replace"))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def camera_struct(cam) -> Camera:
    c = Camera()
    c.ortho = int(cam.ortho)
    for i in range(3):
        c.eye[i], c.target[i], c.up[i] = cam.eye[i], cam.target[i], cam.up[i]
    c.fovy_deg = float(cam.fovy_deg)
    c.ortho_height = float(cam.ortho_height)
    return c


def params_struct(p=None, flags=0, window=None) -> RenderParams:
    q = RenderParams()
    q.rk_tol = p.rk_tol if p else 1e-5
    q.ds = p.ds if p else 0.0
    q.supersample_k = p.supersample_k if p else 4
    q.c = p.c if p else 1.0
    q.early_alpha = p.early_alpha if p else 1.0 - 1e-4
    q.use_mlp_guess = getattr(p, "use_mlp_guess", 0) if p else 0
    q.precision = p.precision if p else 0
    q.method = getattr(p, "method", 0) if p else 0
    q.rf_tol = getattr(p, "rf_tol", 0.05) if p else 0.05
    q.rk_method = getattr(p, "rk_method", 0) if p else 0
    q.near_clip = getattr(p, "near_clip", 0.0) if p else 0.0
    planes = list(getattr(p, "cut_planes", ())) if p else []
    if len(planes) > 4:
        raise IvvError(1, "at most 4 cutting planes")
    q.n_cut_planes = len(planes)
    for k, pl in enumerate(planes):
        for c in range(4):
            q.cut_planes[k][c] = float(pl[c])
    q.flags = flags
    if window is not None:
        q.x0, q.y0, q.full_width, q.full_height = window
    return q


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def block_descs(blocks):
    """ctypes block descriptors plus the arrays they point into (keep both alive)."""
    keep = []
    arr = (BlockDesc * len(blocks))()
    for bi, b in enumerate(blocks):
        kn = [_f64(k) for k in b.knots]
        g = _f64(b.geom_cp)
        s = _f64(b.scalar_cp) if b.scalar_cp is not None else None
        u = _f64(b.disp_cp) if getattr(b, "disp_cp", None) is not None else None
        keep += kn + [g] + [x for x in (s, u) if x is not None]
        nu, nv, nw = b.n_cp
        for d in range(3):
            arr[bi].degree[d] = int(b.degree[d])
            arr[bi].knots[d] = kn[d].ctypes.data_as(c_double_p)
        arr[bi].n_cp[0], arr[bi].n_cp[1], arr[bi].n_cp[2] = nu, nv, nw
        arr[bi].geom_cp = g.ctypes.data_as(c_double_p)
        arr[bi].scalar_cp = s.ctypes.data_as(c_double_p) if s is not None else c_double_p()
        arr[bi].disp_cp = u.ctypes.data_as(c_double_p) if u is not None else c_double_p()
    return arr, keep


def host_eval(blocks, scalar_mode, block, p):
    """FP64 host evaluation of the library's Bezier-extracted representation."""
    arr, keep = block_descs(blocks)
    p = _f64(np.atleast_2d(p))
    n = p.shape[0]
    phi = np.zeros((n, 3))
    jac = np.zeros((n, 3, 3))
    rho = np.zeros(n)
    _check(load().ivv_host_eval(arr, len(blocks), int(scalar_mode), int(block), n, p.ctypes.data_as(c_double_p),
                                phi.ctypes.data_as(c_double_p), jac.ctypes.data_as(c_double_p),
                                rho.ctypes.data_as(c_double_p)))
    return phi, jac, rho


def host_render_pairs(blocks, scalar_mode, camera, params, width, height, max_pairs=16, window=None):
    """Stage 1-2 code of the device path executed on the host (inspection)."""
    arr, keep = block_descs(blocks)
    npix = width * height
    cnt = np.zeros(npix, np.int32)
    pairs = np.zeros((max_pairs, npix, 8))
    blk = np.zeros((max_pairs, npix), np.int32)
    cam = camera_struct(camera)
    prm = params_struct(params, 0, window)
    _check(load().ivv_host_render_pairs(arr, len(blocks), int(scalar_mode), C.byref(cam), C.byref(prm), width,
                                        height, max_pairs, C.c_void_p(cnt.ctypes.data),
                                        C.c_void_p(pairs.ctypes.data), C.c_void_p(blk.ctypes.data)))
    return cnt, pairs, blk


class Volume:
    """A multi-block spline volume resident on the current CUDA device."""

    def __init__(self, blocks, scalar_mode, stream=None):
        L = load()
        arr, keep = block_descs(blocks)
        h = C.c_void_p()
        _check(L.ivv_create_volume(arr, len(blocks), int(scalar_mode), C.c_void_p(_stream_ptr(stream)),
                                   C.byref(h)))
        self.h = h
        self.scalar_mode = scalar_mode
        self._ws = None

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            load().ivv_destroy_volume(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        v = [C.c_int() for _ in range(4)]
        _check(load().ivv_volume_info(self.h, *[C.byref(x) for x in v]))
        return dict(zip(("n_blocks", "n_elements", "n_faces", "degree"), (x.value for x in v)))

    def set_transfer_function(self, tf):
        r = np.ascontiguousarray(tf.r, dtype=np.float32)
        rgba = np.ascontiguousarray(tf.rgba, dtype=np.float32)
        lo = tf.lo if math.isfinite(tf.lo) else float("nan")
        hi = tf.hi if math.isfinite(tf.hi) else float("nan")
        _check(load().ivv_set_transfer_function(self.h, len(r), r.ctypes.data_as(c_float_p),
                                                rgba.ctypes.data_as(c_float_p), float(tf.sigma), lo, hi))

    def scalar_range(self):
        lo, hi = C.c_double(), C.c_double()
        _check(load().ivv_get_scalar_range(self.h, C.byref(lo), C.byref(hi)))
        return lo.value, hi.value

    def workspace_size(self, width, height, precision=0):
        n = C.c_size_t()
        _check(load().ivv_workspace_size(self.h, width, height, precision, C.byref(n)))
        return n.value

    def workspace(self, width, height, precision=0):
        """A cached torch uint8 workspace tensor large enough for the window."""
        import torch
        need = self.workspace_size(width, height, precision)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
        base = self._ws.data_ptr()
        off = (-base) % 256
        return base + off, need

    def render(self, camera, params=None, width=None, height=None, out=None, stream=None, flags=0,
               window=None):
        """Render into a float32 [H][W][4] CUDA tensor (allocated if out is None)."""
        import torch
        if out is None:
            out = torch.empty((height, width, 4), dtype=torch.float32, device="cuda")
        prm = params_struct(params, flags, window)
        ws, need = self.workspace(width, height, prm.precision)
        cam = camera_struct(camera)
        _check(load().ivv_render(self.h, C.byref(cam), C.byref(prm), width, height,
                                 C.c_void_p(out.data_ptr()), C.c_void_p(ws), need,
                                 C.c_void_p(_stream_ptr(stream))))
        return out

    def render_noalloc(self, camera, params, width, height, out, stream=None, flags=0):
        """Render a small window into the caller's float32 [H][W][4] CUDA tensor
        without any device allocation (the library's fixed scratch array)."""
        prm = params_struct(params, flags)
        cam = camera_struct(camera)
        _check(load().ivv_render_noalloc(self.h, C.byref(cam), C.byref(prm), width, height,
                                         C.c_void_p(out.data_ptr()), C.c_void_p(_stream_ptr(stream))))
        return out

    def render_to_host(self, camera, params, width, height, out_host, stream=None, flags=0, window=None):
        """Render and copy into host memory (numpy float32 [H][W][4] or a pinned tensor)."""
        prm = params_struct(params, flags, window)
        cam = camera_struct(camera)
        ptr = out_host.ctypes.data if isinstance(out_host, np.ndarray) else out_host.data_ptr()
        _check(load().ivv_render_to_host(self.h, C.byref(cam), C.byref(prm), width, height, C.c_void_p(ptr),
                                         C.c_void_p(_stream_ptr(stream))))
        return out_host

    def render_to_host_async(self, camera, params, width, height, out_host, stream=None, flags=0, window=None):
        """Queue a render whose image is copied into pinned host memory (a
        pinned tensor or numpy array) while later frames render; the image is
        valid after wait_host()."""
        prm = params_struct(params, flags, window)
        cam = camera_struct(camera)
        ptr = out_host.ctypes.data if isinstance(out_host, np.ndarray) else out_host.data_ptr()
        _check(load().ivv_render_to_host_async(self.h, C.byref(cam), C.byref(prm), width, height, C.c_void_p(ptr),
                                               C.c_void_p(_stream_ptr(stream))))
        return out_host

    def wait_host(self):
        """Block until every image queued by render_to_host_async is on the host."""
        _check(load().ivv_render_to_host_wait(self.h))

    def render_pairs(self, camera, params, width, height, max_pairs=16, stream=None, flags=0):
        """Stages 1-2: per-pixel entry/exit pairs (counts [H*W], pairs [M][H*W][8], blocks [M][H*W])."""
        import torch
        npix = width * height
        cnt = torch.empty(npix, dtype=torch.int32, device="cuda")
        pairs = torch.zeros((max_pairs, npix, 8), dtype=torch.float32, device="cuda")
        blk = torch.zeros((max_pairs, npix), dtype=torch.int32, device="cuda")
        prm = params_struct(params, flags)
        ws, need = self.workspace(width, height, prm.precision)
        cam = camera_struct(camera)
        _check(load().ivv_render_pairs(self.h, C.byref(cam), C.byref(prm), width, height, max_pairs,
                                       C.c_void_p(cnt.data_ptr()), C.c_void_p(pairs.data_ptr()),
                                       C.c_void_p(blk.data_ptr()), C.c_void_p(ws), need,
                                       C.c_void_p(_stream_ptr(stream))))
        return cnt, pairs, blk

    def eval_points(self, block, p, stream=None):
        """phi [n][3], J [n][3][3], rho [n] at float32 CUDA points p [n][3]."""
        import torch
        p = p.contiguous()
        n = p.shape[0]
        phi = torch.empty((n, 3), dtype=torch.float32, device=p.device)
        jac = torch.empty((n, 3, 3), dtype=torch.float32, device=p.device)
        rho = torch.empty(n, dtype=torch.float32, device=p.device)
        _check(load().ivv_eval_points(self.h, block, n, C.c_void_p(p.data_ptr()), C.c_void_p(phi.data_ptr()),
                                      C.c_void_p(jac.data_ptr()), C.c_void_p(rho.data_ptr()),
                                      C.c_void_p(_stream_ptr(stream))))
        return phi, jac, rho

    def stage_times(self):
        """{stage: ms} of the last render made with FLAG_TIMING."""
        ms = (C.c_float * len(STAGES))()
        _check(load().ivv_get_stage_times(self.h, ms))
        return dict(zip(STAGES, list(ms)))

    # ---- learned initial guess
    def train_guess(self, samples_per_block=1 << 20, epochs=8, batch=4096, lr=3e-3, seed=1, stream=None):
        """Train every block's guess network on the device; returns the final
        mean squared error per block."""
        nb = self.info()["n_blocks"]
        out = (C.c_float * nb)()
        prm = GuessTrainParams(samples_per_block, epochs, batch, lr, seed)
        _check(load().ivv_train_guess(self.h, C.byref(prm), out, C.c_void_p(_stream_ptr(stream))))
        return list(out)

    def guess_points(self, g4, block_of, stream=None):
        """Tensor-core guess p_hat [n][4] for CUDA tensors g4 [n][4] (float32)
        and block_of [n] (int32)."""
        import torch
        g4 = g4.contiguous()
        block_of = block_of.contiguous()
        out = torch.empty_like(g4)
        _check(load().ivv_guess_points(self.h, g4.shape[0], C.c_void_p(g4.data_ptr()), C.c_void_p(block_of.data_ptr()),
                                       C.c_void_p(out.data_ptr()), C.c_void_p(_stream_ptr(stream))))
        return out

    def invert_points(self, g4, block_of, guess=0, tol=1e-5, stream=None):
        """(p [n][4] with the final residual in column 3, iterations [n]) of the
        batched Newton inversion from the chosen initial guess."""
        import torch
        g4 = g4.contiguous()
        block_of = block_of.contiguous()
        out = torch.empty_like(g4)
        its = torch.empty(g4.shape[0], dtype=torch.int32, device=g4.device)
        _check(load().ivv_invert_points(self.h, g4.shape[0], C.c_void_p(g4.data_ptr()), C.c_void_p(block_of.data_ptr()),
                                        int(guess), float(tol), C.c_void_p(out.data_ptr()), C.c_void_p(its.data_ptr()),
                                        C.c_void_p(_stream_ptr(stream))))
        return out, its

    def guess_loss_grad(self, block, x4, p4, stream=None):
        """(loss, gradient) of the device training kernel on one batch."""
        grad = np.zeros(GUESS_PARAMS, np.float32)
        loss = C.c_float()
        _check(load().ivv_guess_loss_grad(self.h, block, x4.shape[0], C.c_void_p(x4.contiguous().data_ptr()),
                                          C.c_void_p(p4.contiguous().data_ptr()), grad.ctypes.data_as(c_float_p),
                                          C.byref(loss), C.c_void_p(_stream_ptr(stream))))
        return loss.value, grad

    def get_guess_weights(self, block):
        w = np.zeros(GUESS_PARAMS, np.float32)
        c = np.zeros(3, np.float32)
        ih = np.zeros(3, np.float32)
        _check(load().ivv_get_guess_weights(self.h, block, w.ctypes.data_as(c_float_p), c.ctypes.data_as(c_float_p),
                                            ih.ctypes.data_as(c_float_p)))
        return w, c, ih

    def set_guess_weights(self, block, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        _check(load().ivv_set_guess_weights(self.h, block, w.ctypes.data_as(c_float_p)))

    def stats(self):
        s = Stats()
        _check(load().ivv_get_stats(self.h, C.byref(s)))
        return s.as_dict()

    def set_limits(self, **kw):
        """Capacities and caps (ivv_limits); unnamed fields keep their value;
        no arguments restores the defaults."""
        if not kw:
            _check(load().ivv_set_limits(self.h, None))
            return
        lim = Limits()
        _check(load().ivv_get_limits(self.h, C.byref(lim)))
        for k, v in kw.items():
            setattr(lim, k, int(v))
        _check(load().ivv_set_limits(self.h, C.byref(lim)))

    def limits(self):
        lim = Limits()
        _check(load().ivv_get_limits(self.h, C.byref(lim)))
        return {n: getattr(lim, n) for n, _ in Limits._fields_}

    def check_frame(self):
        """(status, message) of the renders since the last check: IVV_OK,
        IVV_ERR_ABUF_OVERFLOW or IVV_ERR_NONCONVERGED."""
        st = load().ivv_check_frame(self.h)
        return st, load().ivv_last_error().decode(errors="replace") if st != IVV_OK else ""

    def reset_stats(self):
        _check(load().ivv_reset_stats(self.h))


def volume_for(scene, stream=None) -> Volume:
    v = Volume(scene.blocks, scene.scalar_mode, stream)
    v.set_transfer_function(scene.tf)
    return v


class Batch:
    """Many render requests rendered together (one launch per stage, replayed
    from a CUDA graph).  items: sequence of (volume, camera, width, height, tf)
    with tf a TransferFunction or None (the volume's own); outputs are float32
    [H][W][4] CUDA tensors in self.outputs (given ones are used as they are)."""

    def __init__(self, items, params=None, outputs=None, stream=None):
        import torch
        L = load()
        n = len(items)
        reqs = (Request * n)()
        keep = []
        self.outputs = []
        for i, (vol, cam, w, h, tf) in enumerate(items):
            out = outputs[i] if outputs is not None else torch.empty((h, w, 4), dtype=torch.float32, device="cuda")
            self.outputs.append(out)
            q = reqs[i]
            q.volume = vol.h.value
            q.camera = camera_struct(cam)
            q.width, q.height = int(w), int(h)
            q.out_rgba = out.data_ptr()
            if tf is not None:
                r = np.ascontiguousarray(tf.r, dtype=np.float32)
                rgba = np.ascontiguousarray(tf.rgba, dtype=np.float32)
                keep += [r, rgba]
                q.tf_n = len(r)
                q.tf_r = r.ctypes.data_as(c_float_p)
                q.tf_rgba = rgba.ctypes.data_as(c_float_p)
                q.tf_sigma = float(tf.sigma)
                q.scalar_lo = tf.lo if math.isfinite(tf.lo) else float("nan")
                q.scalar_hi = tf.hi if math.isfinite(tf.hi) else float("nan")
        prm = params_struct(params)
        h = C.c_void_p()
        _check(L.ivv_batch_create(reqs, n, C.byref(prm), C.c_void_p(_stream_ptr(stream)), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            load().ivv_batch_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def render(self, flags=0, stream=None):
        _check(load().ivv_batch_render(self.h, int(flags), C.c_void_p(_stream_ptr(stream))))
        return self.outputs

    def set_camera(self, i, camera, stream=None):
        cam = camera_struct(camera)
        _check(load().ivv_batch_set_camera(self.h, int(i), C.byref(cam), C.c_void_p(_stream_ptr(stream))))

    @property
    def tuning(self):
        t = BatchTuning()
        _check(load().ivv_batch_get_tuning(self.h, C.byref(t)))
        return t.as_dict()

    @tuning.setter
    def tuning(self, d):
        t = BatchTuning(int(d["tile_w"]), int(d["tile_h"]), int(d["k5_ctas_per_sm"]), int(d["step_samples"]))
        _check(load().ivv_batch_set_tuning(self.h, C.byref(t)))

    def autotune(self, reps=3, stream=None):
        """Time the candidate launch shapes; applies and returns (tuning, ms per frame)."""
        t = BatchTuning()
        ms = C.c_float()
        _check(load().ivv_batch_autotune(self.h, int(reps), C.byref(t), C.byref(ms),
                                         C.c_void_p(_stream_ptr(stream))))
        return t.as_dict(), ms.value

    def stats(self):
        s = Stats()
        _check(load().ivv_batch_get_stats(self.h, C.byref(s)))
        return s.as_dict()

    def reset_stats(self):
        _check(load().ivv_batch_reset_stats(self.h))

    def stage_times(self):
        ms = (C.c_float * len(STAGES))()
        _check(load().ivv_batch_get_stage_times(self.h, ms))
        return dict(zip(STAGES, list(ms)))

    def info(self):
        n, px, ws, g = C.c_int(), C.c_longlong(), C.c_size_t(), C.c_int()
        _check(load().ivv_batch_info(self.h, C.byref(n), C.byref(px), C.byref(ws), C.byref(g)))
        return {"n_requests": n.value, "n_pixels": px.value, "workspace_bytes": ws.value, "graph_ready": bool(g.value)}
