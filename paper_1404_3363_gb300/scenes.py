"""Seeded synthetic inputs: spline volumes, transfer functions, cameras.

This module only *builds inputs*.  It holds none of the rendering arithmetic
(no spline evaluation, no intersection, no inversion, no compositing), so both
the CUDA path and the FP64 CPU oracle can consume the same inputs without
sharing any of the method.

The paper's three application models (twisted bar, TERRIFIC demonstrator,
backstep CFD; §6) are not available, so the workloads below are seeded
stand-ins with the same workload classes:

* ``twisted_cube``   one cubic Bezier element, unit cube twisted 90 deg (4^3 cp).
* ``twisted_bar``    single-block cubic B-spline bar 1x1x8 twisted 180 deg,
                     8x8x32 control points, open uniform knots; scalar field is
                     the parametrisation quality of §6.1 (Eq. 23), derived on
                     the fly (no scalar control points).
* ``bent_beam``      16 cubic blocks (2x2x4) of 6x6x12 cp, C0 across shared
                     faces, bent 60 deg; scalar = sum of 8 Gaussians.
* ``backstep``       3 blocks of a backward-facing-step channel, quadratic,
                     64x16x16 control points in total, stretched grid; scalar
                     is a sharp tanh shear layer with seeded Perlin noise.

Scalar control points are set by Schoenberg quasi-interpolation (the field's
value at each control point's Greville abscissa), so no spline arithmetic is
needed here.

Every generator takes a seed; the default seed of config ``i`` is 12345 + i.
Random numbers come from numpy's PCG64 (``numpy.random.default_rng``).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

SCALAR_CP = 0       # rho from scalar control points
SCALAR_DETJ = 1     # rho = det J_phi
SCALAR_QUALITY = 2  # rho = det J_phi / ||J_phi||_F  (Eq. 23)
SCALAR_VONMISES = 3  # rho = von Mises value of the strain of a displacement u (§6.2, Eq. 24)

PRECISION_FP32 = 0
PRECISION_MIXED = 1
PRECISION_FP64 = 2


@dataclasses.dataclass
class Block:
    """One volume block: tensor-product B-spline geometry (and scalar)."""
    degree: tuple          # (p_u, p_v, p_w)
    knots: List[np.ndarray]  # 3 float64 arrays, len n_cp[d] + degree[d] + 1
    geom_cp: np.ndarray    # float64 [n_w][n_v][n_u][3], u fastest
    scalar_cp: Optional[np.ndarray] = None  # float64 [n_w][n_v][n_u]
    disp_cp: Optional[np.ndarray] = None    # float64 [n_w][n_v][n_u][3], displacement u (§6.2)

    @property
    def n_cp(self):
        nw, nv, nu = self.geom_cp.shape[:3]
        return (nu, nv, nw)


@dataclasses.dataclass
class TransferFunction:
    """Piecewise-linear RGBA over normalised scalar r in [0,1].

    A is an extinction weight in [0,1]; sigma scales it.  lo/hi map the scalar
    to r; NaN means "library default" (see the boundary header).
    """
    r: np.ndarray       # float32 [n], ascending, r[0]=0, r[-1]=1
    rgba: np.ndarray    # float32 [n][4]
    sigma: float
    lo: float = float("nan")
    hi: float = float("nan")


@dataclasses.dataclass
class Camera:
    ortho: bool
    eye: tuple
    target: tuple
    up: tuple
    fovy_deg: float = 35.0
    ortho_height: float = 1.0


@dataclasses.dataclass
class RenderParams:
    rk_tol: float = 1e-5
    ds: float = 0.0            # sample distance in G; <= 0 means diag/128
    supersample_k: int = 4
    c: float = 1.0
    early_alpha: float = 1.0 - 1e-4
    precision: int = PRECISION_FP32
    use_mlp_guess: int = 0
    method: int = 0            # 0: ODE (§5.2), 1: per-sample root finding (§5.1)
    rf_tol: float = 0.05       # RF stop: fraction of the pixel half width
    rk_method: int = 0         # 0: BS3(2) with error control; 1-6: fixed-step family of §5.2-5.3
    near_clip: float = 0.0     # > 0: near plane at this distance along the view direction (§5.5)
    cut_planes: tuple = ()     # up to 4 (n_x, n_y, n_z, w): points with n.g + w > 0 are cut away (§5.5)


@dataclasses.dataclass
class Scene:
    name: str
    blocks: List[Block]
    scalar_mode: int
    tf: TransferFunction
    camera: Camera
    width: int
    height: int
    params: RenderParams

    def cp_bbox(self):
        pts = np.concatenate([b.geom_cp.reshape(-1, 3) for b in self.blocks])
        return pts.min(0), pts.max(0)

    def cp_diag(self):
        lo, hi = self.cp_bbox()
        return float(np.linalg.norm(hi - lo))

    def with_size(self, width, height):
        return dataclasses.replace(self, width=int(width), height=int(height))


# ---------------------------------------------------------------- helpers

def open_uniform_knots(n_cp: int, degree: int) -> np.ndarray:
    """Clamped (open) uniform knot vector on [0,1] with n_cp - degree spans."""
    spans = n_cp - degree
    inner = np.arange(1, spans) / spans
    return np.concatenate([np.zeros(degree + 1), inner, np.ones(degree + 1)])


def greville(knots: np.ndarray, degree: int) -> np.ndarray:
    """Greville abscissae: averages of `degree` consecutive interior knots."""
    n = len(knots) - degree - 1
    if degree == 0:
        return 0.5 * (knots[:n] + knots[1:n + 1])
    return np.array([knots[i + 1:i + degree + 1].mean() for i in range(n)])


def _grid(gu, gv, gw):
    """[n_w][n_v][n_u][3] array of (u, v, w) Greville points."""
    W, V, U = np.meshgrid(gw, gv, gu, indexing="ij")
    return np.stack([U, V, W], axis=-1)


def _random_tf(rng, n=8, sigma=4.0, a_min=0.0, min_gap=0.0):
    r = np.sort(rng.uniform(0, 1, n - 2))
    if min_gap > 0:
        # spread the sorted interior knots to at least min_gap apart (and from
        # 0 and 1) without drawing again: r_i -> i*g + (1 - (n-1) g) r_i
        r = min_gap * np.arange(1, n - 1) + (1.0 - (n - 1) * min_gap) * r
    r = np.concatenate([[0.0], r, [1.0]])
    rgba = rng.uniform(0, 1, (n, 4))
    if a_min > 0:
        rgba[:, 3] = a_min + (1 - a_min) * rgba[:, 3]
    return TransferFunction(r.astype(np.float32), rgba.astype(np.float32), float(sigma))


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def _random_dir(rng):
    z = rng.uniform(-1, 1)
    a = rng.uniform(0, 2 * math.pi)
    s = math.sqrt(max(0.0, 1 - z * z))
    return np.array([s * math.cos(a), s * math.sin(a), z])


def _ortho_camera_for(blocks, rng, dist_diag=3.0, height_scale=1.1):
    pts = np.concatenate([b.geom_cp.reshape(-1, 3) for b in blocks])
    lo, hi = pts.min(0), pts.max(0)
    centre = 0.5 * (lo + hi)
    diag = float(np.linalg.norm(hi - lo))
    d = _random_dir(rng)
    up = np.array([0.0, 0.0, 1.0])
    if abs(d[2]) > 0.95:
        up = np.array([0.0, 1.0, 0.0])
    eye = centre + dist_diag * diag * d
    return Camera(True, tuple(eye), tuple(centre), tuple(up),
                  ortho_height=height_scale * diag)


def _perspective_camera(centre, dist, elev_deg, azim, fovy=35.0, up_axis=2):
    e = math.radians(elev_deg)
    axes = [0, 1, 2]
    axes.remove(up_axis)
    dvec = np.zeros(3)
    dvec[axes[0]] = math.cos(e) * math.cos(azim)
    dvec[axes[1]] = math.cos(e) * math.sin(azim)
    dvec[up_axis] = math.sin(e)
    eye = np.asarray(centre) + dist * dvec
    up = np.zeros(3)
    up[up_axis] = 1.0
    return Camera(False, tuple(eye), tuple(centre), tuple(up), fovy_deg=fovy)


def _default_ds(blocks):
    pts = np.concatenate([b.geom_cp.reshape(-1, 3) for b in blocks])
    return float(np.linalg.norm(pts.max(0) - pts.min(0))) / 128.0


# ---------------------------------------------------------------- configs

def twisted_cube(seed: int = 12345, width: int = 64, height: int = 64,
                 precision: int = PRECISION_FP64) -> Scene:
    """Single cubic Bezier element (4x4x4 cp) of the unit cube twisted 90 deg
    about the axis x=y=0.5 (angle proportional to z), plus U(-0.02,0.02)
    jitter; scalar: 64 coefficients ~U(0,1); 8-knot TF with sigma=4;
    orthographic camera from a seeded direction."""
    rng = np.random.default_rng(seed)
    kn = np.array([0, 0, 0, 0, 1, 1, 1, 1], dtype=np.float64)
    g = np.linspace(0, 1, 4)
    P = _grid(g, g, g)                      # [w][v][u][3] = (u, v, w)
    th = 0.5 * math.pi * P[..., 2]
    x, y = P[..., 0] - 0.5, P[..., 1] - 0.5
    cp = np.stack([0.5 + x * np.cos(th) - y * np.sin(th),
                   0.5 + x * np.sin(th) + y * np.cos(th),
                   P[..., 2]], axis=-1)
    cp = cp + rng.uniform(-0.02, 0.02, cp.shape)
    scal = rng.uniform(0, 1, (4, 4, 4))
    blk = Block((3, 3, 3), [kn.copy(), kn.copy(), kn.copy()], cp, scal)
    tf = _random_tf(rng, 8, 4.0)
    cam = _ortho_camera_for([blk], rng)
    params = RenderParams(rk_tol=1e-8, ds=_default_ds([blk]), precision=precision)
    return Scene("twisted_cube", [blk], SCALAR_CP, tf, cam, width, height, params)


def twisted_bar(seed: int = 12346, width: int = 1920, height: int = 1080,
                scalar_mode: int = SCALAR_QUALITY,
                precision: int = PRECISION_FP32) -> Scene:
    """Cubic B-spline bar, 8x8x32 cp, open uniform knots; control points at
    the Greville points of the box [0,1]x[0,1]x[0,8] twisted by pi*z/8 about
    the box axis.  Scalar: parametrisation quality (Eq. 23) or det J.
    Perspective camera at distance 14 from the centre, elevation 15-35 deg,
    seeded azimuth, fovy 35 deg."""
    rng = np.random.default_rng(seed)
    p = 3
    ku, kv, kw = (open_uniform_knots(8, p), open_uniform_knots(8, p),
                  open_uniform_knots(32, p))
    P = _grid(greville(ku, p), greville(kv, p), 8.0 * greville(kw, p))
    th = math.pi * P[..., 2] / 8.0
    x, y = P[..., 0] - 0.5, P[..., 1] - 0.5
    cp = np.stack([0.5 + x * np.cos(th) - y * np.sin(th),
                   0.5 + x * np.sin(th) + y * np.cos(th),
                   P[..., 2]], axis=-1)
    blk = Block((p, p, p), [ku, kv, kw], cp, None)
    tf = _random_tf(rng, 8, 4.0)
    elev = rng.uniform(15, 35)
    azim = rng.uniform(0, 2 * math.pi)
    cam = _perspective_camera((0.5, 0.5, 4.0), 14.0, elev, azim, 35.0)
    params = RenderParams(rk_tol=1e-5, ds=_default_ds([blk]), precision=precision)
    return Scene("twisted_bar", [blk], scalar_mode, tf, cam, width, height, params)


def bent_beam(seed: int = 12347, width: int = 1920, height: int = 1080,
              precision: int = PRECISION_MIXED, displacement: bool = False) -> Scene:
    """16 cubic blocks (2x2 cross-section, 4 along) of the beam
    [0,1]^2 x [0,8], each 6x6x12 cp, sharing face control points (C0); the
    global net is jittered by U(-a,a), a = 0.5% of the smallest block edge,
    then bent 60 deg about the y axis along a circular arc.  Scalar: sum of 8
    seeded Gaussians on the unbent beam, quasi-interpolated at Greville
    points.  The TF leaves r in [0,0.4] transparent.

    displacement=True adds a displacement spline per block and renders its
    von Mises value (§6.2): a cantilever clamped at z = 0 under a tip load
    along x (Euler-Bernoulli: deflection w(z) = delta (z/L)^2 (3 - z/L) / 2,
    axial u_z = -(x - 1/2) w'(z), delta = 0.05), plus three seeded
    sinusoids of amplitude delta/5 per component (generator seed + 1000),
    taken at the Greville points of the unbent beam and turned with the bend
    into world axes."""
    rng = np.random.default_rng(seed)
    p = 3
    nb = (2, 2, 4)
    ncp = (6, 6, 12)
    ext = (1.0, 1.0, 8.0)
    kn = [open_uniform_knots(n, p) for n in ncp]
    gr = [greville(kn[d], p) for d in range(3)]
    # global Greville positions of the assembled C0 net
    glob = []
    for d in range(3):
        seg = ext[d] / nb[d]
        pts = []
        for b in range(nb[d]):
            g = b * seg + seg * gr[d]
            pts.extend(g if b == 0 else g[1:])
        glob.append(np.array(pts))
    G = _grid(glob[0], glob[1], glob[2])    # [Nw][Nv][Nu][3]
    a = 0.005 * min(e / n for e, n in zip(ext, nb))
    Gj = G + rng.uniform(-a, a, G.shape)
    # bend: arc of angle 60 deg over the beam length, about the y axis
    ang = math.pi / 3.0
    R = ext[2] / ang
    th = Gj[..., 2] / R
    rr = R + (Gj[..., 0] - 0.5)
    bent = np.stack([0.5 + rr * np.cos(th) - R, Gj[..., 1], rr * np.sin(th)], axis=-1)
    # scalar field on the unbent, un-jittered beam coordinates
    cen = np.stack([rng.uniform(0, 1, 8), rng.uniform(0, 1, 8), rng.uniform(0, 8, 8)], 1)
    sig = rng.uniform(0.1, 0.3, 8) * 1.0
    amp = rng.uniform(0.5, 1.0, 8)
    f = np.zeros(G.shape[:3])
    for k in range(8):
        f += amp[k] * np.exp(-np.sum((G - cen[k]) ** 2, -1) / (2 * sig[k] ** 2))
    U = None
    if displacement:
        drng = np.random.default_rng(seed + 1000)
        L, delta = ext[2], 0.05
        zl = G[..., 2] / L
        w = delta * zl ** 2 * (3.0 - zl) / 2.0
        dw = delta * 3.0 * zl * (2.0 - zl) / (2.0 * L)
        loc = np.stack([w, np.zeros_like(w), -(G[..., 0] - 0.5) * dw], -1)
        for _ in range(3):
            kv = _random_dir(drng) * drng.uniform(0.5, 2.0)
            loc += (0.2 * delta * drng.uniform(-1, 1, 3)) * np.sin(G @ kv + drng.uniform(0, 2 * math.pi))[..., None]
        ct, st_ = np.cos(G[..., 2] / R), np.sin(G[..., 2] / R)
        U = np.stack([loc[..., 0] * ct - loc[..., 2] * st_, loc[..., 1], loc[..., 0] * st_ + loc[..., 2] * ct], -1)
    blocks = []
    for bw in range(nb[2]):
        for bv in range(nb[1]):
            for bu in range(nb[0]):
                su = slice(bu * (ncp[0] - 1), bu * (ncp[0] - 1) + ncp[0])
                sv = slice(bv * (ncp[1] - 1), bv * (ncp[1] - 1) + ncp[1])
                sw = slice(bw * (ncp[2] - 1), bw * (ncp[2] - 1) + ncp[2])
                blocks.append(Block((p, p, p), [k.copy() for k in kn],
                                    bent[sw, sv, su].copy(), f[sw, sv, su].copy(),
                                    U[sw, sv, su].copy() if U is not None else None))
    r = np.concatenate([[0.0, 0.4], np.sort(rng.uniform(0.4, 1.0, 5)), [1.0]])
    rgba = rng.uniform(0, 1, (8, 4))
    rgba[:2, 3] = 0.0
    rgba[2:, 3] = 0.2 + 0.8 * rgba[2:, 3]
    tf = TransferFunction(r.astype(np.float32), rgba.astype(np.float32), 4.0)
    pts = bent.reshape(-1, 3)
    centre = 0.5 * (pts.min(0) + pts.max(0))
    cam = _perspective_camera(centre, 14.0, rng.uniform(15, 35),
                              rng.uniform(0, 2 * math.pi), 35.0, up_axis=1)
    params = RenderParams(rk_tol=1e-5, ds=_default_ds(blocks), precision=precision)
    if displacement:
        return Scene("loaded_beam", blocks, SCALAR_VONMISES, tf, cam, width, height, params)
    return Scene("bent_beam", blocks, SCALAR_CP, tf, cam, width, height, params)


def _perlin3(rng, pts, freq=4.0):
    """Seeded 3-D gradient (Perlin) noise in [-1,1] at points [..., 3]."""
    perm = rng.permutation(256)
    perm = np.concatenate([perm, perm])
    grads = rng.normal(size=(256, 3))
    grads /= np.linalg.norm(grads, axis=1, keepdims=True)
    q = pts * freq
    i0 = np.floor(q).astype(np.int64)
    fr = q - i0
    fade = fr * fr * fr * (fr * (fr * 6 - 15) + 10)
    out = np.zeros(pts.shape[:-1])
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                ix = (i0[..., 0] + dx) & 255
                iy = (i0[..., 1] + dy) & 255
                iz = (i0[..., 2] + dz) & 255
                h = perm[perm[perm[ix] + iy] + iz]
                off = fr - np.array([dx, dy, dz])
                dot = np.sum(grads[h] * off, -1)
                wx = fade[..., 0] if dx else 1 - fade[..., 0]
                wy = fade[..., 1] if dy else 1 - fade[..., 1]
                wz = fade[..., 2] if dz else 1 - fade[..., 2]
                out += wx * wy * wz * dot
    return np.clip(out * 1.5, -1, 1)


def backstep(seed: int = 12349, width: int = 3840, height: int = 2160,
             precision: int = PRECISION_MIXED) -> Scene:
    """Backward-facing-step channel of height 1 with step height 0.5: an
    inlet block x in [-1,0], y in [0.5,1] (16x8x16 cp) and two outlet blocks
    x in [0,3] above and below y=0.5 (48x8x16 cp each), span z in [0,1];
    quadratic, x spacing stretched towards the step.  Scalar: turbulent
    viscosity-like 1e-5 + 1e-2 (1+tanh((y-h(x))/0.01))/2 (1 + 0.2 Perlin)."""
    rng = np.random.default_rng(seed)
    p = 2

    def stretch_out(g):          # cluster near x = 0 (the step)
        return 3.0 * g ** 1.5

    def stretch_in(g):           # cluster near x = 0 from the inlet side
        return -1.0 * (1.0 - g) ** 1.5

    specs = [(16, 8, 16, stretch_in, (0.5, 1.0)),
             (48, 8, 16, stretch_out, (0.5, 1.0)),
             (48, 8, 16, stretch_out, (0.0, 0.5))]
    noise_rng = np.random.default_rng(seed + 1000)
    perm_state = noise_rng.bit_generator.state
    blocks = []
    for nu, nv, nw, sx, (y0, y1) in specs:
        kn = [open_uniform_knots(n, p) for n in (nu, nv, nw)]
        gu, gv, gw = (greville(kn[d], p) for d in range(3))
        P = _grid(sx(gu), y0 + (y1 - y0) * gv, gw)
        x, y = P[..., 0], P[..., 1]
        h = np.where(x < 0, 0.5, 0.5 - 0.5 * np.clip(x / 3.0, 0, 1) ** 0.8)
        noise_rng.bit_generator.state = perm_state
        nz = _perlin3(noise_rng, P, 3.0)
        f = 1e-5 + 1e-2 * 0.5 * (1 + np.tanh((y - h) / 0.01)) * (1 + 0.2 * nz)
        blocks.append(Block((p, p, p), kn, P.copy(), f))
    r = np.concatenate([[0.0], np.sort(rng.uniform(0, 1, 62)), [1.0]])
    rgba = rng.uniform(0, 1, (64, 4))
    rgba[:, 3] = 0.05 + 0.95 * rgba[:, 3] ** 2
    tf = TransferFunction(r.astype(np.float32), rgba.astype(np.float32), 4.0)
    cam = _perspective_camera((1.0, 0.5, 0.5), 6.5, rng.uniform(20, 35),
                              rng.uniform(0.3, 1.2) + math.pi, 35.0, up_axis=1)
    # rk_tol 7e-7: at 1e-6 the embedded pair's along-ray drift (the field of
    # Eq. 10 does not pull it back) puts a few pixels of the shear layer
    # 1.1e-3 off the exact image; 7e-7 keeps every sampled pixel within 1e-3
    params = RenderParams(rk_tol=7e-7, ds=_default_ds(blocks), precision=precision)
    return Scene("backstep", blocks, SCALAR_CP, tf, cam, width, height, params)


def degenerate_cube(seed: int = 12350, width: int = 256, height: int = 256, precision: int = PRECISION_FP32,
                    twist: float = 0.5 * math.pi, jitter: float = 0.02, scalar=None, direction=(0.35, 0.25, 0.9),
                    ortho: bool = True) -> Scene:
    """Cubic Bezier element (4x4x4 cp) of the unit cube, twisted by `twist`
    about the axis x=y=0.5, whose three upper control-point layers coincide
    (the top layer repeated, as a designer's collapsed layers): z(w) =
    1 - (1 - w)^3, so d phi / d w and det J vanish on the whole top face w = 1
    (a singular Jacobian on the boundary, §5.4).  Jitter U(-jitter, jitter)
    per control point of the bottom layer and of the (shared) top layer;
    scalar control points U(0,1) (or the constant `scalar`); 8-knot TF,
    sigma = 4; camera looking down along -direction so that rays enter
    through the top face."""
    rng = np.random.default_rng(seed)
    kn = np.array([0, 0, 0, 0, 1, 1, 1, 1], dtype=np.float64)
    g = np.linspace(0, 1, 4)
    P = _grid(g, g, g)
    P[..., 2] = np.where(P[..., 2] > 0, 1.0, 0.0)           # layers k = 1, 2, 3 at z = 1
    th = twist * P[..., 2]
    x, y = P[..., 0] - 0.5, P[..., 1] - 0.5
    cp = np.stack([0.5 + x * np.cos(th) - y * np.sin(th),
                   0.5 + x * np.sin(th) + y * np.cos(th),
                   P[..., 2]], axis=-1)
    jit = rng.uniform(-jitter, jitter, (2, 4, 4, 3))
    cp[0] += jit[0]
    cp[1:] += jit[1][None]                                   # the top layers stay coincident
    scal = np.full((4, 4, 4), float(scalar)) if scalar is not None else rng.uniform(0, 1, (4, 4, 4))
    blk = Block((3, 3, 3), [kn.copy(), kn.copy(), kn.copy()], cp, scal)
    tf = _random_tf(rng, 8, 4.0)
    pts = cp.reshape(-1, 3)
    lo, hi = pts.min(0), pts.max(0)
    centre, diag = 0.5 * (lo + hi), float(np.linalg.norm(hi - lo))
    dvec = _unit(direction)
    up = np.array([0.0, 1.0, 0.0]) if abs(dvec[1]) < 0.9 else np.array([1.0, 0.0, 0.0])
    if ortho:
        cam = Camera(True, tuple(centre + 3 * diag * dvec), tuple(centre), tuple(up), ortho_height=1.1 * diag)
    else:
        cam = Camera(False, tuple(centre + 2.2 * diag * dvec), tuple(centre), tuple(up), fovy_deg=35.0)
    params = RenderParams(rk_tol=1e-5, ds=_default_ds([blk]), precision=precision)
    return Scene("degenerate_cube", [blk], SCALAR_CP, tf, cam, width, height, params)


CONFIG_BUILDERS = {0: twisted_cube, 1: twisted_bar, 2: bent_beam, 4: backstep}


def config(i: int, **kw) -> Scene:
    """Scene for workload index i (0, 1, 2, 4) with its default seed."""
    return CONFIG_BUILDERS[i](seed=12345 + i, **kw)


@dataclasses.dataclass
class Request:
    volume: int          # 0, 1 or 2: which of the three volumes
    width: int
    height: int
    camera: Camera
    tf: TransferFunction


def batch_requests(seed: int = 12348, n: int = 64):
    """64 render requests over the volumes of workloads 0-2, sizes uniform
    over {256,512,768,1024}^2, seeded cameras and transfer functions.

    The transfer functions' knots lie at least 1/64 apart, so that no segment
    is steeper than 64 per unit of normalised scalar.  A near-step (two knots
    ~1e-4 apart) multiplies the few-ulp FP32 error of the scalar by ~7000 on
    the twisted bar, whose scalar spans a narrow range, which no FP32 sampler
    holds to 1e-3 in RGBA."""
    rng = np.random.default_rng(seed)
    vols = [twisted_cube(), twisted_bar(), bent_beam()]
    reqs = []
    for _ in range(n):
        v = int(rng.integers(0, 3))
        s = int(rng.choice([256, 512, 768, 1024]))
        blocks = vols[v].blocks
        pts = np.concatenate([b.geom_cp.reshape(-1, 3) for b in blocks])
        lo, hi = pts.min(0), pts.max(0)
        centre = 0.5 * (lo + hi)
        diag = float(np.linalg.norm(hi - lo))
        d = _random_dir(rng)
        up = np.array([0.0, 0.0, 1.0]) if abs(d[2]) < 0.95 else np.array([0.0, 1.0, 0.0])
        cam = Camera(False, tuple(centre + 1.6 * diag * d), tuple(centre), tuple(up),
                     fovy_deg=float(rng.uniform(30, 45)))
        reqs.append(Request(v, s, s, cam, _random_tf(rng, 8, 4.0, min_gap=1.0 / 64)))
    return vols, reqs
