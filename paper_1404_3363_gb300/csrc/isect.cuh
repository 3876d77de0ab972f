// Per-ray work of stages 1 and 2, written once for the device kernels and the
// host inspection entry point (ivv_host_pixel_pairs):
//   * face_screen_box  -- conservative pixel box of a face patch (convex hull
//                          of its control points projected to the screen);
//   * patch_roots       -- all parameters (a,b) where a Bezier face patch meets
//                          a ray: control points are expressed in a 2-D frame
//                          perpendicular to the ray, so roots are zeros of a
//                          planar Bezier map.  A sub-patch whose hull misses the
//                          origin is dropped; one whose Jacobian sign is fixed
//                          (interval bound over its hodographs) holds at most one
//                          root and is solved by damped Newton from its centre;
//                          otherwise it is split at 1/2 (de Casteljau) down to a
//                          fixed depth;
//   * make_fragment     -- 3-D point, depth t, facing and block parameter point
//                          of a root;
//   * pair_fragments    -- depth sort, duplicate merge and Alg. 2 of §4.2.
#pragma once

#include <cuda_runtime.h>

#include <math.h>

#include "ivv_internal.h"

namespace ivv {

#ifndef IVV_HD
#define IVV_HD __host__ __device__ __forceinline__
#endif

template <typename R> IVV_HD R clamp01r(R x) { return x < R(0) ? R(0) : (x > R(1) ? R(1) : x); }
template <typename R> IVV_HD R minr(R a, R b) { return a < b ? a : b; }
template <typename R> IVV_HD R maxr(R a, R b) { return a > b ? a : b; }

template <int P, typename R>
IVV_HD void bern_hd(R x, R b[P + 1], R db[P + 1]) {
  const R y = R(1) - x;
  if (P == 2) {
    b[0] = y * y; b[1] = R(2) * x * y; b[2] = x * x;
    db[0] = R(-2) * y; db[1] = R(2) - R(4) * x; db[2] = R(2) * x;
  } else {
    const R x2 = x * x, y2 = y * y;
    b[0] = y2 * y; b[1] = R(3) * x * y2; b[2] = R(3) * x2 * y; b[3] = x2 * x;
    db[0] = R(-3) * y2; db[1] = R(3) * y * (R(1) - R(3) * x);
    db[2] = R(3) * x * (R(2) - R(3) * x); db[3] = R(3) * x2;
  }
}

// ------------------------------------------------------------ ray frame
template <typename R>
IVV_HD void ray_frame(const R d[3], R e1[3], R e2[3]) {
  R ax[3] = {R(1), R(0), R(0)};
  if (fabs(d[0]) > R(0.6)) { ax[0] = R(0); ax[1] = R(1); }
  e1[0] = d[1] * ax[2] - d[2] * ax[1];
  e1[1] = d[2] * ax[0] - d[0] * ax[2];
  e1[2] = d[0] * ax[1] - d[1] * ax[0];
  const R n = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  e1[0] /= n; e1[1] /= n; e1[2] /= n;
  e2[0] = d[1] * e1[2] - d[2] * e1[1];
  e2[1] = d[2] * e1[0] - d[0] * e1[2];
  e2[2] = d[0] * e1[1] - d[1] * e1[0];
}


// ------------------------------------------------------------ camera
template <typename R>
struct DevCamera {
  R eye[3], f[3], r[3], u[3];
  R sx, sy;             // perspective: tan(fovy/2)*aspect, tan(fovy/2); ortho: half widths
  int ortho;
  int W, H;             // full image
  int x0, y0, w, h;     // window
};

// Pixel ray (matches the boundary header's camera definition).
template <typename R>
IVV_HD void make_ray(const DevCamera<R>& c, int px, int py, R o[3], R d[3]) {
  const R nx = (R(px) + R(0.5)) / R(c.W) * R(2) - R(1);
  const R ny = R(1) - (R(py) + R(0.5)) / R(c.H) * R(2);
  if (c.ortho) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      o[i] = c.eye[i] + nx * c.sx * c.r[i] + ny * c.sy * c.u[i];
      d[i] = c.f[i];
    }
  } else {
    R dd[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      o[i] = c.eye[i];
      dd[i] = c.f[i] + nx * c.sx * c.r[i] + ny * c.sy * c.u[i];
    }
    const R n = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
#pragma unroll
    for (int i = 0; i < 3; ++i) d[i] = dd[i] / n;
  }
}

// Screen position (pixel units, pixel centres at integers) of a point g.
template <typename R>
IVV_HD void project(const DevCamera<R>& c, const R g[3], R& sx, R& sy) {
  R w[3] = {g[0] - c.eye[0], g[1] - c.eye[1], g[2] - c.eye[2]};
  R x = w[0] * c.r[0] + w[1] * c.r[1] + w[2] * c.r[2];
  R y = w[0] * c.u[0] + w[1] * c.u[1] + w[2] * c.u[2];
  if (!c.ortho) {
    const R z = w[0] * c.f[0] + w[1] * c.f[1] + w[2] * c.f[2];
    x /= z;
    y /= z;
  }
  const R nx = x / c.sx, ny = y / c.sy;
  sx = (nx + R(1)) * R(0.5) * R(c.W) - R(0.5);
  sy = (R(1) - ny) * R(0.5) * R(c.H) - R(0.5);
}

// Conservative pixel box (x0, y0, x1, y1; empty if x0 > x1) of a face patch
// with control points org + cp[k]: the patch lies in the convex hull of its
// control points, whose projection bounds the patch's projection when every
// control point is in front of the eye.  Patches crossing the eye plane get
// the whole window; patches entirely behind it get an empty box.
template <int NN>
IVV_HD int4 face_screen_box(const DevCamera<float>& cam, const float4* cp, const float org[3], float diag) {
  float xmin = 1e30f, xmax = -1e30f, ymin = 1e30f, ymax = -1e30f;
  bool behind_all = true, straddle = false;
  const float znear = 1e-6f * diag;
  for (int q = 0; q < NN; ++q) {
    const float4 c = cp[q];
    const float g[3] = {org[0] + c.x, org[1] + c.y, org[2] + c.z};
    const float w[3] = {g[0] - cam.eye[0], g[1] - cam.eye[1], g[2] - cam.eye[2]};
    const float z = w[0] * cam.f[0] + w[1] * cam.f[1] + w[2] * cam.f[2];
    if (z > 0.f) behind_all = false;
    if (!cam.ortho && z <= znear) straddle = true;
    float sx, sy;
    project<float>(cam, g, sx, sy);
    xmin = fminf(xmin, sx); xmax = fmaxf(xmax, sx);
    ymin = fminf(ymin, sy); ymax = fmaxf(ymax, sy);
  }
  int4 b;
  if (behind_all) {
    b = make_int4(1, 1, 0, 0);
  } else if (straddle) {
    b = make_int4(cam.x0, cam.y0, cam.x0 + cam.w - 1, cam.y0 + cam.h - 1);
  } else {
    const float lim = 1e9f;
    xmin = fmaxf(xmin, -lim); ymin = fmaxf(ymin, -lim);
    xmax = fminf(xmax, lim); ymax = fminf(ymax, lim);
    const int bx0 = (int)floorf(xmin) - 1, by0 = (int)floorf(ymin) - 1;
    const int bx1 = (int)ceilf(xmax) + 1, by1 = (int)ceilf(ymax) + 1;
    b.x = bx0 > cam.x0 ? bx0 : cam.x0;
    b.y = by0 > cam.y0 ? by0 : cam.y0;
    b.z = bx1 < cam.x0 + cam.w - 1 ? bx1 : cam.x0 + cam.w - 1;
    b.w = by1 < cam.y0 + cam.h - 1 ? by1 : cam.y0 + cam.h - 1;
  }
  return b;
}

// ------------------------------------------------------------ 2-D patch
template <int P, typename R>
struct Patch2 {
  static constexpr int N = P + 1, NN = N * N;
  R x[NN], y[NN];        // index j*N + i: i along a, j along b
};

template <int P, typename R>
IVV_HD bool hull_has_origin(const Patch2<P, R>& q, R pad) {
  R x0 = q.x[0], x1 = q.x[0], y0 = q.y[0], y1 = q.y[0];
#pragma unroll
  for (int k = 1; k < Patch2<P, R>::NN; ++k) {
    x0 = minr(x0, q.x[k]); x1 = maxr(x1, q.x[k]);
    y0 = minr(y0, q.y[k]); y1 = maxr(y1, q.y[k]);
  }
  return !(x0 > pad || x1 < -pad || y0 > pad || y1 < -pad);
}

// The Jacobian det of the planar map is a sum of positive weights times
// cross(du_i, dv_j) over hodograph control vectors; if the interval of those
// cross products excludes 0 the map is locally one-to-one on the patch.
template <int P, typename R>
IVV_HD bool fixed_jacobian_sign(const Patch2<P, R>& q) {
  constexpr int N = P + 1;
  R ax0 = R(1e30), ax1 = R(-1e30), ay0 = R(1e30), ay1 = R(-1e30);
  R bx0 = R(1e30), bx1 = R(-1e30), by0 = R(1e30), by1 = R(-1e30);
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int i = 0; i < P; ++i) {
      const R ux = q.x[j * N + i + 1] - q.x[j * N + i], uy = q.y[j * N + i + 1] - q.y[j * N + i];
      ax0 = minr(ax0, ux); ax1 = maxr(ax1, ux); ay0 = minr(ay0, uy); ay1 = maxr(ay1, uy);
      const R vx = q.x[(i + 1) * N + j] - q.x[i * N + j], vy = q.y[(i + 1) * N + j] - q.y[i * N + j];
      bx0 = minr(bx0, vx); bx1 = maxr(bx1, vx); by0 = minr(by0, vy); by1 = maxr(by1, vy);
    }
  // interval of ux*vy - uy*vx
  const R p0 = ax0 * by0, p1 = ax0 * by1, p2 = ax1 * by0, p3 = ax1 * by1;
  const R q0 = ay0 * bx0, q1 = ay0 * bx1, q2 = ay1 * bx0, q3 = ay1 * bx1;
  const R plo = minr(minr(p0, p1), minr(p2, p3)), phi = maxr(maxr(p0, p1), maxr(p2, p3));
  const R qlo = minr(minr(q0, q1), minr(q2, q3)), qhi = maxr(maxr(q0, q1), maxr(q2, q3));
  return (plo - qhi) > R(0) || (phi - qlo) < R(0);
}

template <typename R> struct RootEps;
template <> struct RootEps<float> {
  static constexpr float step = 1e-6f, accept = 1e-4f, dup = 2e-5f;
};
template <> struct RootEps<double> {
  static constexpr double step = 1e-13, accept = 1e-9, dup = 1e-10;
};

// Damped Newton on the planar map of patch q (local parameters) from (a,b).
// lo / hi: the iterate is abandoned once it leaves [lo, hi]^2; max_it: the
// iteration budget.
template <int P, typename R>
IVV_HD bool newton2(const Patch2<P, R>& q, R& a, R& b, int& iters, R lo = R(-0.5), R hi = R(1.5), int max_it = 16) {
  constexpr int N = P + 1;
#pragma unroll 1
  for (int it = 0; it < max_it; ++it) {
    R ba[N], dba[N], bb[N], dbb[N];
    bern_hd<P, R>(a, ba, dba);
    bern_hd<P, R>(b, bb, dbb);
    R Fx = 0, Fy = 0, Ax = 0, Ay = 0, Bx = 0, By = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      R tx0 = 0, ty0 = 0, tx1 = 0, ty1 = 0;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        tx0 += ba[i] * q.x[j * N + i]; ty0 += ba[i] * q.y[j * N + i];
        tx1 += dba[i] * q.x[j * N + i]; ty1 += dba[i] * q.y[j * N + i];
      }
      Fx += bb[j] * tx0; Fy += bb[j] * ty0;
      Ax += bb[j] * tx1; Ay += bb[j] * ty1;
      Bx += dbb[j] * tx0; By += dbb[j] * ty0;
    }
    ++iters;
    const R det = Ax * By - Bx * Ay;
    if (det == R(0)) return false;
    const R inv = R(1) / det;
    R da = (-Fx * By + Fy * Bx) * inv;
    R db = (-Ax * Fy + Ay * Fx) * inv;
    const R mx = maxr(fabs(da), fabs(db));
    if (mx > R(0.5)) { da *= R(0.5) / mx; db *= R(0.5) / mx; }
    a += da;
    b += db;
    if (a < lo || a > hi || b < lo || b > hi) return false;
    if (fabs(da) + fabs(db) < RootEps<R>::step) return true;
  }
  return false;
}

constexpr int kMaxPatchRoots = 4;
constexpr int kSplitDepth = 8;
// Newton inside a certified box of the subdivision search: a root of the box
// lies within it, so an iterate that leaves the box by a quarter of its size,
// or a budget of 10 iterations without convergence, only means the box is
// split again (its halves are nearly bilinear).
template <typename R> IVV_HD constexpr R kBoxNewtonLo() { return R(-0.25); }
template <typename R> IVV_HD constexpr R kBoxNewtonHi() { return R(1.25); }
constexpr int kBoxNewtonIters = 10;

// Starting point for Newton on patch q: the zero of the bilinear map through
// its four corners (which lie on the patch), c00 + a e + b f + a b g = 0 with
// e = c10 - c00, f = c01 - c00, g = c11 - c10 - c01 + c00.  Eliminating a
// (cross product with e + b g) leaves k2 b^2 + k1 b + k0 = 0; a follows from
// the better conditioned component.  Falls back to the centre when the
// quadratic has no usable root; the result is clamped to [0,1]^2.
template <int P, typename R>
IVV_HD void bilinear_start(const Patch2<P, R>& q, R& a, R& b) {
  constexpr int N = P + 1;
  const R c00x = q.x[0], c00y = q.y[0], c10x = q.x[P], c10y = q.y[P];
  const R c01x = q.x[P * N], c01y = q.y[P * N], c11x = q.x[P * N + P], c11y = q.y[P * N + P];
  const R ex = c10x - c00x, ey = c10y - c00y, fx = c01x - c00x, fy = c01y - c00y;
  const R gx = c11x - c10x - c01x + c00x, gy = c11y - c10y - c01y + c00y;
  const R k2 = fx * gy - fy * gx;
  const R k1 = (c00x * gy - c00y * gx) + (fx * ey - fy * ex);
  const R k0 = c00x * ey - c00y * ex;
  a = b = R(0.5);
  R bb;
  const R scale = fabs(k1) + fabs(k0) + R(1e-30);
  if (fabs(k2) <= R(1e-6) * scale) {
    if (k1 == R(0)) return;
    bb = -k0 / k1;
  } else {
    const R disc = k1 * k1 - R(4) * k2 * k0;
    if (!(disc >= R(0))) return;
    const R sq = sqrt(disc);
    const R q1 = R(-0.5) * (k1 + (k1 >= R(0) ? sq : -sq));       // stable pair of roots
    const R r1 = q1 / k2, r2 = q1 != R(0) ? k0 / q1 : r1;
    const R d1 = fabs(r1 - clamp01r(r1)), d2 = fabs(r2 - clamp01r(r2));
    bb = d1 <= d2 ? r1 : r2;
  }
  const R dx = ex + bb * gx, dy = ey + bb * gy;
  const R aa = fabs(dx) >= fabs(dy) ? -(c00x + bb * fx) / dx : -(c00y + bb * fy) / dy;
  if (!(aa == aa) || !(bb == bb) || fabs(aa) > R(1e30)) return;
  a = clamp01r(aa);
  b = clamp01r(bb);
}

// Accept a root (a,b) of a sub-patch covering [a0,a1] x [b0,b1] of the face
// patch: inside the sub-patch (tolerance scaled to its size) and inside the
// patch, and not a duplicate of a root already found.
// Returns false if (a,b) lies outside the sub-patch (the caller then looks
// for the sub-patch's own root in smaller pieces).
// With in_box = false (the uncertified smallest pieces of the subdivision
// search, which may hold two roots on either side of a fold of the
// projected patch) a root anywhere inside the patch is kept: Newton from the
// piece's starts may reach the second root of the fold just beyond the
// piece, and the neighbouring piece's starts may all reach the first one.
// Copies of one root found from several pieces are merged here and, as
// fragments of equal facing, by the depth sort.
template <typename R>
IVV_HD bool accept_root(R a, R b, R a0, R a1, R b0, R b1, R ra[kMaxPatchRoots], R rb[kMaxPatchRoots], int& nr,
                        bool in_box = true) {
  const R wa = a1 - a0, wb = b1 - b0;
  const R ea = RootEps<R>::accept / wa, eb = RootEps<R>::accept / wb;
  if (in_box && (a < -ea || a > R(1) + ea || b < -eb || b > R(1) + eb)) return false;
  const R ga = a0 + a * wa, gb = b0 + b * wb;
  const R e = RootEps<R>::accept;
  if (ga < -e || ga > R(1) + e || gb < -e || gb > R(1) + e) return true;
  for (int k = 0; k < nr; ++k)
    if (fabs(ra[k] - ga) + fabs(rb[k] - gb) < RootEps<R>::dup) return true;
  if (nr < kMaxPatchRoots) {
    ra[nr] = ga;
    rb[nr] = gb;
    ++nr;
  }
  return true;
}

// Sub-patch of q covering [a0,a1] x [b0,b1] (de Casteljau: split at the
// upper end, then split the left part at the relative lower end).
template <int P, typename R>
IVV_HD void sub_patch(const Patch2<P, R>& q, R a0, R a1, R b0, R b1, Patch2<P, R>& out) {
  constexpr int N = P + 1;
  out = q;
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
    const R t0 = dir == 0 ? a0 : b0, t1 = dir == 0 ? a1 : b1;
    const R s = t1 > R(0) ? t0 / t1 : R(0);
#pragma unroll
    for (int line = 0; line < N; ++line) {
      R wx[N], wy[N], lx[N], ly[N];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const int idx = dir == 0 ? line * N + k : k * N + line;
        wx[k] = out.x[idx];
        wy[k] = out.y[idx];
      }
      // left part of the split at t1
      lx[0] = wx[0]; ly[0] = wy[0];
#pragma unroll
      for (int lev = 1; lev <= P; ++lev) {
#pragma unroll
        for (int k = 0; k + lev <= P; ++k) {
          wx[k] = wx[k] + t1 * (wx[k + 1] - wx[k]);
          wy[k] = wy[k] + t1 * (wy[k + 1] - wy[k]);
        }
        lx[lev] = wx[0]; ly[lev] = wy[0];
      }
      // right part of the split of that at s
      R rx[N], ry[N];
      rx[P] = lx[P]; ry[P] = ly[P];
#pragma unroll
      for (int lev = 1; lev <= P; ++lev) {
#pragma unroll
        for (int k = 0; k + lev <= P; ++k) {
          lx[k] = lx[k] + s * (lx[k + 1] - lx[k]);
          ly[k] = ly[k] + s * (ly[k + 1] - ly[k]);
        }
        rx[P - lev] = lx[P - lev]; ry[P - lev] = ly[P - lev];
      }
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const int idx = dir == 0 ? line * N + k : k * N + line;
        out.x[idx] = rx[k];
        out.y[idx] = ry[k];
      }
    }
  }
}

// Subdivision search for the roots of q0 (rare path: patches whose single
// root is not certified).  The stack keeps parameter boxes only; each piece
// is re-extracted from q0.
template <int P, typename R>
__host__ __device__ __noinline__ int patch_roots_split(const Patch2<P, R>* q0p, R pad, R* ra, R* rb, int& iters) {
  struct Box {
    R a0, a1, b0, b1;
    int depth;
  };
  const Patch2<P, R>& q0 = *q0p;
  Box stack[kSplitDepth + 1];
  stack[0].a0 = R(0); stack[0].a1 = R(1); stack[0].b0 = R(0); stack[0].b1 = R(1);
  stack[0].depth = 0;
  int sp = 1, nr = 0;
  while (sp > 0) {
    const Box nd = stack[--sp];
    Patch2<P, R> q;
    sub_patch<P, R>(q0, nd.a0, nd.a1, nd.b0, nd.b1, q);
    if (!hull_has_origin<P, R>(q, pad)) continue;
    bool split = true;
    if (fixed_jacobian_sign<P, R>(q)) {
      // Newton from the centre; if it fails or converges to a root outside
      // this piece, look for the piece's root in smaller pieces
      R a = R(0.5), b = R(0.5);
      split = !(newton2<P, R>(q, a, b, iters, kBoxNewtonLo<R>(), kBoxNewtonHi<R>(), kBoxNewtonIters) &&
                accept_root<R>(a, b, nd.a0, nd.a1, nd.b0, nd.b1, ra, rb, nr));
    } else if (nd.depth >= kSplitDepth) {
      // smallest piece, not certified: Newton from the centre and the four
      // quarter points, keeping every distinct root inside the piece
      for (int s0 = 0; s0 < 5; ++s0) {
        R a = s0 == 0 ? R(0.5) : ((s0 & 1) ? R(0.25) : R(0.75));
        R b = s0 == 0 ? R(0.5) : ((s0 & 2) ? R(0.25) : R(0.75));
        if (newton2<P, R>(q, a, b, iters)) accept_root<R>(a, b, nd.a0, nd.a1, nd.b0, nd.b1, ra, rb, nr, false);
      }
      split = false;
    }
    if (!split || nd.depth >= kSplitDepth || sp + 2 > kSplitDepth + 1) continue;
    // split along the parameter direction with the longer control polygon
    constexpr int N = P + 1;
    R la = 0, lb = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      la += fabs(q.x[k * N + P] - q.x[k * N]) + fabs(q.y[k * N + P] - q.y[k * N]);
      lb += fabs(q.x[P * N + k] - q.x[k]) + fabs(q.y[P * N + k] - q.y[k]);
    }
    Box& hi = stack[sp];
    Box& lo = stack[sp + 1];               // lower half is processed next
    lo = nd;
    hi = nd;
    lo.depth = hi.depth = nd.depth + 1;
    if (la >= lb) {
      const R m = R(0.5) * (nd.a0 + nd.a1);
      lo.a1 = m;
      hi.a0 = m;
    } else {
      const R m = R(0.5) * (nd.b0 + nd.b1);
      lo.b1 = m;
      hi.b0 = m;
    }
    sp += 2;
  }
  return nr;
}

// The common case of the root search of patch_roots: a one-to-one patch
// (fixed Jacobian sign) holds at most one root, found by Newton from the
// bilinear start; a solution outside the patch gets one restart from the
// nearest patch point.  Returns false when the patch needs the subdivision
// search (sign not fixed, or Newton broke down); otherwise nr roots are in
// ra, rb.
template <int P, typename R>
IVV_HD bool patch_roots_fast(const Patch2<P, R>& q0, R ra[kMaxPatchRoots], R rb[kMaxPatchRoots], int& nr,
                             int& iters) {
  nr = 0;
  if (!fixed_jacobian_sign<P, R>(q0)) return false;
  R a, b;
  bilinear_start<P, R>(q0, a, b);
#pragma unroll 1
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (!newton2<P, R>(q0, a, b, iters)) return false;
    if (accept_root<R>(a, b, R(0), R(1), R(0), R(1), ra, rb, nr)) return true;
    if (attempt == 1) return true;       // converged twice outside: no root
    a = clamp01r(a);
    b = clamp01r(b);
  }
  return true;
}

// All roots (a,b) in [0,1]^2 (within a tolerance) of the planar patch q0,
// whose hull is known to contain the origin.  Returns the count
// (<= kMaxPatchRoots); `iters` accumulates Newton steps.
template <int P, typename R>
IVV_HD int patch_roots(const Patch2<P, R>& q0, R pad, R ra[kMaxPatchRoots], R rb[kMaxPatchRoots], int& iters) {
  int nr;
  if (patch_roots_fast<P, R>(q0, ra, rb, nr, iters)) return nr;
  return patch_roots_split<P, R>(&q0, pad, ra, rb, iters);
}

// ------------------------------------------------------------ 3-D patch
// S(a,b) relative to the patch origin, with partials; cp are (x,y,z,_) rows.
template <int P, typename R, typename V4>
IVV_HD void patch_eval3_rel(const V4* cp, R a, R b, R S[3], R Sa[3], R Sb[3]) {
  constexpr int N = P + 1;
  R ba[N], dba[N], bb[N], dbb[N];
  bern_hd<P, R>(a, ba, dba);
  bern_hd<P, R>(b, bb, dbb);
#pragma unroll
  for (int r = 0; r < 3; ++r) S[r] = Sa[r] = Sb[r] = R(0);
#pragma unroll
  for (int j = 0; j < N; ++j) {
    R t0[3] = {0, 0, 0}, t1[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const V4 c = cp[j * N + i];
      t0[0] += ba[i] * R(c.x); t0[1] += ba[i] * R(c.y); t0[2] += ba[i] * R(c.z);
      t1[0] += dba[i] * R(c.x); t1[1] += dba[i] * R(c.y); t1[2] += dba[i] * R(c.z);
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      S[r] += bb[j] * t0[r];
      Sa[r] += bb[j] * t1[r];
      Sb[r] += dbb[j] * t0[r];
    }
  }
}

// Planar control points of a face patch in the frame (e1, e2) of a ray from
// o: x_k = ((org - o) + c_k) . e1, with c_k relative to the patch origin.
template <int P, typename R, typename V4>
IVV_HD void project_patch(const V4* cp, const R org[3], const R o[3], const R e1[3], const R e2[3],
                          Patch2<P, R>& q) {
  const R D[3] = {org[0] - o[0], org[1] - o[1], org[2] - o[2]};
  const R x0 = D[0] * e1[0] + D[1] * e1[1] + D[2] * e1[2];
  const R y0 = D[0] * e2[0] + D[1] * e2[1] + D[2] * e2[2];
#pragma unroll
  for (int k = 0; k < (P + 1) * (P + 1); ++k) {
    const V4 c = cp[k];
    q.x[k] = x0 + (R(c.x) * e1[0] + R(c.y) * e1[1] + R(c.z) * e1[2]);
    q.y[k] = y0 + (R(c.x) * e2[0] + R(c.y) * e2[1] + R(c.z) * e2[2]);
  }
}

// Ray vs axis-aligned box [lo, hi] (padded); true if it meets the box at
// t >= 0.  inv_d = 1 / d per component.
template <typename R>
IVV_HD bool ray_box(const R o[3], const R inv_d[3], const float lo[3], const float hi[3], R pad) {
  R t0 = R(-1e30), t1 = R(1e30);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const R inv = inv_d[r];
    R ta = (R(lo[r]) - pad - o[r]) * inv, tb = (R(hi[r]) + pad - o[r]) * inv;
    if (ta > tb) { const R x = ta; ta = tb; tb = x; }
    t0 = ta > t0 ? ta : t0;
    t1 = tb < t1 ? tb : t1;
  }
  return t1 >= t0 && t1 >= R(0);
}

// Ray vs the oriented box of a face patch (padded); true if it meets the box
// at t >= 0.
template <typename R>
IVV_HD bool ray_obb(const R o[3], const R d[3], const FaceMeta& m, R pad) {
  const R w[3] = {o[0] - R(m.obb_c[0]), o[1] - R(m.obb_c[1]), o[2] - R(m.obb_c[2])};
  R t0 = R(-1e30), t1 = R(1e30);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const R oa = R(m.obb_ax[a][0]) * w[0] + R(m.obb_ax[a][1]) * w[1] + R(m.obb_ax[a][2]) * w[2];
    const R da = R(m.obb_ax[a][0]) * d[0] + R(m.obb_ax[a][1]) * d[1] + R(m.obb_ax[a][2]) * d[2];
    const R hw = R(m.obb_h[a]) + pad;
    if (fabs(da) < R(1e-30)) {
      if (oa < -hw || oa > hw) return false;
      continue;
    }
    const R inv = R(1) / da;
    R ta = (-hw - oa) * inv, tb = (hw - oa) * inv;
    if (ta > tb) { const R x = ta; ta = tb; tb = x; }
    t0 = ta > t0 ? ta : t0;
    t1 = tb < t1 ? tb : t1;
  }
  return t1 >= t0 && t1 >= R(0);
}

// Fragment of a root (a,b) of face `m`: depth t, facing, block parameter point.
// (a,b) may lie outside the patch by the root acceptance tolerance (a root on
// the seam of two patches, found by both): the patch polynomial is evaluated
// there as it is, and only the block parameter point is clamped to [0,1]^3,
// so both copies of a seam root carry the same accurate point.
template <int P, typename R, typename V4>
IVV_HD void make_fragment(const V4* cp, const R org[3], const FaceMeta& m, const R pa0, const R pa1, const R pb0,
                          const R pb1, const R o[3], const R d[3], R a, R b, R& t, bool& front, R pp[3], R& cosang) {
  R S[3], Sa[3], Sb[3];
  patch_eval3_rel<P, R, V4>(cp, a, b, S, Sa, Sb);
  t = ((org[0] - o[0]) * d[0] + (org[1] - o[1]) * d[1] + (org[2] - o[2]) * d[2]) +
      (S[0] * d[0] + S[1] * d[1] + S[2] * d[2]);
  const R n[3] = {Sa[1] * Sb[2] - Sa[2] * Sb[1], Sa[2] * Sb[0] - Sa[0] * Sb[2], Sa[0] * Sb[1] - Sa[1] * Sb[0]};
  const R dn = n[0] * d[0] + n[1] * d[1] + n[2] * d[2];
  const R nl = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  cosang = nl > R(0) ? fabs(dn) / nl : R(0);
  front = (m.face & 1) ? (dn < R(0)) : (dn > R(0));
  const int nd = m.face >> 1, ad = (nd + 1) % 3, bd = (nd + 2) % 3;
  pp[nd] = (m.face & 1) ? R(1) : R(0);
  pp[ad] = clamp01r(pa0 + a * (pa1 - pa0));
  pp[bd] = clamp01r(pb0 + b * (pb1 - pb0));
}

// Mixed precision: hits where |cos| of the ray and the face normal is below
// this get the FP64 polish.  An FP32 hit is accurate to about 4e-6 / |cos|
// in the block parameters (positions of magnitude ~10 carry ~1e-6 of
// rounding), so 0.35 keeps every hit within 1e-5.
constexpr float kPolishCos = 0.35f;

// Patch value S(a,b) relative to the patch origin (no partials).
template <int P, typename R, typename V4>
IVV_HD void patch_value3_rel(const V4* cp, R a, R b, R S[3]) {
  constexpr int N = P + 1;
  R ba[N], dba[N], bb[N], dbb[N];
  bern_hd<P, R>(a, ba, dba);
  bern_hd<P, R>(b, bb, dbb);
#pragma unroll
  for (int r = 0; r < 3; ++r) S[r] = R(0);
#pragma unroll
  for (int j = 0; j < N; ++j) {
    R t0[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const V4 c = cp[j * N + i];
      t0[0] += ba[i] * R(c.x); t0[1] += ba[i] * R(c.y); t0[2] += ba[i] * R(c.z);
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) S[r] += bb[j] * t0[r];
  }
}

// Mixed-precision polish of a hit near a silhouette: Newton on
// S(a,b) - o - t d = 0 whose residual is evaluated in FP64 (the FP64 face
// patch cp64, control points relative to org64) while the Jacobian
// [S_a S_b -d] and the 3x3 solve stay in FP32 (the FP32 patch cp32): the
// classic refinement by an accurate residual.  Each step shrinks the error by
// about |cos|^-1 times the FP32 rounding, so a few steps reach the FP64 root;
// the FP64 work is the patch value alone.
template <int P, typename V4D>
IVV_HD void refine_hit_mixed(const V4D* cp64, const float4* cp32, const double org[3], const double o[3],
                             const double d[3], double& a, double& b, double& t) {
  for (int it = 0; it < 4; ++it) {
    double S[3];
    patch_value3_rel<P, double, V4D>(cp64, a, b, S);
    float F[3];
    for (int r = 0; r < 3; ++r) F[r] = (float)(-((org[r] - o[r]) + S[r] - t * d[r]));
    float S32[3], Sa[3], Sb[3];
    patch_eval3_rel<P, float, float4>(cp32, (float)a, (float)b, S32, Sa, Sb);
    const float df[3] = {(float)d[0], (float)d[1], (float)d[2]};
    const float A[3][3] = {{Sa[0], Sb[0], -df[0]}, {Sa[1], Sb[1], -df[1]}, {Sa[2], Sb[2], -df[2]}};
    const float c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    const float c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
    const float c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    const float det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
    if (det == 0.f) break;
    const float c10 = A[0][2] * A[2][1] - A[0][1] * A[2][2];
    const float c11 = A[0][0] * A[2][2] - A[0][2] * A[2][0];
    const float c12 = A[0][1] * A[2][0] - A[0][0] * A[2][1];
    const float c20 = A[0][1] * A[1][2] - A[0][2] * A[1][1];
    const float c21 = A[0][2] * A[1][0] - A[0][0] * A[1][2];
    const float c22 = A[0][0] * A[1][1] - A[0][1] * A[1][0];
    const float inv = 1.f / det;
    const float x0 = (c00 * F[0] + c10 * F[1] + c20 * F[2]) * inv;
    const float x1 = (c01 * F[0] + c11 * F[1] + c21 * F[2]) * inv;
    const float x2 = (c02 * F[0] + c12 * F[1] + c22 * F[2]) * inv;
    if (!(fabsf(x0) < 0.5f && fabsf(x1) < 0.5f)) break;
    a += x0; b += x1; t += x2;
    // the fragment keeps FP32 parameters: corrections below 1e-9 of the
    // patch are beyond what it stores
    if (fabsf(x0) + fabsf(x1) < 1e-9f) break;
  }
}

// ------------------------------------------------------------ stage 2
// Sort fragments by (t, block, facing), merge duplicates of one block with
// equal facing closer than tau_dup, and pair by Alg. 2.  meta = block << 4 |
// face << 1 | front.  Writes (front index, back index) per pair in order.
// Strict order of fragments: depth, block, facing, face, then parameters
// (so the result never depends on the order fragments were appended).
template <typename R>
IVV_HD bool frag_less(R ta, unsigned ma, const R* pa, R tb, unsigned mb, const R* pb) {
  if (ta != tb) return ta < tb;
  if ((ma >> 4) != (mb >> 4)) return (ma >> 4) < (mb >> 4);
  if ((ma & 1u) != (mb & 1u)) return (ma & 1u) < (mb & 1u);
  if (ma != mb) return ma < mb;
  if (pa[0] != pb[0]) return pa[0] < pb[0];
  if (pa[1] != pb[1]) return pa[1] < pb[1];
  return pa[2] < pb[2];
}

template <typename R>
IVV_HD int pair_fragments(int n, const R* t, const unsigned* m, const R (*pp)[3], R tau_dup, int max_pairs,
                          int* in_idx, int* out_idx, unsigned& unmatched, unsigned& overflow) {
  unsigned char ord[kMaxFrags];
  for (int i = 0; i < n; ++i) {
    int j = i;
    while (j > 0) {
      const int a = ord[j - 1];
      const bool gt = frag_less<R>(t[i], m[i], pp[i], t[a], m[a], pp[a]);
      if (!gt) break;
      ord[j] = ord[j - 1];
      --j;
    }
    ord[j] = (unsigned char)i;
  }
  // duplicates: of two copies of one hit (a seam of two patches or an edge
  // of two faces, both within the root acceptance tolerance) keep the one
  // with fewer parameter coordinates on the block boundary -- the copy from
  // the face that holds the hit, not the one clamped onto the edge
  auto on_bound = [](const R* p) {
    return (int)(p[0] == R(0) || p[0] == R(1)) + (int)(p[1] == R(0) || p[1] == R(1)) +
           (int)(p[2] == R(0) || p[2] == R(1));
  };
  unsigned used = 0;
  for (int i = 0; i < n; ++i) {
    const int a = ord[i];
    for (int j = 0; j < i; ++j) {
      const int b = ord[j];
      if (!((used >> j) & 1u) && (m[a] >> 4) == (m[b] >> 4) && (m[a] & 1u) == (m[b] & 1u) && t[a] - t[b] <= tau_dup) {
        if (on_bound(pp[a]) < on_bound(pp[b]))
          used |= 1u << j;
        else
          used |= 1u << i;
        break;
      }
    }
  }
  // a lone hit on a block edge (two or three parameter coordinates on the
  // block boundary) next to a hit of the same block and the same facing:
  // the ray touches the edge within the root tolerance on one face while
  // the other face's copy of the touch falls outside it, so the touch has no
  // partner of the opposite facing.  Entry and exit alternate along a ray
  // through a block (its boundary is closed), so of two consecutive hits of
  // one block with the same facing the edge hit is the spurious one, and a
  // block's first hit cannot be an exit: such edge hits are dropped before
  // Alg. 2.
  for (int i = 0; i < n; ++i) {
    if ((used >> i) & 1u) continue;
    const unsigned blk = m[ord[i]] >> 4;
    int prev = -1;
    for (int j = i - 1; j >= 0; --j)
      if (!((used >> j) & 1u) && (m[ord[j]] >> 4) == blk) { prev = j; break; }
    const bool front = m[ord[i]] & 1u;
    if (prev < 0) {
      if (!front && on_bound(pp[ord[i]]) >= 2) used |= 1u << i;
      continue;
    }
    if (((m[ord[prev]] & 1u) != 0) != front) continue;
    const bool edge_i = on_bound(pp[ord[i]]) >= 2, edge_p = on_bound(pp[ord[prev]]) >= 2;
    if (edge_p && !edge_i)
      used |= 1u << prev;
    else if (edge_i && !edge_p)
      used |= 1u << i;
  }
  int np = 0;
  for (;;) {
    int back = -1;
    for (int i = 0; i < n; ++i)
      if (!((used >> i) & 1u) && !(m[ord[i]] & 1u)) { back = i; break; }
    if (back < 0) break;
    const unsigned blk = m[ord[back]] >> 4;
    int front = -1;
    for (int i = 0; i < n; ++i)
      if (!((used >> i) & 1u) && (m[ord[i]] & 1u) && (m[ord[i]] >> 4) == blk) { front = i; break; }
    used |= 1u << back;
    if (front < 0) { ++unmatched; continue; }
    used |= 1u << front;
    if (np < max_pairs) {
      in_idx[np] = ord[front];
      out_idx[np] = ord[back];
      ++np;
    } else {
      ++overflow;
    }
  }
  for (int i = 0; i < n; ++i)
    if (!((used >> i) & 1u)) ++unmatched;
  return np;
}

}  // namespace ivv
