// Stage 1 (§4.1): intersections of every pixel ray with the boundary surfaces
// of every block.  The paper rasterises a view-dependent pixel-accurate
// tessellation; here every ray is intersected with the Bezier face patches
// directly:
//   K0 face_project  -- conservative screen box of each face patch from its
//                       control points (convex hull property).
//   K2 intersect     -- one CTA per 16x16 screen tile: cull the face boxes
//                       against the tile, stage the surviving patches in
//                       shared memory, and per pixel solve S(a,b) = o + t d by
//                       Newton on the two coordinates perpendicular to the ray
//                       (hull test first), from four starts; hits go into the
//                       pixel's fragment slots (the A-buffer of §4.2).
#include <cuda_runtime.h>

#include "ivv_device.cuh"

namespace ivv {

namespace {

__global__ void k0_face_project(DevVolume V, DevCamera<float> cam, int4* __restrict__ boxes) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= V.n_faces) return;
  const int NN = (V.P + 1) * (V.P + 1);
  const float4* cp = V.face32 + (size_t)f * NN;
  float xmin = 1e30f, xmax = -1e30f, ymin = 1e30f, ymax = -1e30f;
  bool behind_all = true, straddle = false;
  const float znear = 1e-6f * V.diag;
  for (int q = 0; q < NN; ++q) {
    const float4 c = cp[q];
    const float w[3] = {c.x - cam.eye[0], c.y - cam.eye[1], c.z - cam.eye[2]};
    const float z = w[0] * cam.f[0] + w[1] * cam.f[1] + w[2] * cam.f[2];
    if (z > 0.f) behind_all = false;
    if (!cam.ortho && z <= znear) straddle = true;
    const float g[3] = {c.x, c.y, c.z};
    float sx, sy;
    project<float>(cam, g, sx, sy);
    xmin = fminf(xmin, sx); xmax = fmaxf(xmax, sx);
    ymin = fminf(ymin, sy); ymax = fmaxf(ymax, sy);
  }
  int4 b;
  if (behind_all) {
    b = make_int4(1, 1, 0, 0);                                   // empty
  } else if (straddle) {
    b = make_int4(cam.x0, cam.y0, cam.x0 + cam.w - 1, cam.y0 + cam.h - 1);
  } else {
    const float lim = 1e9f;
    xmin = fmaxf(xmin, -lim); ymin = fmaxf(ymin, -lim);
    xmax = fminf(xmax, lim); ymax = fminf(ymax, lim);
    b.x = max((int)floorf(xmin) - 1, cam.x0);
    b.y = max((int)floorf(ymin) - 1, cam.y0);
    b.z = min((int)ceilf(xmax) + 1, cam.x0 + cam.w - 1);
    b.w = min((int)ceilf(ymax) + 1, cam.y0 + cam.h - 1);
  }
  boxes[f] = b;
}

template <typename R> __device__ __forceinline__ R clamp01(R x) { return x < R(0) ? R(0) : (x > R(1) ? R(1) : x); }

template <typename R> struct Eps;
template <> struct Eps<float> {
  static constexpr float step = 1e-6f, accept = 1e-4f;
};
template <> struct Eps<double> {
  static constexpr double step = 1e-13, accept = 1e-9;
};

// 3-D patch point and partials at (a, b) from control points in shared memory.
template <int P, typename R, typename V4>
__device__ __forceinline__ void patch_eval3(const V4* cp, R a, R b, R S[3], R Sa[3], R Sb[3]) {
  constexpr int N = P + 1;
  R ba[N], dba[N], bb[N], dbb[N];
  bernstein<P, R>(a, ba, dba);
  bernstein<P, R>(b, bb, dbb);
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

// FP64 polish of a hit near a silhouette: Newton on S(a,b) - o - t d = 0.
template <int P>
__device__ __noinline__ void refine_fp64(const DevVolume& V, int face, const DevCamera<double>& cam64, int px, int py,
                            double& a, double& b, double& t) {
  constexpr int N = P + 1;
  const Dbl4* cp = V.face64 + (size_t)face * N * N;
  double o[3], d[3];
  make_ray<double>(cam64, px, py, o, d);
  for (int it = 0; it < 4; ++it) {
    double S[3], Sa[3], Sb[3];
    patch_eval3<P, double, Dbl4>(cp, a, b, S, Sa, Sb);
    double J[3][3], F[3], x[3];
    for (int r = 0; r < 3; ++r) {
      J[r][0] = Sa[r]; J[r][1] = Sb[r]; J[r][2] = -d[r];
      F[r] = -(S[r] - o[r] - t * d[r]);
    }
    solve3<double>(J, F, x);
    if (!(fabs(x[0]) < 0.5 && fabs(x[1]) < 0.5)) break;
    a += x[0]; b += x[1]; t += x[2];
  }
}

template <int P, typename R, bool MIXED, bool STATS>
__global__ void __launch_bounds__(256) k2_intersect(DevVolume V, DevCamera<R> cam, DevCamera<double> cam64,
                                                    const int4* __restrict__ boxes,
                                                    typename Vec4T<R>::type* __restrict__ frag_tp,
                                                    unsigned* __restrict__ frag_meta, int* __restrict__ frag_count,
                                                    DevStats* __restrict__ st) {
  typedef typename Vec4T<R>::type V4;
  constexpr int N = P + 1, NN = N * N;
  constexpr int CH = 32;
  __shared__ int s_cand[256];
  __shared__ int s_wcnt[8];
  __shared__ V4 s_cp[CH * NN];
  __shared__ FaceMeta s_meta[CH];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tiles_x = (cam.w + kTileW - 1) / kTileW;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int xw = tx * kTileW + (tid % kTileW), yw = ty * kTileH + (tid / kTileW);
  const bool valid = xw < cam.w && yw < cam.h;
  const int px = cam.x0 + xw, py = cam.y0 + yw;
  const int npix = cam.w * cam.h;
  const int pix = yw * cam.w + xw;
  const int rx0 = cam.x0 + tx * kTileW, ry0 = cam.y0 + ty * kTileH;
  const int rx1 = min(rx0 + kTileW - 1, cam.x0 + cam.w - 1), ry1 = min(ry0 + kTileH - 1, cam.y0 + cam.h - 1);

  R o[3], d[3], e1[3], e2[3];
  make_ray<R>(cam, px, py, o, d);
  {
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
  const R hull_pad = R(1e-6) * R(V.diag);
  int nfrag = 0;
  unsigned long long c_tests = 0, c_newton = 0, c_fp64 = 0;

  for (int base = 0; base < V.n_faces; base += 256) {
    const int f = base + tid;
    bool keep = false;
    if (f < V.n_faces) {
      const int4 b = __ldg(boxes + f);
      keep = b.x <= rx1 && b.z >= rx0 && b.y <= ry1 && b.w >= ry0;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) s_wcnt[warp] = __popc(bal);
    __syncthreads();
    int off = 0, total = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const int c = s_wcnt[w];
      off += (w < warp) ? c : 0;
      total += c;
    }
    if (keep) s_cand[off + __popc(bal & ((1u << lane) - 1u))] = f;
    __syncthreads();
    for (int c0 = 0; c0 < total; c0 += CH) {
      const int nst = min(CH, total - c0);
      for (int q = tid; q < nst * NN; q += 256) {
        const int fi = s_cand[c0 + q / NN];
        if constexpr (sizeof(R) == 4) {
          s_cp[q] = __ldg(V.face32 + (size_t)fi * NN + (q % NN));
        } else {
          s_cp[q] = V.face64[(size_t)fi * NN + (q % NN)];
        }
      }
      for (int q = tid; q < nst; q += 256) s_meta[q] = V.faces[s_cand[c0 + q]];
      __syncthreads();
      if (valid) {
        for (int q = 0; q < nst; ++q) {
          const FaceMeta& m = s_meta[q];
          // ray vs control-point box
          R t0 = R(-1e30), t1 = R(1e30);
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            const R inv = R(1) / d[r];
            R ta = (R(m.lo[r]) - hull_pad - o[r]) * inv, tb = (R(m.hi[r]) + hull_pad - o[r]) * inv;
            if (ta > tb) { const R x = ta; ta = tb; tb = x; }
            t0 = ta > t0 ? ta : t0;
            t1 = tb < t1 ? tb : t1;
          }
          if (!(t1 >= t0 && t1 >= R(0))) continue;
          // control points in the ray frame; hull must contain the ray
          const V4* cp = s_cp + q * NN;
          R X[NN], Y[NN];
          R xmin = R(1e30), xmax = R(-1e30), ymin = R(1e30), ymax = R(-1e30);
#pragma unroll
          for (int k = 0; k < NN; ++k) {
            const V4 c = cp[k];
            const R w0 = R(c.x) - o[0], w1 = R(c.y) - o[1], w2 = R(c.z) - o[2];
            X[k] = w0 * e1[0] + w1 * e1[1] + w2 * e1[2];
            Y[k] = w0 * e2[0] + w1 * e2[1] + w2 * e2[2];
            xmin = X[k] < xmin ? X[k] : xmin; xmax = X[k] > xmax ? X[k] : xmax;
            ymin = Y[k] < ymin ? Y[k] : ymin; ymax = Y[k] > ymax ? Y[k] : ymax;
          }
          if (xmin > hull_pad || xmax < -hull_pad || ymin > hull_pad || ymax < -hull_pad) continue;
          if (STATS) ++c_tests;
          R ra[4], rb[4];
          int nr = 0;
#pragma unroll 1
          for (int s0 = 0; s0 < 4; ++s0) {
            R a = (s0 & 1) ? R(0.75) : R(0.25), b = (s0 & 2) ? R(0.75) : R(0.25);
            bool conv = false;
#pragma unroll 1
            for (int it = 0; it < 16; ++it) {
              R ba[N], dba[N], bb[N], dbb[N];
              bernstein<P, R>(a, ba, dba);
              bernstein<P, R>(b, bb, dbb);
              R Fx = 0, Fy = 0, Ax = 0, Ay = 0, Bx = 0, By = 0;
#pragma unroll
              for (int j = 0; j < N; ++j) {
                R tx0 = 0, ty0 = 0, tx1 = 0, ty1 = 0;
#pragma unroll
                for (int i = 0; i < N; ++i) {
                  tx0 += ba[i] * X[j * N + i]; ty0 += ba[i] * Y[j * N + i];
                  tx1 += dba[i] * X[j * N + i]; ty1 += dba[i] * Y[j * N + i];
                }
                Fx += bb[j] * tx0; Fy += bb[j] * ty0;
                Ax += bb[j] * tx1; Ay += bb[j] * ty1;
                Bx += dbb[j] * tx0; By += dbb[j] * ty0;
              }
              const R det = Ax * By - Bx * Ay;
              if (STATS) ++c_newton;
              if (det == R(0)) break;
              R da = (-Fx * By + Fy * Bx) / det;
              R db = (-Ax * Fy + Ay * Fx) / det;
              const R mx = fabs(da) > fabs(db) ? fabs(da) : fabs(db);
              if (mx > R(0.5)) { da *= R(0.5) / mx; db *= R(0.5) / mx; }
              a += da;
              b += db;
              if (a < R(-1) || a > R(2) || b < R(-1) || b > R(2)) break;
              if (fabs(da) + fabs(db) < Eps<R>::step) { conv = true; break; }
            }
            if (!conv) continue;
            const R ea = Eps<R>::accept;
            if (a < -ea || a > R(1) + ea || b < -ea || b > R(1) + ea) continue;
            bool dup = false;
            for (int k = 0; k < nr; ++k)
              if (fabs(ra[k] - a) + fabs(rb[k] - b) < R(1e-3)) dup = true;
            if (dup) continue;
            ra[nr] = a; rb[nr] = b; ++nr;
            a = clamp01(a);
            b = clamp01(b);
            R S[3], Sa[3], Sb[3];
            patch_eval3<P, R, V4>(cp, a, b, S, Sa, Sb);
            R t = (S[0] - o[0]) * d[0] + (S[1] - o[1]) * d[1] + (S[2] - o[2]) * d[2];
            R nrm[3] = {Sa[1] * Sb[2] - Sa[2] * Sb[1], Sa[2] * Sb[0] - Sa[0] * Sb[2], Sa[0] * Sb[1] - Sa[1] * Sb[0]};
            R dn = nrm[0] * d[0] + nrm[1] * d[1] + nrm[2] * d[2];
            if constexpr (MIXED) {
              const R nl = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
              if (fabs(dn) < R(0.05) * nl) {
                double a64 = a, b64 = b, t64 = t;
                refine_fp64<P>(V, s_cand[c0 + q], cam64, px, py, a64, b64, t64);
                a = clamp01(R(a64));
                b = clamp01(R(b64));
                t = R(t64);
                if (STATS) ++c_fp64;
              }
            }
            if (!(t > R(0))) continue;
            const bool front = (m.face & 1) ? (dn < R(0)) : (dn > R(0));
            const int nd = m.face >> 1, ad = (nd + 1) % 3, bd = (nd + 2) % 3;
            R pp[3];
            pp[nd] = (m.face & 1) ? R(1) : R(0);
            pp[ad] = R(m.a0) + a * (R(m.a1) - R(m.a0));
            pp[bd] = R(m.b0) + b * (R(m.b1) - R(m.b0));
            if constexpr (sizeof(R) == 8) {
              const FaceMeta64 m64 = V.faces64[s_cand[c0 + q]];
              pp[ad] = R(m64.a0) + a * (R(m64.a1) - R(m64.a0));
              pp[bd] = R(m64.b0) + b * (R(m64.b1) - R(m64.b0));
            }
            if (nfrag < kMaxFrags) {
              V4 rec;
              rec.x = t; rec.y = pp[0]; rec.z = pp[1]; rec.w = pp[2];
              frag_tp[(size_t)nfrag * npix + pix] = rec;
              frag_meta[(size_t)nfrag * npix + pix] = ((unsigned)m.block << 4) | ((unsigned)m.face << 1) | (front ? 1u : 0u);
              ++nfrag;
            } else {
              atomicAdd(&st->abuf_overflow, 1ull);
            }
          }
        }
      }
      __syncthreads();
    }
  }
  if (valid) frag_count[pix] = nfrag;
  if (STATS) {
    unsigned long long nf = valid ? (unsigned long long)nfrag : 0ull;
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
      c_tests += __shfl_down_sync(0xffffffffu, c_tests, o2);
      c_newton += __shfl_down_sync(0xffffffffu, c_newton, o2);
      c_fp64 += __shfl_down_sync(0xffffffffu, c_fp64, o2);
      nf += __shfl_down_sync(0xffffffffu, nf, o2);
    }
    if (lane == 0) {
      atomicAdd(&st->isect_tests, c_tests);
      atomicAdd(&st->isect_newton, c_newton);
      atomicAdd(&st->fp64_solves, c_fp64);
      atomicAdd(&st->fragments, nf);
    }
  }
}

}  // namespace

void launch_face_project(const DevVolume& V, const DevCamera<float>& cam, int4* boxes, cudaStream_t s) {
  if (V.n_faces <= 0) return;
  k0_face_project<<<(V.n_faces + 127) / 128, 128, 0, s>>>(V, cam, boxes);
}

template <typename R>
void launch_intersect(const DevVolume& V, const DevCamera<R>& cam, const DevCamera<double>& cam64, bool mixed,
                      bool stats, const int4* boxes, typename Vec4T<R>::type* frag_tp, unsigned* frag_meta,
                      int* frag_count, DevStats* st, cudaStream_t s) {
  const int tiles = ((cam.w + kTileW - 1) / kTileW) * ((cam.h + kTileH - 1) / kTileH);
  if (tiles <= 0) return;
#define IVV_K2(PP, MM, SS) \
  k2_intersect<PP, R, MM, SS><<<tiles, 256, 0, s>>>(V, cam, cam64, boxes, frag_tp, frag_meta, frag_count, st)
  if constexpr (sizeof(R) == 4) {
    if (V.P == 2) {
      if (mixed) { if (stats) IVV_K2(2, true, true); else IVV_K2(2, true, false); }
      else { if (stats) IVV_K2(2, false, true); else IVV_K2(2, false, false); }
    } else {
      if (mixed) { if (stats) IVV_K2(3, true, true); else IVV_K2(3, true, false); }
      else { if (stats) IVV_K2(3, false, true); else IVV_K2(3, false, false); }
    }
  } else {
    (void)mixed;
    if (V.P == 2) { if (stats) IVV_K2(2, false, true); else IVV_K2(2, false, false); }
    else { if (stats) IVV_K2(3, false, true); else IVV_K2(3, false, false); }
  }
#undef IVV_K2
}

template void launch_intersect<float>(const DevVolume&, const DevCamera<float>&, const DevCamera<double>&, bool,
                                      bool, const int4*, float4*, unsigned*, int*, DevStats*, cudaStream_t);
template void launch_intersect<double>(const DevVolume&, const DevCamera<double>&, const DevCamera<double>&, bool,
                                       bool, const int4*, Dbl4*, unsigned*, int*, DevStats*, cudaStream_t);

}  // namespace ivv
