// Stage 1 (§4.1) device bodies shared by the single-frame kernels
// (k_surface.cu) and the batched kernels (k_batch.cu).
//   face_box    -- conservative screen box of one face patch from its control
//                  points (convex hull property).
//   k2_tile     -- one CTA per TW x TH screen tile: cull the face boxes
//                  against the tile and stage the surviving patches in shared
//                  memory; every pixel tests its ray against each staged
//                  patch's screen box and bounding box and queues the
//                  survivors in a tile work list, which all threads then drain
//                  densely: every root of S(a,b) = o + t d (hull test,
//                  certified single-root Newton or subdivision; isect.cuh)
//                  becomes a fragment appended to the pixel's slots through a
//                  per-pixel atomic counter in shared memory (the A-buffer of
//                  §4.2).
#pragma once

#include <cuda_runtime.h>

#include "ivv_device.cuh"

namespace ivv {

template <int P>
__device__ __forceinline__ int4 face_box(const DevVolume& V, const DevCamera<float>& cam, int f, float diag) {
  constexpr int NN = (P + 1) * (P + 1);
  return face_screen_box<NN>(cam, V.face32 + (size_t)f * NN, V.faces[f].org, diag);
}

// FP64 polish of a grazing hit (mixed precision), kept out of line.
template <int P>
__device__ __noinline__ void refine_fp64(const DevVolume& V, int face, const DevCamera<double>& cam64, int px, int py,
                                         double& a, double& b, double& t) {
  const FaceMeta64 m = V.faces64[face];
  double o[3], d[3];
  make_ray<double>(cam64, px, py, o, d);
  refine_hit_fp64<P, Dbl4>(V.face64 + (size_t)face * (P + 1) * (P + 1), m.org, o, d, a, b, t);
}

// Fragments of tile (tx, ty) of the window of `cam`.  Faces face0 ..
// face0+nface-1 of V are candidates; boxes[f] is the screen box of face
// face0+f.  Pixel (xw, yw) of the window writes its slots at index
// slot * stride + pix0 + yw * cam.w + xw and its count at pix0 + yw * cam.w + xw.
template <int P, typename R, bool MIXED, bool STATS, int TW, int TH>
__device__ __forceinline__ void k2_tile(const DevVolume& V, const DevCamera<R>& cam, const DevCamera<double>& cam64,
                                        int tx, int ty, int face0, int nface, const int4* __restrict__ boxes,
                                        float diag, size_t pix0, size_t stride,
                                        typename Vec4T<R>::type* __restrict__ frag_tp,
                                        unsigned* __restrict__ frag_meta, int* __restrict__ frag_count,
                                        DevStats* __restrict__ st) {
  typedef typename Vec4T<R>::type V4;
  constexpr int N = P + 1, NN = N * N;
  constexpr int CH = 32;                       // face patches staged per round
  constexpr int kThreads = TW * TH;            // one thread per tile pixel
  static_assert(kThreads % 32 == 0 && kThreads <= 1024, "tile must be whole warps");
  __shared__ int s_cand[kThreads];
  __shared__ int s_wcnt[kThreads / 32];
  __shared__ V4 s_cp[CH * NN];
  __shared__ FaceMeta s_meta[CH];
  __shared__ int4 s_box[CH];
  __shared__ R s_o[kThreads][3], s_d[kThreads][3];
  __shared__ unsigned short s_work[kThreads * CH];   // (pixel << 5) | staged face
  __shared__ int s_nwork;
  __shared__ int s_count[kThreads];                  // fragments per tile pixel
  (void)N;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int xw = tx * TW + (tid % TW), yw = ty * TH + (tid / TW);
  const bool valid = xw < cam.w && yw < cam.h;
  const int px = cam.x0 + xw, py = cam.y0 + yw;
  const int rx0 = cam.x0 + tx * TW, ry0 = cam.y0 + ty * TH;
  const int rx1 = min(rx0 + TW - 1, cam.x0 + cam.w - 1), ry1 = min(ry0 + TH - 1, cam.y0 + cam.h - 1);

  R o[3], d[3], inv_d[3];
  make_ray<R>(cam, px, py, o, d);
#pragma unroll
  for (int r = 0; r < 3; ++r) inv_d[r] = R(1) / d[r];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    s_o[tid][r] = o[r];
    s_d[tid][r] = d[r];
  }
  s_count[tid] = 0;
  if (tid == 0) s_nwork = 0;
  const R hull_pad = R(1e-6) * R(diag);
  int c_newton = 0;
  unsigned long long c_tests = 0, c_fp64 = 0;

  for (int base = 0; base < nface; base += kThreads) {
    // ---- faces whose screen box meets the tile, in index order
    const int f = base + tid;
    bool keep = false;
    int4 fb = make_int4(1, 1, 0, 0);
    if (f < nface) {
      fb = __ldg(boxes + f);
      keep = fb.x <= rx1 && fb.z >= rx0 && fb.y <= ry1 && fb.w >= ry0;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) s_wcnt[warp] = __popc(bal);
    __syncthreads();
    int off = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) {
      const int c = s_wcnt[w];
      off += (w < warp) ? c : 0;
      total += c;
    }
    if (keep) s_cand[off + __popc(bal & ((1u << lane) - 1u))] = f;
    __syncthreads();
    for (int c0 = 0; c0 < total; c0 += CH) {
      const int nst = min(CH, total - c0);
      for (int q = tid; q < nst * NN; q += kThreads) {
        const int fi = face0 + s_cand[c0 + q / NN];
        if constexpr (sizeof(R) == 4) {
          s_cp[q] = __ldg(V.face32 + (size_t)fi * NN + (q % NN));
        } else {
          s_cp[q] = V.face64[(size_t)fi * NN + (q % NN)];
        }
      }
      for (int q = tid; q < nst; q += kThreads) {
        s_meta[q] = V.faces[face0 + s_cand[c0 + q]];
        s_box[q] = __ldg(boxes + s_cand[c0 + q]);
      }
      __syncthreads();
      // ---- cheap per-pixel tests; survivors go to the tile's work list
      for (int q = 0; q < nst; ++q) {
        bool pass = false;
        if (valid) {
          const int4 b = s_box[q];
          pass = px >= b.x && px <= b.z && py >= b.y && py <= b.w &&
                 ray_box<R>(o, inv_d, s_meta[q].lo, s_meta[q].hi, hull_pad) &&
                 ray_obb<R>(o, d, s_meta[q], R(4) * hull_pad);
        }
        const unsigned wb = __ballot_sync(0xffffffffu, pass);
        if (wb) {
          int wbase = 0;
          if (lane == 0) wbase = atomicAdd(&s_nwork, __popc(wb));
          wbase = __shfl_sync(0xffffffffu, wbase, 0);
          if (pass) s_work[wbase + __popc(wb & ((1u << lane) - 1u))] = (unsigned short)((tid << 5) | q);
        }
      }
      __syncthreads();
      // ---- ray/patch roots, one (pixel, face) item per thread
      const int nwork = s_nwork;
      for (int w = tid; w < nwork; w += kThreads) {
        const int item = s_work[w];
        const int pl = item >> 5, qf = item & 31;
        const FaceMeta& m = s_meta[qf];
        R ro[3], rd[3], e1[3], e2[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          ro[r] = s_o[pl][r];
          rd[r] = s_d[pl][r];
        }
        ray_frame<R>(rd, e1, e2);
        const int fi = face0 + s_cand[c0 + qf];
        R org[3], pa0, pa1, pb0, pb1;
        if constexpr (sizeof(R) == 8) {
          const FaceMeta64 m64 = V.faces64[fi];
          org[0] = m64.org[0]; org[1] = m64.org[1]; org[2] = m64.org[2];
          pa0 = m64.a0; pa1 = m64.a1; pb0 = m64.b0; pb1 = m64.b1;
        } else {
          org[0] = m.org[0]; org[1] = m.org[1]; org[2] = m.org[2];
          pa0 = m.a0; pa1 = m.a1; pb0 = m.b0; pb1 = m.b1;
        }
        const V4* cp = s_cp + qf * NN;
        Patch2<P, R> pq;
        project_patch<P, R, V4>(cp, org, ro, e1, e2, pq);
        if (!hull_has_origin<P, R>(pq, hull_pad)) continue;
        if (STATS) ++c_tests;
        R ra[kMaxPatchRoots], rb[kMaxPatchRoots];
        const int nr = patch_roots<P, R>(pq, hull_pad, ra, rb, c_newton);
        const int ppx = rx0 + (pl % TW), ppy = ry0 + (pl / TW);
        const size_t ppix = pix0 + (size_t)((ppy - cam.y0) * cam.w + (ppx - cam.x0));
        for (int k = 0; k < nr; ++k) {
          R a = clamp01r(ra[k]), b = clamp01r(rb[k]);
          R t, pp[3], cosang;
          bool front;
          make_fragment<P, R, V4>(cp, org, m, pa0, pa1, pb0, pb1, ro, rd, a, b, t, front, pp, cosang);
          if constexpr (MIXED) {
            if (cosang < R(0.2)) {
              double a64 = a, b64 = b, t64 = t;
              refine_fp64<P>(V, fi, cam64, ppx, ppy, a64, b64, t64);
              a64 = a64 < 0.0 ? 0.0 : (a64 > 1.0 ? 1.0 : a64);
              b64 = b64 < 0.0 ? 0.0 : (b64 > 1.0 ? 1.0 : b64);
              t = R(t64);
              const int nd = m.face >> 1, ad = (nd + 1) % 3, bd = (nd + 2) % 3;
              const FaceMeta64 m64 = V.faces64[fi];
              pp[ad] = R(m64.a0 + a64 * (m64.a1 - m64.a0));
              pp[bd] = R(m64.b0 + b64 * (m64.b1 - m64.b0));
              if (STATS) ++c_fp64;
            }
          }
          if (!(t > R(0))) continue;
          const int slot = atomicAdd(&s_count[pl], 1);
          if (slot < kMaxFrags) {
            V4 rec;
            rec.x = t; rec.y = pp[0]; rec.z = pp[1]; rec.w = pp[2];
            frag_tp[(size_t)slot * stride + ppix] = rec;
            frag_meta[(size_t)slot * stride + ppix] =
                ((unsigned)m.block << 4) | ((unsigned)m.face << 1) | (front ? 1u : 0u);
          } else {
            atomicAdd(&st->abuf_overflow, 1ull);
          }
        }
      }
      __syncthreads();
      if (tid == 0) s_nwork = 0;
      __syncthreads();
    }
  }
  const int nfrag = min(s_count[tid], kMaxFrags);
  if (valid) frag_count[pix0 + (size_t)(yw * cam.w + xw)] = nfrag;
  if (STATS) {
    unsigned long long nf = valid ? (unsigned long long)nfrag : 0ull;
    unsigned long long cn = (unsigned long long)c_newton;
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
      c_tests += __shfl_down_sync(0xffffffffu, c_tests, o2);
      cn += __shfl_down_sync(0xffffffffu, cn, o2);
      c_fp64 += __shfl_down_sync(0xffffffffu, c_fp64, o2);
      nf += __shfl_down_sync(0xffffffffu, nf, o2);
    }
    if (lane == 0) {
      atomicAdd(&st->isect_tests, c_tests);
      atomicAdd(&st->isect_newton, cn);
      atomicAdd(&st->fp64_solves, c_fp64);
      atomicAdd(&st->fragments, nf);
    }
  }
}

}  // namespace ivv
