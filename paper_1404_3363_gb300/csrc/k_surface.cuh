// Stage 1 (§4.1) device bodies shared by the single-frame kernels
// (k_surface.cu) and the batched kernels (k_batch.cu).  The paper rasterises
// a view-dependent pixel-accurate tessellation of the boundary surfaces; here
// every pixel ray is intersected with the Bezier face patches directly, in
// three steps:
//   K0  face_box / group box -- conservative screen box of each face patch
//       from its control points (convex hull property) and the union box of
//       each group of 32 consecutive patches (neighbours on one block face).
//   K2a cull_warp_tile -- one warp per 8x4-pixel tile (one lane per pixel):
//       group boxes, then patch boxes against the tile, then each lane's own
//       ray against the patch's screen box, bounding box and oriented box;
//       survivors are appended as (pixel, patch) items to a global list,
//       patch by patch, so that consecutive items share a patch.
//   K2b roots_item -- one thread per item: the patch's control points in the
//       ray's frame, hull test, every root of S(a,b) = o + t d (certified
//       single-root Newton or subdivision; isect.cuh), and each root appended
//       as a fragment to the pixel's slots through a per-pixel atomic counter
//       (the A-buffer of §4.2).
// No step waits on another warp: K2a is short and light, K2b carries the
// register-heavy root finding without barriers.
#pragma once

#include <cuda_runtime.h>

#include "ivv_device.cuh"

namespace ivv {

template <int P>
__device__ __forceinline__ int4 face_box(const DevVolume& V, const DevCamera<float>& cam, int f, float diag) {
  constexpr int NN = (P + 1) * (P + 1);
  return face_screen_box<NN>(cam, V.face32 + (size_t)f * NN, V.faces[f].org, diag);
}

__device__ __forceinline__ bool box_nonempty(int4 b) { return b.x <= b.z && b.y <= b.w; }
__device__ __forceinline__ bool box_meets(int4 b, int x0, int y0, int x1, int y1) {
  return b.x <= x1 && b.z >= x0 && b.y <= y1 && b.w >= y0;
}

// Screen box of local patch f (face0 + f of V) into boxes[f]; lane 0 of each
// warp writes the union of its 32 patches' boxes into gboxes[f / 32].  All 32
// lanes of the warp must call it (f = 32-aligned warp base + lane).
template <int P>
__device__ __forceinline__ void project_faces(const DevVolume& V, const DevCamera<float>& cam, int f, int nface,
                                              int face0, float diag, int4* __restrict__ boxes,
                                              int4* __restrict__ gboxes) {
  int4 b = make_int4(1, 1, 0, 0);
  if (f < nface) {
    b = face_box<P>(V, cam, face0 + f, diag);
    boxes[f] = b;
  }
  const bool ok = box_nonempty(b);
  int x0 = ok ? b.x : 0x7fffffff, y0 = ok ? b.y : 0x7fffffff;
  int x1 = ok ? b.z : -0x7fffffff, y1 = ok ? b.w : -0x7fffffff;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    x0 = min(x0, __shfl_xor_sync(0xffffffffu, x0, o));
    y0 = min(y0, __shfl_xor_sync(0xffffffffu, y0, o));
    x1 = max(x1, __shfl_xor_sync(0xffffffffu, x1, o));
    y1 = max(y1, __shfl_xor_sync(0xffffffffu, y1, o));
  }
  if ((threadIdx.x & 31) == 0 && f < nface)
    gboxes[f / kGroup] = x0 <= x1 ? make_int4(x0, y0, x1, y1) : make_int4(1, 1, 0, 0);
}

// Polish of a grazing hit with an FP64 residual (mixed precision), kept out
// of line.
template <int P>
__device__ __noinline__ void refine_fp64(const DevVolume& V, int face, const DevCamera<double>& cam64, int px, int py,
                                         double& a, double& b, double& t) {
  const FaceMeta64 m = V.faces64[face];
  double o[3], d[3];
  make_ray<double>(cam64, px, py, o, d);
  refine_hit_mixed<P>(V.face64 + (size_t)face * (P + 1) * (P + 1), V.face32 + (size_t)face * (P + 1) * (P + 1), m.org,
                      o, d, a, b, t);
}

// Stores the fragment of root (a, b) of face patch fi (FP32 depth t and
// block point pp) in the pixel's next slot.  Mixed precision: a hit within
// |cos| < kPolishCos of grazing gets the FP64 polish -- listed for the polish
// pass (k2p_polish) where the frame has a list with room, so that the FP64
// work runs on full warps, else here.
template <int P, typename R, bool MIXED, bool STATS>
__device__ __forceinline__ void emit_fragment(const DevVolume& V, const DevCamera<double>& cam64, int fi, int face,
                                              int block, int px, int py, int pix, size_t stride, R a, R b, R t,
                                              R pp[3], bool front, R cosang,
                                              typename Vec4T<R>::type* __restrict__ frag_tp,
                                              unsigned* __restrict__ frag_meta, int* __restrict__ frag_count,
                                              DevStats* __restrict__ st, unsigned long long& c_fp64,
                                              unsigned long long& c_frag) {
  typedef typename Vec4T<R>::type V4;
  if (!(t > R(0))) return;
  const int slot = atomicAdd(frag_count + pix, 1);
  if (slot >= V.max_frags) {
    atomicAdd(&st->abuf_overflow, 1ull);
    return;
  }
  if constexpr (MIXED) {
    if (cosang < R(kPolishCos)) {
      int k = V.polish_cap;
      if (V.polish != nullptr) k = atomicAdd(V.n_polish, 1);
      if (k < V.polish_cap) {
        V.polish[2 * (size_t)k] = make_float4(__int_as_float(pix), __int_as_float(slot), __int_as_float(fi), 0.f);
        V.polish[2 * (size_t)k + 1] = make_float4(float(a), float(b), float(t), 0.f);
      } else {
        double a64 = a, b64 = b, t64 = t;
        refine_fp64<P>(V, fi, cam64, px, py, a64, b64, t64);
        t = R(t64);
        const int nd = face >> 1, ad = (nd + 1) % 3, bd = (nd + 2) % 3;
        const FaceMeta64 m64 = V.faces64[fi];
        pp[ad] = R(fmin(fmax(m64.a0 + a64 * (m64.a1 - m64.a0), 0.0), 1.0));
        pp[bd] = R(fmin(fmax(m64.b0 + b64 * (m64.b1 - m64.b0), 0.0), 1.0));
        if (STATS) ++c_fp64;
      }
    }
  }
  V4 rec;
  rec.x = t; rec.y = pp[0]; rec.z = pp[1]; rec.w = pp[2];
  frag_tp[(size_t)slot * stride + pix] = rec;
  frag_meta[(size_t)slot * stride + pix] = ((unsigned)block << 4) | ((unsigned)face << 1) | (front ? 1u : 0u);
  if (STATS) ++c_frag;
}

// K2a body: tile (tx, ty) of TW x TH = 32 pixels of the window of cam, one
// lane per pixel; candidate patches face0 .. face0+nface-1 (their boxes and
// group boxes for this camera in boxes / gboxes).  Items carry the pixel's
// index pix0 + yw * cam.w + xw and tag | (the patch's index in V) (batches
// put the request into the high bits of tag).  Zeroes the fragment counters
// of the tile's pixels; returns whether the tile has any candidate (the same
// on every lane).
template <typename R, int TW, int TH>
__device__ __forceinline__ bool cull_warp_tile(const DevVolume& V, const DevCamera<R>& cam, int tx, int ty, int face0,
                                               int nface, const int4* __restrict__ boxes,
                                               const int4* __restrict__ gboxes, float diag, int pix0, int tag,
                                               int2* __restrict__ items, int cap, int* __restrict__ n_items,
                                               int* __restrict__ frag_count, DevStats* __restrict__ st) {
  static_assert(TW * TH == 32, "one lane per pixel");
  const int lane = threadIdx.x & 31;
  const int xw = tx * TW + (lane % TW), yw = ty * TH + (lane / TW);
  const bool valid = xw < cam.w && yw < cam.h;
  const int px = cam.x0 + xw, py = cam.y0 + yw;
  const int pix = pix0 + yw * cam.w + xw;
  if (valid) frag_count[pix] = 0;
  const int rx0 = cam.x0 + tx * TW, ry0 = cam.y0 + ty * TH;
  const int rx1 = min(rx0 + TW - 1, cam.x0 + cam.w - 1), ry1 = min(ry0 + TH - 1, cam.y0 + cam.h - 1);
  R o[3], d[3], inv_d[3];
  make_ray<R>(cam, px, py, o, d);
#pragma unroll
  for (int r = 0; r < 3; ++r) inv_d[r] = R(1) / d[r];
  const R pad = R(1e-6) * R(diag);
  const int ngroups = (nface + kGroup - 1) / kGroup;
  unsigned dropped = 0;
  bool any = false;
  for (int g0 = 0; g0 < ngroups; g0 += 32) {
    const int g = g0 + lane;
    const bool ghit = g < ngroups && box_meets(__ldg(gboxes + g), rx0, ry0, rx1, ry1);
    unsigned gm = __ballot_sync(0xffffffffu, ghit);
    while (gm) {
      const int gg = g0 + __ffs(gm) - 1;
      gm &= gm - 1;
      const int f = gg * kGroup + lane;
      int4 fb = make_int4(1, 1, 0, 0);
      if (f < nface) fb = __ldg(boxes + f);
      unsigned fm = __ballot_sync(0xffffffffu, box_meets(fb, rx0, ry0, rx1, ry1));
      while (fm) {
        const int fl = __ffs(fm) - 1;
        fm &= fm - 1;
        const int4 b = make_int4(__shfl_sync(0xffffffffu, fb.x, fl), __shfl_sync(0xffffffffu, fb.y, fl),
                                 __shfl_sync(0xffffffffu, fb.z, fl), __shfl_sync(0xffffffffu, fb.w, fl));
        const int fi = face0 + gg * kGroup + fl;
        bool pass = false;
        if (valid && px >= b.x && px <= b.z && py >= b.y && py <= b.w) {
          const FaceMeta& m = V.faces[fi];
          pass = ray_box<R>(o, inv_d, m.lo, m.hi, pad) && ray_obb<R>(o, d, m, R(4) * pad);
        }
        const unsigned pm = __ballot_sync(0xffffffffu, pass);
        if (pm) {
          any = true;
          int base = 0;
          if (lane == 0) base = atomicAdd(n_items, __popc(pm));
          base = __shfl_sync(0xffffffffu, base, 0);
          const int at = base + __popc(pm & ((1u << lane) - 1u));
          if (pass) {
            if (at < cap)
              items[at] = make_int2(pix, tag | fi);
            else
              ++dropped;
          }
        }
      }
    }
  }
  if (dropped) atomicAdd(&st->abuf_overflow, (unsigned long long)dropped);
  return any;
}

// K2b body: item (pixel, patch) with the pixel's ray (o, d) for pixel
// (px, py) of cam64's image; fragments at slot * stride + pix.  Takes the
// certified fast path only and returns false when the item needs the
// subdivision search (K2c).
template <int P, typename R, bool MIXED, bool STATS>
__device__ __forceinline__ bool roots_item(const DevVolume& V, const DevCamera<double>& cam64, int pix, int fi,
                                           int px, int py, const R o[3], const R d[3], float diag, size_t stride,
                                           typename Vec4T<R>::type* __restrict__ frag_tp,
                                           unsigned* __restrict__ frag_meta, int* __restrict__ frag_count,
                                           DevStats* __restrict__ st, unsigned long long& c_tests, int& c_newton,
                                           unsigned long long& c_fp64, unsigned long long& c_frag) {
  typedef typename Vec4T<R>::type V4;
  constexpr int NN = (P + 1) * (P + 1);
  const R pad = R(1e-6) * R(diag);
  R e1[3], e2[3];
  ray_frame<R>(d, e1, e2);
  const FaceMeta& m = V.faces[fi];
  R org[3], pa0, pa1, pb0, pb1;
  const V4* cp;
  if constexpr (sizeof(R) == 8) {
    const FaceMeta64 m64 = V.faces64[fi];
    org[0] = m64.org[0]; org[1] = m64.org[1]; org[2] = m64.org[2];
    pa0 = m64.a0; pa1 = m64.a1; pb0 = m64.b0; pb1 = m64.b1;
    cp = V.face64 + (size_t)fi * NN;
  } else {
    org[0] = m.org[0]; org[1] = m.org[1]; org[2] = m.org[2];
    pa0 = m.a0; pa1 = m.a1; pb0 = m.b0; pb1 = m.b1;
    cp = V.face32 + (size_t)fi * NN;
  }
  Patch2<P, R> pq;
  project_patch<P, R, V4>(cp, org, o, e1, e2, pq);
  if (!hull_has_origin<P, R>(pq, pad)) return true;
  if (STATS) ++c_tests;
  R ra[kMaxPatchRoots], rb[kMaxPatchRoots];
  int nr;
  if (!patch_roots_fast<P, R>(pq, ra, rb, nr, c_newton)) return false;
  const int face = m.face, block = m.block;
  for (int k = 0; k < nr; ++k) {
    const R a = ra[k], b = rb[k];          // within the acceptance tolerance of the patch
    R t, pp[3], cosang;
    bool front;
    make_fragment<P, R, V4>(cp, org, m, pa0, pa1, pb0, pb1, o, d, a, b, t, front, pp, cosang);
    emit_fragment<P, R, MIXED, STATS>(V, cam64, fi, face, block, px, py, pix, stride, a, b, t, pp, front, cosang,
                                      frag_tp, frag_meta, frag_count, st, c_fp64, c_frag);
  }
  return true;
}

// K2p body: the FP64 polish of listed grazing hit k (mixed precision): Newton
// on the FP64 face patch from the FP32 root, then the fragment's depth and
// block point are rewritten in its slot.
template <int P>
__device__ __forceinline__ void polish_hit(const DevVolume& V, const DevCamera<double>& cam64, int k,
                                           float4* __restrict__ frag_tp) {
  const float4 e0 = V.polish[2 * (size_t)k], e1 = V.polish[2 * (size_t)k + 1];
  const int pix = __float_as_int(e0.x), slot = __float_as_int(e0.y), fi = __float_as_int(e0.z);
  const size_t stride = (size_t)cam64.w * cam64.h;
  const int px = cam64.x0 + pix % cam64.w, py = cam64.y0 + pix / cam64.w;
  double a64 = e1.x, b64 = e1.y, t64 = e1.z;
  refine_fp64<P>(V, fi, cam64, px, py, a64, b64, t64);
  const int face = V.faces[fi].face;
  const int nd = face >> 1, ad = (nd + 1) % 3, bd = (nd + 2) % 3;
  const FaceMeta64 m64 = V.faces64[fi];
  float pp[3];
  pp[nd] = (face & 1) ? 1.f : 0.f;
  pp[ad] = float(fmin(fmax(m64.a0 + a64 * (m64.a1 - m64.a0), 0.0), 1.0));
  pp[bd] = float(fmin(fmax(m64.b0 + b64 * (m64.b1 - m64.b0), 0.0), 1.0));
  frag_tp[(size_t)slot * stride + pix] = make_float4(float(t64), pp[0], pp[1], pp[2]);
}

// ---- K2c: subdivision search of one item by a whole warp, level by level.
// The parameter boxes of patch_roots_split (isect.cuh) are visited in
// breadth-first order, starting from an 8 x 8 grid of the patch (its first
// six levels in one): at each level every lane takes boxes of the level,
// drops those whose hull misses the origin, solves certified boxes by Newton
// from their centre (a root outside the box splits it further), runs the
// multi-start Newton on uncertified boxes at the deepest level and splits
// the rest along the longer control polygon.  Roots are gathered in shared
// memory and merged by lane 0 (duplicates within the merge distance).
constexpr int kBfsCap = 128;         // boxes per level
constexpr int kSplitGrid = 8;        // first level of the warp search: a grid of boxes (1: the whole patch)
constexpr int kSplitWaves = 4;       // warp-per-item search while the items fit this many waves
constexpr int kRootCap = 16;         // gathered roots before merging

template <typename R>
struct SplitBox {
  R a0, a1, b0, b1;
  int depth;
};

constexpr int kMultiStarts = 5;     // Newton starts on an uncertified box of the deepest level
constexpr int kDeepCap = 32;        // such boxes per item solved after the levels, a start per lane

template <typename R>
struct SplitSmem {
  SplitBox<R> box[2][kBfsCap];
  SplitBox<R> deep[kDeepCap];
  R ra[kRootCap], rb[kRootCap];
  int n[2];
  int nr;
  int ndeep;
};

// Start s of the multi-start Newton on an uncertified box: its centre, then
// the centres of its four quarters.
template <typename R>
__device__ __forceinline__ void multi_start(int s0, R& a, R& b) {
  a = s0 == 0 ? R(0.5) : ((s0 & 1) ? R(0.25) : R(0.75));
  b = s0 == 0 ? R(0.5) : ((s0 & 2) ? R(0.25) : R(0.75));
}

// Root (a, b) local to box nd: kept if inside the box (tolerance scaled to
// its size) and the patch; returns false if outside the box.  in_box =
// false (uncertified smallest boxes) keeps a root anywhere in the patch, as
// accept_root (isect.cuh) does.
template <typename R>
__device__ __forceinline__ bool gather_root(const SplitBox<R>& nd, R a, R b, SplitSmem<R>& sm, bool in_box = true) {
  const R wa = nd.a1 - nd.a0, wb = nd.b1 - nd.b0;
  const R ea = RootEps<R>::accept / wa, eb = RootEps<R>::accept / wb;
  if (in_box && (a < -ea || a > R(1) + ea || b < -eb || b > R(1) + eb)) return false;
  const R ga = nd.a0 + a * wa, gb = nd.b0 + b * wb;
  const R e = RootEps<R>::accept;
  if (ga < -e || ga > R(1) + e || gb < -e || gb > R(1) + e) return true;
  const int r = atomicAdd(&sm.nr, 1);
  if (r < kRootCap) {
    sm.ra[r] = ga;
    sm.rb[r] = gb;
  }
  return true;
}

// All lanes of the warp call it; returns the merged roots in sm.ra/rb[0..n)
// (n <= kMaxPatchRoots, the same on every lane).
template <int P, typename R>
__device__ __forceinline__ int split_roots_warp(const Patch2<P, R>& q0, R pad, SplitSmem<R>& sm, int& iters,
                                                unsigned& dropped) {
  constexpr int N = P + 1;
  const int lane = threadIdx.x & 31;
  // the uncertified patch is split into a kSplitGrid x kSplitGrid grid of
  // boxes at once (one level of the warp search instead of 2 log2 kSplitGrid)
  constexpr int G = kSplitGrid;
  for (int k = lane; k < G * G; k += 32) {
    const int ia = k % G, ib = k / G;
    const R w = R(1) / R(G);
    sm.box[0][k] = SplitBox<R>{R(ia) * w, R(ia + 1) * w, R(ib) * w, R(ib + 1) * w, G == 1 ? 0 : 2 * (31 - __clz(G))};
  }
  if (lane == 0) {
    sm.n[0] = G * G;
    sm.n[1] = 0;
    sm.nr = 0;
    sm.ndeep = 0;
  }
  __syncwarp();
  int cur = 0;
#pragma unroll 1
  for (int level = 0; level <= kSplitDepth; ++level) {
    const int n = min(sm.n[cur], kBfsCap);
    if (n == 0) break;
#pragma unroll 1
    for (int k = lane; k < n; k += 32) {
      const SplitBox<R> nd = sm.box[cur][k];
      Patch2<P, R> q;
      sub_patch<P, R>(q0, nd.a0, nd.a1, nd.b0, nd.b1, q);
      if (!hull_has_origin<P, R>(q, pad)) continue;
      bool split = true;
      if (fixed_jacobian_sign<P, R>(q)) {
        R a = R(0.5), b = R(0.5);
        split = !(newton2<P, R>(q, a, b, iters, kBoxNewtonLo<R>(), kBoxNewtonHi<R>(), kBoxNewtonIters) &&
                  gather_root<R>(nd, a, b, sm));
      } else if (nd.depth >= kSplitDepth) {
        // the multi-start Newton of an uncertified deepest box runs after
        // the levels with one start per lane (its starts are independent);
        // boxes beyond the list run their starts here
        const int at = atomicAdd(&sm.ndeep, 1);
        if (at < kDeepCap) {
          sm.deep[at] = nd;
        } else {
#pragma unroll 1
          for (int s0 = 0; s0 < kMultiStarts; ++s0) {
            R a, b;
            multi_start<R>(s0, a, b);
            if (newton2<P, R>(q, a, b, iters)) gather_root<R>(nd, a, b, sm, false);
          }
        }
        split = false;
      }
      if (!split || nd.depth >= kSplitDepth) continue;
      R la = 0, lb = 0;
#pragma unroll
      for (int t = 0; t < N; ++t) {
        la += fabs(q.x[t * N + P] - q.x[t * N]) + fabs(q.y[t * N + P] - q.y[t * N]);
        lb += fabs(q.x[P * N + t] - q.x[t]) + fabs(q.y[P * N + t] - q.y[t]);
      }
      SplitBox<R> lo = nd, hi = nd;
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
      const int at = atomicAdd(&sm.n[cur ^ 1], 2);
      if (at + 2 <= kBfsCap) {
        sm.box[cur ^ 1][at] = lo;
        sm.box[cur ^ 1][at + 1] = hi;
      } else {
        ++dropped;
      }
    }
    __syncwarp();
    if (lane == 0) sm.n[cur] = 0;
    __syncwarp();
    cur ^= 1;
  }
  // the deepest uncertified boxes: every (box, start) pair on its own lane
  const int nd_deep = min(sm.ndeep, kDeepCap);
#pragma unroll 1
  for (int k = lane; k < nd_deep * kMultiStarts; k += 32) {
    const SplitBox<R> nd = sm.deep[k / kMultiStarts];
    Patch2<P, R> q;
    sub_patch<P, R>(q0, nd.a0, nd.a1, nd.b0, nd.b1, q);
    R a, b;
    multi_start<R>(k % kMultiStarts, a, b);
    if (newton2<P, R>(q, a, b, iters)) gather_root<R>(nd, a, b, sm, false);
  }
  __syncwarp();
  // merge duplicates (lane 0), keep at most kMaxPatchRoots
  if (lane == 0) {
    const int m = min(sm.nr, kRootCap);
    int kept = 0;
    for (int r = 0; r < m && kept < kMaxPatchRoots; ++r) {
      bool dup = false;
      for (int k = 0; k < kept; ++k)
        if (fabs(sm.ra[k] - sm.ra[r]) + fabs(sm.rb[k] - sm.rb[r]) < RootEps<R>::dup) dup = true;
      if (!dup) {
        sm.ra[kept] = sm.ra[r];
        sm.rb[kept] = sm.rb[r];
        ++kept;
      }
    }
    sm.nr = kept;
  }
  __syncwarp();
  return sm.nr;
}

// K2c body for one deferred item (all lanes of the warp, same item): the
// warp search, then one lane per root writes its fragment.
template <int P, typename R, bool MIXED, bool STATS>
__device__ __forceinline__ void split_item_warp(const DevVolume& V, const DevCamera<double>& cam64, int pix, int fi,
                                                int px, int py, const R o[3], const R d[3], float diag, size_t stride,
                                                typename Vec4T<R>::type* __restrict__ frag_tp,
                                                unsigned* __restrict__ frag_meta, int* __restrict__ frag_count,
                                                DevStats* __restrict__ st, SplitSmem<R>& sm, int& c_newton,
                                                unsigned long long& c_fp64, unsigned long long& c_frag,
                                                unsigned& dropped) {
  typedef typename Vec4T<R>::type V4;
  constexpr int NN = (P + 1) * (P + 1);
  const R pad = R(1e-6) * R(diag);
  R e1[3], e2[3];
  ray_frame<R>(d, e1, e2);
  const FaceMeta& m = V.faces[fi];
  R org[3], pa0, pa1, pb0, pb1;
  const V4* cp;
  if constexpr (sizeof(R) == 8) {
    const FaceMeta64 m64 = V.faces64[fi];
    org[0] = m64.org[0]; org[1] = m64.org[1]; org[2] = m64.org[2];
    pa0 = m64.a0; pa1 = m64.a1; pb0 = m64.b0; pb1 = m64.b1;
    cp = V.face64 + (size_t)fi * NN;
  } else {
    org[0] = m.org[0]; org[1] = m.org[1]; org[2] = m.org[2];
    pa0 = m.a0; pa1 = m.a1; pb0 = m.b0; pb1 = m.b1;
    cp = V.face32 + (size_t)fi * NN;
  }
  Patch2<P, R> pq;
  project_patch<P, R, V4>(cp, org, o, e1, e2, pq);
  const int nr = split_roots_warp<P, R>(pq, pad, sm, c_newton, dropped);
  const int lane = threadIdx.x & 31;
  if (lane < nr) {
    const R a = sm.ra[lane], b = sm.rb[lane];   // within the acceptance tolerance of the patch
    R t, pp[3], cosang;
    bool front;
    make_fragment<P, R, V4>(cp, org, m, pa0, pa1, pb0, pb1, o, d, a, b, t, front, pp, cosang);
    emit_fragment<P, R, MIXED, STATS>(V, cam64, fi, m.face, m.block, px, py, pix, stride, a, b, t, pp, front, cosang,
                                      frag_tp, frag_meta, frag_count, st, c_fp64, c_frag);
  }
  __syncwarp();
}

// K2c body, one thread per deferred item (many deferred items): the
// depth-first subdivision search of isect.cuh, then the fragments.
template <int P, typename R, bool MIXED, bool STATS>
__device__ __forceinline__ void split_item_thread(const DevVolume& V, const DevCamera<double>& cam64, int pix, int fi,
                                                  int px, int py, const R o[3], const R d[3], float diag,
                                                  size_t stride, typename Vec4T<R>::type* __restrict__ frag_tp,
                                                  unsigned* __restrict__ frag_meta, int* __restrict__ frag_count,
                                                  DevStats* __restrict__ st, int& c_newton,
                                                  unsigned long long& c_fp64, unsigned long long& c_frag) {
  typedef typename Vec4T<R>::type V4;
  constexpr int NN = (P + 1) * (P + 1);
  const R pad = R(1e-6) * R(diag);
  R e1[3], e2[3];
  ray_frame<R>(d, e1, e2);
  const FaceMeta& m = V.faces[fi];
  R org[3], pa0, pa1, pb0, pb1;
  const V4* cp;
  if constexpr (sizeof(R) == 8) {
    const FaceMeta64 m64 = V.faces64[fi];
    org[0] = m64.org[0]; org[1] = m64.org[1]; org[2] = m64.org[2];
    pa0 = m64.a0; pa1 = m64.a1; pb0 = m64.b0; pb1 = m64.b1;
    cp = V.face64 + (size_t)fi * NN;
  } else {
    org[0] = m.org[0]; org[1] = m.org[1]; org[2] = m.org[2];
    pa0 = m.a0; pa1 = m.a1; pb0 = m.b0; pb1 = m.b1;
    cp = V.face32 + (size_t)fi * NN;
  }
  Patch2<P, R> pq;
  project_patch<P, R, V4>(cp, org, o, e1, e2, pq);
  R ra[kMaxPatchRoots], rb[kMaxPatchRoots];
  const int nr = patch_roots_split<P, R>(&pq, pad, ra, rb, c_newton);
  const int face = m.face, block = m.block;
  for (int k = 0; k < nr; ++k) {
    const R a = ra[k], b = rb[k];          // within the acceptance tolerance of the patch
    R t, pp[3], cosang;
    bool front;
    make_fragment<P, R, V4>(cp, org, m, pa0, pa1, pb0, pb1, o, d, a, b, t, front, pp, cosang);
    emit_fragment<P, R, MIXED, STATS>(V, cam64, fi, face, block, px, py, pix, stride, a, b, t, pp, front, cosang,
                                      frag_tp, frag_meta, frag_count, st, c_fp64, c_frag);
  }
}

// K2c thread form with the deepest multi-starts shared by the warp: each
// lane runs the depth-first search of patch_roots_split (isect.cuh) for its
// own item, but the uncertified boxes of the deepest level -- whose five
// Newton starts would hold the warp while one lane runs them -- go to a
// warp list; once every lane's search is done the warp runs the list with
// one (box, start) pair per lane and hands the roots back to their items.
constexpr int kWarpDeepCap = 64;      // deferred boxes per warp and round of 32 items

template <int P>
struct ThreadDeepSmem {
  Patch2<P, float> q[32];             // each lane's projected patch
  SplitBox<float> box[kWarpDeepCap];
  int owner[kWarpDeepCap];
  float2 root[kWarpDeepCap * kMultiStarts];   // per (box, start): the root in patch coordinates, or NaN
  int n;
};

// patch_roots_split with the deepest uncertified boxes deferred to dm
// (inline once the list is full).
template <int P>
__device__ __forceinline__ int split_roots_defer(const Patch2<P, float>& q0, float pad, float* ra, float* rb,
                                                 int& iters, ThreadDeepSmem<P>& dm, int lane) {
  typedef float R;
  constexpr int N = P + 1;
  SplitBox<R> stack[kSplitDepth + 1];
  stack[0] = SplitBox<R>{R(0), R(1), R(0), R(1), 0};
  int sp = 1, nr = 0;
  while (sp > 0) {
    const SplitBox<R> nd = stack[--sp];
    Patch2<P, R> q;
    sub_patch<P, R>(q0, nd.a0, nd.a1, nd.b0, nd.b1, q);
    if (!hull_has_origin<P, R>(q, pad)) continue;
    bool split = true;
    if (fixed_jacobian_sign<P, R>(q)) {
      R a = R(0.5), b = R(0.5);
      split = !(newton2<P, R>(q, a, b, iters, kBoxNewtonLo<R>(), kBoxNewtonHi<R>(), kBoxNewtonIters) &&
                accept_root<R>(a, b, nd.a0, nd.a1, nd.b0, nd.b1, ra, rb, nr));
    } else if (nd.depth >= kSplitDepth) {
      const int at = atomicAdd(&dm.n, 1);
      if (at < kWarpDeepCap) {
        dm.box[at] = nd;
        dm.owner[at] = lane;
      } else {
#pragma unroll 1
        for (int s0 = 0; s0 < kMultiStarts; ++s0) {
          R a, b;
          multi_start<R>(s0, a, b);
          if (newton2<P, R>(q, a, b, iters)) accept_root<R>(a, b, nd.a0, nd.a1, nd.b0, nd.b1, ra, rb, nr, false);
        }
      }
      split = false;
    }
    if (!split || nd.depth >= kSplitDepth || sp + 2 > kSplitDepth + 1) continue;
    R la = 0, lb = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      la += fabs(q.x[k * N + P] - q.x[k * N]) + fabs(q.y[k * N + P] - q.y[k * N]);
      lb += fabs(q.x[P * N + k] - q.x[k]) + fabs(q.y[P * N + k] - q.y[k]);
    }
    SplitBox<R>& hi = stack[sp];
    SplitBox<R>& lo = stack[sp + 1];       // lower half is processed next
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

// One round of the thread form (all lanes of the warp call it; lanes with
// have = false only help with the deferred boxes): the lane's item
// (pixel pix, face patch fi, ray o + t d of pixel (px, py) of cam64's image),
// then its fragments.
template <int P, bool MIXED, bool STATS>
__device__ __forceinline__ void split_round_thread(const DevVolume& V, const DevCamera<double>& cam64, bool have,
                                                   int pix, int fi, int px, int py, const float o[3],
                                                   const float d[3], float diag, size_t stride,
                                                   float4* __restrict__ frag_tp, unsigned* __restrict__ frag_meta,
                                                   int* __restrict__ frag_count, DevStats* __restrict__ st,
                                                   ThreadDeepSmem<P>& dm, int& c_newton,
                                                   unsigned long long& c_fp64, unsigned long long& c_frag) {
  typedef float R;
  constexpr int NN = (P + 1) * (P + 1);
  const int lane = threadIdx.x & 31;
  if (lane == 0) dm.n = 0;
  __syncwarp();
  const R pad = R(1e-6) * R(diag);
  R ra[kMaxPatchRoots], rb[kMaxPatchRoots];
  int nr = 0;
  const FaceMeta* m = nullptr;
  R org[3] = {0, 0, 0};
  const float4* cp = nullptr;
  if (have) {
    R e1[3], e2[3];
    ray_frame<R>(d, e1, e2);
    m = &V.faces[fi];
    org[0] = m->org[0]; org[1] = m->org[1]; org[2] = m->org[2];
    cp = V.face32 + (size_t)fi * NN;
    project_patch<P, R, float4>(cp, org, o, e1, e2, dm.q[lane]);
    nr = split_roots_defer<P>(dm.q[lane], pad, ra, rb, c_newton, dm, lane);
  }
  __syncwarp();
  const int nd_deep = min(dm.n, kWarpDeepCap);
#pragma unroll 1
  for (int k = lane; k < nd_deep * kMultiStarts; k += 32) {
    const SplitBox<R> nd = dm.box[k / kMultiStarts];
    Patch2<P, R> q;
    sub_patch<P, R>(dm.q[dm.owner[k / kMultiStarts]], nd.a0, nd.a1, nd.b0, nd.b1, q);
    R a, b;
    multi_start<R>(k % kMultiStarts, a, b);
    float2 r = make_float2(__int_as_float(0x7fffffff), 0.f);
    if (newton2<P, R>(q, a, b, c_newton)) r = make_float2(nd.a0 + a * (nd.a1 - nd.a0), nd.b0 + b * (nd.b1 - nd.b0));
    dm.root[k] = r;
  }
  __syncwarp();
  if (have) {
    // the item's roots from its deferred boxes, in the order the search
    // deferred them, merged as the inline search merges (accept_root)
    for (int k = 0; k < nd_deep * kMultiStarts; ++k) {
      if (dm.owner[k / kMultiStarts] != lane) continue;
      const float2 r = dm.root[k];
      if (r.x == r.x) accept_root<R>(r.x, r.y, R(0), R(1), R(0), R(1), ra, rb, nr, false);
    }
    const R pa0 = m->a0, pa1 = m->a1, pb0 = m->b0, pb1 = m->b1;
    for (int k = 0; k < nr; ++k) {
      const R a = ra[k], b = rb[k];          // within the acceptance tolerance of the patch
      R t, pp[3], cosang;
      bool front;
      make_fragment<P, R, float4>(cp, org, *m, pa0, pa1, pb0, pb1, o, d, a, b, t, front, pp, cosang);
      emit_fragment<P, R, MIXED, STATS>(V, cam64, fi, m->face, m->block, px, py, pix, stride, a, b, t, pp, front,
                                        cosang, frag_tp, frag_meta, frag_count, st, c_fp64, c_frag);
    }
  }
  __syncwarp();
}

// Appends item i to the list of items that need the subdivision search
// (count at n_items[kSlowCounter - kItemCounter]).
__device__ __forceinline__ void defer_item(int i, int* __restrict__ slow, int cap, int* __restrict__ n_items) {
  const int k = atomicAdd(n_items + (kSlowCounter - kItemCounter), 1);
  if (k < cap) slow[k] = i;
}

// Next 32 consecutive items for the calling warp (all lanes call it), from
// the hand-out head at n_items[kItemHead - kItemCounter]; returns the first
// or n when none are left.
__device__ __forceinline__ int take_items(int* __restrict__ n_items, int n, int head = kItemHead) {
  int base = 0;
  if ((threadIdx.x & 31) == 0) base = atomicAdd(n_items + (head - kItemCounter), 32);
  base = __shfl_sync(0xffffffffu, base, 0);
  return base < n ? base : n;
}

// Counters of K2b / K2c, one atomic per warp; n = items of the launch
// (K2b: all items, K2c: items that needed the subdivision search).
template <bool STATS, bool SPLIT>
__device__ __forceinline__ void roots_counters(unsigned long long c_tests, int c_newton, unsigned long long c_fp64,
                                               unsigned long long c_frag, int n, DevStats* __restrict__ st) {
  if (!STATS) return;
  if (blockIdx.x == 0 && threadIdx.x == 0)
    atomicAdd(SPLIT ? &st->isect_split : &st->isect_items, (unsigned long long)n);
  unsigned long long cn = (unsigned long long)c_newton;
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) {
    c_tests += __shfl_down_sync(0xffffffffu, c_tests, o2);
    cn += __shfl_down_sync(0xffffffffu, cn, o2);
    c_fp64 += __shfl_down_sync(0xffffffffu, c_fp64, o2);
    c_frag += __shfl_down_sync(0xffffffffu, c_frag, o2);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&st->isect_tests, c_tests);
    atomicAdd(&st->isect_newton, cn);
    atomicAdd(&st->fp64_solves, c_fp64);
    atomicAdd(&st->fragments, c_frag);
  }
}

}  // namespace ivv
