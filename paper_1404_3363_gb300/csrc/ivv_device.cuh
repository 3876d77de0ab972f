// Device-side data layout and helpers shared by the kernels.
//
// Layout in HBM (uploaded once per volume):
//   elem   [E][(P+1)^3] float4 (x, y, z, rho) -- Bezier control points of every
//          element, index (i*(P+1)+j)*(P+1)+k with i along u, j along v, k along w
//          (w innermost, so the first contraction streams contiguous float4s);
//          x, y, z relative to the element origin elem_org[E] (its first
//          control point), which keeps FP32 partial derivatives accurate
//   elem64 the same in double ([E][(P+1)^3][4])
//   face   [F][(P+1)^2] float4 (x, y, z, 0) -- boundary face patches, a fastest,
//          relative to the face origin in FaceMeta
//   brk    breakpoints of every block and direction (float and double copies)
// All spline work is Bernstein evaluation of a single element: the geometry
// phi = sum B_i(u) B_j(v) B_k(w) C_ijk (Eq. 1 restricted to one element) with
// first partials by the same sum-factorised contraction.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "ivv_internal.h"
#include "isect.cuh"
#include "strain.h"

namespace ivv {

// Programmatic dependent launch: a kernel launched by launch_pdl may become
// resident while its predecessor on the stream finishes (hiding the launch
// gap between dependent kernels).  Every such kernel calls pdl_wait(), which
// returns once the predecessor grid has completed and its writes are visible,
// unconditionally and before it reads or writes any buffer another kernel of
// the frame touches; so a grid completes only after all earlier ones did.
// Launch errors land in cudaGetLastError as for <<<>>>.  pdl_wait() returns
// at once in a kernel launched the ordinary way.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// The integrators' pixel queue (the active list, consumed through one
// global counter).  A warp takes new pixels only once all its lanes are
// idle, one consecutive item per lane: its lanes then trace neighbouring
// pixels that start together, so their rays run through the same elements
// and their control-point loads coalesce (a lane whose pixel ends early sits
// out, issuing no loads, until its warp refills).  With a block chunk in
// shared memory, a warp's 32 items are cut from 128 consecutive items that
// the block's warps share while the queue is long, so the pixels in flight
// on a block are neighbours too.
struct WarpQueue {
  unsigned drained;             // lanes that found the queue empty (warp-uniform)
  int blk_until;                // block chunks while their base is below this
  unsigned long long* chunk;    // the block's chunk (base << 32 | items handed out), or null
  // With a block chunk every thread of the block constructs it (it
  // synchronises the block).
  __device__ __forceinline__ WarpQueue(int nact, int* queue_head, unsigned long long* s_chunk)
      : drained(0u), blk_until(nact - 2 * 128 * (int)gridDim.x), chunk(s_chunk) {
    if (chunk != nullptr) {
      if (threadIdx.x == 0)
        *chunk = blk_until > 0 ? ((unsigned long long)(unsigned)atomicAdd(queue_head, 128) << 32) : 128ull;
      __syncthreads();
    }
  }
  __device__ __forceinline__ bool done() const { return drained == 0xffffffffu; }
  // Every lane of an idle warp calls it; returns the item of each lane that
  // is not drained (the caller marks lanes whose item is past the end).
  __device__ __forceinline__ int take(int lane, int* queue_head) {
    const unsigned need = ~drained;
    const int nneed = __popc(need);
    const int rank = __popc(need & ((1u << lane) - 1u));
    int base = 0;
    const int leader = __ffs(need) - 1;
    if (lane == leader) {
      if (chunk != nullptr && nneed == 32) {
        const unsigned long long old = atomicAdd(chunk, 32ull);
        const unsigned taken = (unsigned)old;
        const int cb = (int)(old >> 32);
        if (taken < 128u) {
          base = cb + (int)taken;
        } else if (taken == 128u && cb + 128 < blk_until) {
          base = atomicAdd(queue_head, 128);                // a fresh chunk; its first 32 are ours
          atomicExch(chunk, ((unsigned long long)(unsigned)base << 32) | 32ull);
        } else {
          base = atomicAdd(queue_head, 32);
        }
      } else {
        base = atomicAdd(queue_head, nneed);
      }
    }
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + rank;
  }
};

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args&&... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}


// ------------------------------------------------------------- parameters
// 32-byte aligned four-double vector (x, y, z, w).
struct __align__(32) Dbl4 {
  double x, y, z, w;
};

template <typename R> struct Vec4T;
template <> struct Vec4T<float> { typedef float4 type; };
template <> struct Vec4T<double> { typedef Dbl4 type; };

struct DevVolume {
  int P, mode, n_blocks, n_faces;
  const BlockInfo* blocks;
  const float* brk32;
  const double* brk64;
  const float4* elem32;
  const Dbl4* elem64;
  const float4* org32;
  const float* rho32;     // scalar control points alone, rho_stride32(P) per element (NULL in batches)
  const Dbl4* org64;
  // IVV_SCALAR_VONMISES: the displacement u as Bezier elements with their
  // origins, the geometry's layout (null in other modes)
  const float4* disp32;
  const float4* dorg32;
  const Dbl4* disp64;
  const Dbl4* dorg64;
  const float4* face32;
  const Dbl4* face64;
  const FaceMeta* faces;
  const FaceMeta64* faces64;
  float diag;
  int max_frags;          // fragment slots in use per pixel (<= kMaxFrags)
  int max_newton;         // Newton iterations of a per-point inversion (RF method, point location)
  // per frame, mixed precision: the list of grazing hits whose FP64 polish
  // is deferred to its own pass (two float4 per hit), or null (inline polish)
  float4* polish;
  int polish_cap;
  int* n_polish;
};

struct DevTF {
  int n;
  float sigma, lo, inv_range;
  const float* r;       // [n]
  const float4* rgba;   // [n]
};

// Per-launch counters; the overflow/cap counters are always maintained.
struct DevStats {
  unsigned long long rays, pairs, fragments, samples, rk_steps, rk_rejects, rhs_evals,
      isect_newton, isect_tests, fp64_solves, abuf_overflow, pair_overflow, unmatched, step_cap, rf_newton_iters,
      rf_unconverged, isect_items, isect_split, rho_evals, entry_shrinks, entry_newton, async_timeouts;
  unsigned int max_delta_p_bits;   // float bits of max Delta P (non-negative: int order)
  unsigned int pad;
};

// ------------------------------------------------------------- helpers
template <typename R> __device__ __forceinline__ R rcp_(R x) { return R(1) / x; }

template <int P, typename R>
__device__ __forceinline__ void bernstein(R x, R b[P + 1], R db[P + 1]) {
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

template <int P, typename R>
__device__ __forceinline__ void bernstein_v(R x, R b[P + 1]) {
  const R y = R(1) - x;
  if (P == 2) {
    b[0] = y * y; b[1] = R(2) * x * y; b[2] = x * x;
  } else {
    const R x2 = x * x, y2 = y * y;
    b[0] = y2 * y; b[1] = R(3) * x * y2; b[2] = R(3) * x2 * y; b[3] = x2 * x;
  }
}

template <typename R> __device__ __forceinline__ const R* brk_ptr(const DevVolume& V);
template <> __device__ __forceinline__ const float* brk_ptr<float>(const DevVolume& V) { return V.brk32; }
template <> __device__ __forceinline__ const double* brk_ptr<double>(const DevVolume& V) { return V.brk64; }

// Segment s with brk[s] <= x < brk[s+1] (x clamped to [0,1]); local coordinate
// and the chain-rule factor 1/(brk[s+1]-brk[s]).
template <typename R>
__device__ __forceinline__ int locate(const R* __restrict__ brk, int nseg, R x, R& loc, R& scale) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(brk + mid) <= x) lo = mid; else hi = mid - 1;
  }
  const R b0 = __ldg(brk + lo), b1 = __ldg(brk + lo + 1);
  scale = R(1) / (b1 - b0);
  loc = (x - b0) * scale;
  loc = loc < R(0) ? R(0) : (loc > R(1) ? R(1) : loc);
  return lo;
}

template <typename R> struct ElemPtr;
template <> struct ElemPtr<float> {
  static __device__ __forceinline__ float4 ld(const DevVolume& V, size_t i) { return __ldg(V.elem32 + i); }
  static __device__ __forceinline__ float4 org(const DevVolume& V, size_t e) { return __ldg(V.org32 + e); }
};
template <> struct ElemPtr<double> {
  static __device__ __forceinline__ Dbl4 ld(const DevVolume& V, size_t i) {
    const double2* p = reinterpret_cast<const double2*>(V.elem64 + i);
    const double2 a = __ldg(p), b = __ldg(p + 1);
    Dbl4 r;
    r.x = a.x; r.y = a.y; r.z = b.x; r.w = b.y;
    return r;
  }
  static __device__ __forceinline__ Dbl4 org(const DevVolume& V, size_t e) { return ld2(V.org64 + e); }
  static __device__ __forceinline__ Dbl4 ld2(const Dbl4* q) {
    const double2* p = reinterpret_cast<const double2*>(q);
    const double2 a = __ldg(p), b = __ldg(p + 1);
    Dbl4 r;
    r.x = a.x; r.y = a.y; r.z = b.x; r.w = b.y;
    return r;
  }
};

// One row of N control points (fixed i, j) of a cubic element.  For N = 4
// the row is two 256-bit loads: every element starts at a multiple of 64
// control points in an allocation aligned to 256 bytes, so rows and their
// halves are 32-byte aligned.
__device__ __forceinline__ void ldg_cp2(const float4* p, float4& a, float4& b) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
      : "l"(p));
}
template <int N>
__device__ __forceinline__ void ldg_row(const float4* __restrict__ p, float4 c[N]) {
  if constexpr (N == 4) {
    ldg_cp2(p, c[0], c[1]);
    ldg_cp2(p + 2, c[2], c[3]);
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) c[k] = __ldg(p + k);
  }
}

// a[i] for an index the compiler keeps at run time (the outer loop of the
// contractions is not unrolled): a select chain on registers, so the basis
// arrays stay in registers instead of a local-memory stack copy.
template <int N>
__device__ __forceinline__ float pick(const float a[N], int i) {
  float v = a[0];
#pragma unroll
  for (int k = 1; k < N; ++k) v = (i == k) ? a[k] : v;
  return v;
}

// The paired contractions of eval_block (defined below); UI unrolls their
// outer (u) loop, chosen per kernel by measurement.
template <int P, bool WANT_RHO, int UI = 1>
__device__ __forceinline__ void contract_f32x2(const float4* __restrict__ cp, const float bu[P + 1],
                                               const float dbu[P + 1], const float bv[P + 1],
                                               const float dbv[P + 1], const float bw[P + 1],
                                               const float dbw[P + 1], float f[3], float fu[3], float fv[3],
                                               float fw[3], float& rho);
template <int P, int UI = 1>
__device__ __forceinline__ void contract_f32x2_xyz(const float4* __restrict__ cp, const float bu[P + 1],
                                                   const float dbu[P + 1], const float bv[P + 1],
                                                   const float dbv[P + 1], const float bw[P + 1],
                                                   const float dbw[P + 1], float f[3], float fu[3], float fv[3],
                                                   float fw[3]);

// phi, J (J[r][c] = d phi_r / d p_c) and optionally the scalar control-point
// field at parameter point p of block `blk`.  Sum-factorised: for each i the
// (j,k) slab is contracted along w (value and w-derivative), then along v,
// then the u contraction accumulates -- 576 FMA for P = 3.
// XYZ selects the contraction without the scalar channel (fewer paired
// multiply-adds, same results; it pays where the kernel has the registers for
// it: the shading pass and the single-frame trace kernel of cubic volumes).
template <int P, typename R, bool WANT_RHO, bool XYZ = false, int UI = 1>
__device__ __forceinline__ void eval_block(const DevVolume& V, const BlockInfo& B, const R p[3], R phi[3],
                                           R J[3][3], R& rho) {
  constexpr int N = P + 1;
  R loc[3], sc[3];
  int e[3];
  const R* brk = brk_ptr<R>(V);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    R x = p[d];
    x = x < R(0) ? R(0) : (x > R(1) ? R(1) : x);
    if ((B.uniform >> d) & 1) {            // uniform knots: O(1) element lookup
      const R xs = x * R(B.nseg[d]);
      int k = (int)xs;
      k = k < B.nseg[d] - 1 ? k : B.nseg[d] - 1;
      e[d] = k;
      loc[d] = xs - R(k);
      sc[d] = R(B.nseg[d]);
    } else {
      e[d] = locate<R>(brk + B.brk_off[d], B.nseg[d], x, loc[d], sc[d]);
    }
  }
  const size_t eid = (size_t)(B.elem_off + (e[2] * B.nseg[1] + e[1]) * B.nseg[0] + e[0]);
  const size_t base = eid * (N * N * N);
  R bu[N], dbu[N], bv[N], dbv[N], bw[N], dbw[N];
  bernstein<P, R>(loc[0], bu, dbu);
  bernstein<P, R>(loc[1], bv, dbv);
  bernstein<P, R>(loc[2], bw, dbw);
  R f[3] = {0, 0, 0}, fu[3] = {0, 0, 0}, fv[3] = {0, 0, 0}, fw[3] = {0, 0, 0};
  R s = 0;
  if constexpr (sizeof(R) == 4) {
    if constexpr (XYZ && !WANT_RHO)
      contract_f32x2_xyz<P, UI>(V.elem32 + base, bu, dbu, bv, dbv, bw, dbw, f, fu, fv, fw);
    else
      contract_f32x2<P, WANT_RHO, UI>(V.elem32 + base, bu, dbu, bv, dbv, bw, dbw, f, fu, fv, fw, s);
  } else {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    R s00[3] = {0, 0, 0}, s01[3] = {0, 0, 0}, s10[3] = {0, 0, 0};
    R ss = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      R t0[3] = {0, 0, 0}, t1[3] = {0, 0, 0};
      R ts = 0;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const typename Vec4T<R>::type c = ElemPtr<R>::ld(V, base + (i * N + j) * N + k);
        t0[0] += bw[k] * c.x; t0[1] += bw[k] * c.y; t0[2] += bw[k] * c.z;
        t1[0] += dbw[k] * c.x; t1[1] += dbw[k] * c.y; t1[2] += dbw[k] * c.z;
        if (WANT_RHO) ts += bw[k] * c.w;
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        s00[r] += bv[j] * t0[r];
        s01[r] += dbv[j] * t0[r];
        s10[r] += bv[j] * t1[r];
      }
      if (WANT_RHO) ss += bv[j] * ts;
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      f[r] += bu[i] * s00[r];
      fu[r] += dbu[i] * s00[r];
      fv[r] += bu[i] * s01[r];
      fw[r] += bu[i] * s10[r];
    }
    if (WANT_RHO) s += bu[i] * ss;
  }
  }
  const typename Vec4T<R>::type og = ElemPtr<R>::org(V, eid);
  f[0] += R(og.x);
  f[1] += R(og.y);
  f[2] += R(og.z);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    phi[r] = f[r];
    J[r][0] = fu[r] * sc[0];
    J[r][1] = fv[r] * sc[1];
    J[r][2] = fw[r] * sc[2];
  }
  rho = s;
}

// FP32 form of the contraction above on paired lanes (__ffma2_rn: two fused
// multiply-adds per instruction): (x, y) and (z, rho) of each control point
// travel together through the w, v and u contractions; the second lane of the
// (z, rho) pair of a derivative is not needed and costs nothing.
template <int P, bool WANT_RHO, int UI>
__device__ __forceinline__ void contract_f32x2(const float4* __restrict__ cp, const float bu[P + 1],
                                               const float dbu[P + 1], const float bv[P + 1],
                                               const float dbv[P + 1], const float bw[P + 1],
                                               const float dbw[P + 1], float f[3], float fu[3], float fv[3],
                                               float fw[3], float& rho) {
  constexpr int N = P + 1;
  const float2 z2 = make_float2(0.f, 0.f);
  float2 fxy = z2, fzr = z2, fuxy = z2, fuzr = z2, fvxy = z2, fvzr = z2, fwxy = z2, fwzr = z2;
#pragma unroll UI
  for (int i = 0; i < N; ++i) {
    float2 s00xy = z2, s00zr = z2, s01xy = z2, s01zr = z2, s10xy = z2, s10zr = z2;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float2 t0xy = z2, t0zr = z2, t1xy = z2, t1zr = z2;
      float4 row[N];
      ldg_row<N>(cp + (i * N + j) * N, row);
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const float4 c = row[k];
        const float2 cxy = make_float2(c.x, c.y), czr = make_float2(c.z, c.w);
        const float2 b = make_float2(bw[k], bw[k]), db = make_float2(dbw[k], dbw[k]);
        t0xy = __ffma2_rn(b, cxy, t0xy);
        t0zr = __ffma2_rn(b, czr, t0zr);
        t1xy = __ffma2_rn(db, cxy, t1xy);
        t1zr = __ffma2_rn(db, czr, t1zr);
      }
      const float2 b = make_float2(bv[j], bv[j]), db = make_float2(dbv[j], dbv[j]);
      s00xy = __ffma2_rn(b, t0xy, s00xy);
      s00zr = __ffma2_rn(b, t0zr, s00zr);
      s01xy = __ffma2_rn(db, t0xy, s01xy);
      s01zr = __ffma2_rn(db, t0zr, s01zr);
      s10xy = __ffma2_rn(b, t1xy, s10xy);
      s10zr = __ffma2_rn(b, t1zr, s10zr);
    }
    const float bui = pick<N>(bu, i), dbui = pick<N>(dbu, i);
    const float2 b = make_float2(bui, bui), db = make_float2(dbui, dbui);
    fxy = __ffma2_rn(b, s00xy, fxy);
    fzr = __ffma2_rn(b, s00zr, fzr);
    fuxy = __ffma2_rn(db, s00xy, fuxy);
    fuzr = __ffma2_rn(db, s00zr, fuzr);
    fvxy = __ffma2_rn(b, s01xy, fvxy);
    fvzr = __ffma2_rn(b, s01zr, fvzr);
    fwxy = __ffma2_rn(b, s10xy, fwxy);
    fwzr = __ffma2_rn(b, s10zr, fwzr);
  }
  f[0] = fxy.x; f[1] = fxy.y; f[2] = fzr.x;
  fu[0] = fuxy.x; fu[1] = fuxy.y; fu[2] = fuzr.x;
  fv[0] = fvxy.x; fv[1] = fvxy.y; fv[2] = fvzr.x;
  fw[0] = fwxy.x; fw[1] = fwxy.y; fw[2] = fwzr.x;
  rho = fzr.y;
}

// The same contraction without the scalar channel: the pairs are (x, y) of
// the value and of each derivative, and the z channel travels paired with
// itself under two different weights ((b, db) or (b_u, b_u) on two partial
// sums).  Every output is the same chain of fused multiply-adds in the same
// order as above, so phi and J agree bit for bit; the w contraction of a
// cubic point takes 192 paired multiply-adds instead of 256.
template <int P, int UI>
__device__ __forceinline__ void contract_f32x2_xyz(const float4* __restrict__ cp, const float bu[P + 1],
                                                   const float dbu[P + 1], const float bv[P + 1],
                                                   const float dbv[P + 1], const float bw[P + 1],
                                                   const float dbw[P + 1], float f[3], float fu[3], float fv[3],
                                                   float fw[3]) {
  constexpr int N = P + 1;
  const float2 z2 = make_float2(0.f, 0.f);
  // (f, fu).z and (fv, fw).z share pairs
  float2 fxy = z2, fuxy = z2, fvxy = z2, fwxy = z2, f_fu_z = z2, fv_fw_z = z2;
#pragma unroll UI
  for (int i = 0; i < N; ++i) {
    float2 s00xy = z2, s01xy = z2, s10xy = z2, s00_s01_z = z2;
    float s10z = 0.f;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float2 t0xy = z2, t1xy = z2, t01z = z2;   // t01z = (t0.z, t1.z)
      float4 row[N];
      ldg_row<N>(cp + (i * N + j) * N, row);
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const float4 c = row[k];
        const float2 cxy = make_float2(c.x, c.y), czz = make_float2(c.z, c.z);
        t0xy = __ffma2_rn(make_float2(bw[k], bw[k]), cxy, t0xy);
        t1xy = __ffma2_rn(make_float2(dbw[k], dbw[k]), cxy, t1xy);
        t01z = __ffma2_rn(make_float2(bw[k], dbw[k]), czz, t01z);
      }
      const float2 b = make_float2(bv[j], bv[j]), db = make_float2(dbv[j], dbv[j]);
      s00xy = __ffma2_rn(b, t0xy, s00xy);
      s01xy = __ffma2_rn(db, t0xy, s01xy);
      s10xy = __ffma2_rn(b, t1xy, s10xy);
      s00_s01_z = __ffma2_rn(make_float2(bv[j], dbv[j]), make_float2(t01z.x, t01z.x), s00_s01_z);
      s10z = __fmaf_rn(bv[j], t01z.y, s10z);
    }
    const float bui = pick<N>(bu, i), dbui = pick<N>(dbu, i);
    const float2 b = make_float2(bui, bui), db = make_float2(dbui, dbui);
    fxy = __ffma2_rn(b, s00xy, fxy);
    fuxy = __ffma2_rn(db, s00xy, fuxy);
    fvxy = __ffma2_rn(b, s01xy, fvxy);
    fwxy = __ffma2_rn(b, s10xy, fwxy);
    f_fu_z = __ffma2_rn(make_float2(bui, dbui), make_float2(s00_s01_z.x, s00_s01_z.x), f_fu_z);
    fv_fw_z = __ffma2_rn(b, make_float2(s00_s01_z.y, s10z), fv_fw_z);
  }
  f[0] = fxy.x; f[1] = fxy.y; f[2] = f_fu_z.x;
  fu[0] = fuxy.x; fu[1] = fuxy.y; fu[2] = f_fu_z.y;
  fv[0] = fvxy.x; fv[1] = fvxy.y; fv[2] = fv_fw_z.x;
  fw[0] = fwxy.x; fw[1] = fwxy.y; fw[2] = fv_fw_z.y;
}

template <typename R>
__device__ __forceinline__ R det3(const R J[3][3]) {
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

// Solve J x = b by the adjugate (Cramer); returns det J.
template <typename R>
__device__ __forceinline__ R solve3(const R J[3][3], const R b[3], R x[3]) {
  const R c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  const R c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  const R c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  const R det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  const R inv = R(1) / det;
  const R c10 = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  const R c11 = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  const R c12 = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  const R c20 = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  const R c21 = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  const R c22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  x[0] = (c00 * b[0] + c10 * b[1] + c20 * b[2]) * inv;
  x[1] = (c01 * b[0] + c11 * b[1] + c21 * b[2]) * inv;
  x[2] = (c02 * b[0] + c12 * b[1] + c22 * b[2]) * inv;
  return det;
}

// J_u(p) of the displacement field (IVV_SCALAR_VONMISES): the geometry's
// element lookup and contraction, run on the displacement elements.
template <int P, typename R>
__device__ __forceinline__ void eval_disp_jac(const DevVolume& V, const BlockInfo& B, const R p[3], R Ju[3][3]) {
  DevVolume U = V;
  U.elem32 = V.disp32;
  U.org32 = V.dorg32;
  U.elem64 = V.disp64;
  U.org64 = V.dorg64;
  R u[3], unused;
  eval_block<P, R, false, true>(U, B, p, u, Ju, unused);
}

// The scalar rho at parameter point p for the volume's mode, from
// J = J_phi(p) and the control-point scalar rc there: rc (IVV_SCALAR_CP),
// det J, Eq. 23's det J / ||J||_F, or the von Mises value of §6.2.
template <int P, typename R>
__device__ __forceinline__ R scalar_at(const DevVolume& V, const BlockInfo& B, int mode, const R p[3],
                                       const R J[3][3], R rc) {
  if (mode == IVV_SCALAR_CP) return rc;
  if (mode == IVV_SCALAR_VONMISES) {
    R Ju[3][3];
    eval_disp_jac<P, R>(V, B, p, Ju);
    return von_mises<R>(J, Ju);
  }
  const R det = det3<R>(J);
  if (mode == IVV_SCALAR_DETJ) return det;
  R f = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) f += J[a][b] * J[a][b];
  return det / sqrt(f);
}

// Piecewise-linear TF (knots in shared memory): colour and extinction weight.
// seg[i] (kTfTable entries) is the last segment starting at or below
// i / kTfTable, so the segment of x is found from seg[floor(x kTfTable)] by a
// short forward scan.
constexpr int kTfTable = 256;

__device__ __forceinline__ float4 tf_eval(const float* __restrict__ r, const float4* __restrict__ rgba,
                                          const unsigned char* __restrict__ seg, int n, float x) {
  if (x <= r[0]) return rgba[0];
  if (x >= r[n - 1]) return rgba[n - 1];
  int c = (int)(x * (float)kTfTable);
  c = c < kTfTable - 1 ? c : kTfTable - 1;
  int lo = seg[c];                     // segment i with r[i] <= x < r[i+1]
  while (lo < n - 2 && r[lo + 1] <= x) ++lo;
  const float w = r[lo + 1] - r[lo];
  const float t = w > 0.f ? (x - r[lo]) / w : 1.f;
  const float4 a = rgba[lo], b = rgba[lo + 1];
  return make_float4(a.x + t * (b.x - a.x), a.y + t * (b.y - a.y), a.z + t * (b.z - a.z), a.w + t * (b.w - a.w));
}

// ------------------------------------------------------------- batches
// One request of a batch.  The batch's pixels are numbered request after
// request: request rq owns pixels pix0[rq] .. pix0[rq+1]-1 (row-major within
// its image); its K2a warp tiles (of the tuned shape) are tile0[rq] ..
// tile0[rq+1]-1, row-major over the image; its volume's faces are face0 ..
// face0 + n_faces - 1 of the batch's pool, their screen boxes for this camera
// start at box0 and their group boxes at gbox0.
struct DevRequest {
  DevCamera<float> cam;
  DevCamera<double> cam64;
  int face0, n_faces, box0, gbox0;
  float diag;          // control-point bbox diagonal of the volume
  float ds;            // sample distance
  float4* out;         // caller-owned RGBA image
};

// The request's transfer function; seg as in tf_eval.
constexpr int kBatchTfMax = IVV_BATCH_TF_MAX;
struct DevTFSlot {
  float r[kBatchTfMax];
  float4 rgba[kBatchTfMax];
  unsigned char seg[kTfTable];
  int n;
  float sigma, lo, inv_range;
};

struct BatchArgs {
  const DevRequest* req;   // [nreq]
  const int* pix0;         // [nreq + 1] first pixel of each request, then the total
  const int* tile0;        // [nreq + 1] first K2 tile of each request, then the total
  const int* tile16;       // [nreq + 1] the same for 16x16 tiles (K4's pixel order)
  const DevTFSlot* tf;     // [nreq]
  int nreq;
};

// The request rq with first[rq] <= x < first[rq + 1] (first ascending).
__device__ __forceinline__ int batch_find(const int* __restrict__ first, int nreq, int x) {
  int lo = 0, hi = nreq - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(first + mid) <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int batch_request(const BatchArgs& ba, int pix) { return batch_find(ba.pix0, ba.nreq, pix); }

// As tf_eval for an unclamped normalised scalar x, also returning the piece
// of the TF that x falls in: -1 for x <= r[0] and n-1 for x >= r[n-1] (the
// constant ends), otherwise the segment i with r[i] <= x < r[i+1].
__device__ __forceinline__ float4 tf_eval_seg(const float* __restrict__ r, const float4* __restrict__ rgba,
                                              const unsigned char* __restrict__ seg, int n, float x, int& piece) {
  if (x <= r[0]) {
    piece = -1;
    return rgba[0];
  }
  if (x >= r[n - 1]) {
    piece = n - 1;
    return rgba[n - 1];
  }
  int c = (int)(x * (float)kTfTable);
  c = c < kTfTable - 1 ? c : kTfTable - 1;
  int lo = seg[c];
  while (lo < n - 2 && r[lo + 1] <= x) ++lo;
  piece = lo;
  const float w = r[lo + 1] - r[lo];
  const float t = w > 0.f ? __fdividef(x - r[lo], w) : 1.f;
  const float4 a = rgba[lo], b = rgba[lo + 1];
  return make_float4(a.x + t * (b.x - a.x), a.y + t * (b.y - a.y), a.z + t * (b.z - a.z), a.w + t * (b.w - a.w));
}

// Counters block of a render: [0] active pixels, [2] sample total, [3]
// spare, [4] stage-1 items, [5] their hand-out head, [6] deferred items, [7]
// their hand-out head, [8] and [9] the batch's overflow list and its queue
// head, [10] the shading pass's queue head, [11] the learned-guess list of
// stage 2, [12] the FP64 polish list of stage 1; the integrator's queue head
// at kQueueHeadOff.
constexpr int kQueueHeadOff = 1;
constexpr int kItemCounter = 4;
constexpr int kItemHead = 5;         // next stage-1 item to hand out (K2b)
constexpr int kSlowCounter = 6;      // items deferred to the subdivision search
constexpr int kSlowHead = 7;         // next deferred item to hand out (K2c)
constexpr int kOverflowCounter = 8;  // batch: pixels beyond the sample buffer
constexpr int kOverflowHead = 9;     // batch: the fused integrator's queue head over them
constexpr int kShadeHead = 10;       // the shading pass's queue head (split integration)
constexpr int kCountersBytes = 256;

__device__ __forceinline__ void atomic_max_nonneg_float(unsigned int* addr, float v) {
  if (v > 0.f) atomicMax(addr, __float_as_uint(v));
}

// ------------------------------------------------------------- launchers
struct Workspace;   // see ivv_api.cu

// Stage-1 buffers of a render: face screen boxes [F], group boxes [ceil(F/32)],
// the (pixel, patch) item list (cap entries, count at *n_items) and the
// A-buffer (frag_tp / frag_meta slot-major, frag_count per pixel).
constexpr int kItemsPerPixel = 16;   // capacity of the (pixel, patch) list per pixel
constexpr int kBatchFaceBits = 20;   // batch items: request << 20 | pool patch
constexpr int kGroup = 32;           // patches per group box
struct SurfaceWs {
  int4* boxes;
  int4* gboxes;
  int2* items;
  int* slow;          // [cap] items deferred to the subdivision search
  int cap;
  int* n_items;
  void* frag_tp;
  unsigned* frag_meta;
  int* frag_count;
  // single frames: a flag per 16 x 16 tile, set where a warp tile has
  // candidate patches (K4 processes flagged tiles only and clears their
  // flags); the warp tiles without candidates get pair_count 0 and, if
  // zero_out is set, a zero pixel from the cull.  Null: no tile skipping.
  int* tile_flag = nullptr;
  int* pair_count = nullptr;
  float4* zero_out = nullptr;
};

void launch_face_project(const DevVolume& V, const DevCamera<float>& cam, int4* boxes, int4* gboxes, cudaStream_t s);

template <typename R>
void launch_intersect(const DevVolume& V, const DevCamera<R>& cam, const DevCamera<double>& cam64, bool mixed,
                      bool stats, const SurfaceWs& w, DevStats* st, int num_sms, cudaStream_t s);
constexpr int kPolishCounter = 12;   // counters slot: grazing hits listed for the FP64 polish pass

// Cutting and near-clip planes (§5.5) applied by K4 to the depth-sorted
// intersections of each pixel.  Ends that move onto a plane are flagged in
// pair_block (kSolveIn / kSolveOut, with the chord guess in the pair record)
// and solved by the clip fix-up kernel before stage 3.
constexpr int kMaxCutPlanes = IVV_MAX_CUT_PLANES;
// kGuessIn marks an entry without chord context (an entry on the near plane
// or a moved singular entry), whose Newton may start from the learned guess;
// kShrunk an entry moved by §5.4's singular-entry rule.
constexpr int kSolveIn = 1 << 30, kSolveOut = 1 << 29, kGuessIn = 1 << 28, kShrunk = 1 << 27,
              kBlockMask = (1 << 27) - 1;
constexpr int kGuessCounter = 11;    // counters slot: entries in the learned-guess list
template <typename R>
struct ClipArgs {
  int on;                       // any plane active
  R near;                       // > 0: near plane distance along f
  R f[3];                       // view direction
  int n_cut;
  R cut[kMaxCutPlanes][4];      // (n, w): n.g + w > 0 is cut away
  DevCamera<R> cam;             // the pixels' rays
};

// Learned initial guesses of the fix-up solves: entries flagged kGuessIn are
// listed (world point, block) for the guess network; guess_p receives its
// parameter guesses, gidx [kMaxPairs][npix] the list index of each slot.
struct GuessList {
  float4* g;        // [n] world points (x, y, z, 0)
  int* blk;         // [n] blocks
  float4* p;        // [n] parameter guesses
  int* gidx;        // [kMaxPairs][npix]
  int* n;           // list length (device counter)
};

template <typename R>
void launch_clip_solve(const DevVolume& V, const DevCamera<R>& cam, int npix, typename Vec4T<R>::type* pair_in,
                       typename Vec4T<R>::type* pair_out, int* pair_block, const int* pair_count, const int* active,
                       const int* n_active, bool mixed, const GuessList* guess, DevStats* st, int num_sms,
                       cudaStream_t s);

// Lists the entries that take the learned guess (kGuessIn), first moving the
// singular entries of flagged blocks (§5.4) when `singular` is set.
template <typename R>
void launch_guess_mark(const DevVolume& V, const DevCamera<R>& cam, int npix, typename Vec4T<R>::type* pair_in,
                       typename Vec4T<R>::type* pair_out, int* pair_block, const int* pair_count, const int* active,
                       const int* n_active, bool singular, bool mixed, const GuessList& guess, DevStats* st,
                       int num_sms, cudaStream_t s);

// §5.4 (Eq. 22): entries with a singular Jacobian, in blocks with a flagged
// face, move along the ray and get a new parameter point (k_pair.cu).
template <typename R>
void launch_entry_fix(const DevVolume& V, const DevCamera<R>& cam, int npix, typename Vec4T<R>::type* pair_in,
                      typename Vec4T<R>::type* pair_out, const int* pair_block, const int* pair_count,
                      const int* active, const int* n_active, bool mixed, DevStats* st, int num_sms, cudaStream_t s);

// Samples of a pair of length L > 0 at spacing ds: s_j = j ds for j = 0 ..
// floor(L / ds), plus the exit s = L when the remainder exceeds tail_eps --
// the rule every integrator and the sample lists follow.
__device__ __forceinline__ int pair_sample_count(float L, float ds, float tail_eps) {
  const float fl = floorf(L / ds);
  return (int)fl + ((L - fl * ds > tail_eps) ? 1 : 0) + 1;
}

// Sample lists counted by K4 itself (frames without stage-2 fix-ups): each
// 16 x 16 tile claims one run of the list for its active pixels, in the
// order of their queue items; off / cnt [active items], total[0] the running
// total, total[1] set when it passed INT_MAX.  off == nullptr: not counted.
struct SampleCount {
  float ds, tail_eps;
  int* off;
  int* cnt;
  int* total;
};

template <typename R>
void launch_pair(const DevVolume& V, int w, int npix, float diag, const typename Vec4T<R>::type* frag_tp,
                 const unsigned* frag_meta, const int* frag_count, typename Vec4T<R>::type* pair_in,
                 typename Vec4T<R>::type* pair_out, int* pair_block, int* pair_count, int max_pairs,
                 int* active, int* n_active, float4* out_rgba_zero, const ClipArgs<R>& clip, int* tile_flag,
                 DevStats* st, cudaStream_t s, const SampleCount* count = nullptr);

struct IntegrateArgs {
  float rk_tol, ds, c, early_alpha;
  int K;
  int max_steps;
  int max_step_samples;   // longest RK step, in sample distances
  int npix;
};

template <typename R>
void launch_integrate(const DevVolume& V, const DevCamera<R>& cam, const DevTF& tf, const IntegrateArgs& a,
                      bool mixed, bool stats, const typename Vec4T<R>::type* pair_in,
                      const typename Vec4T<R>::type* pair_out, const int* pair_block, const int* pair_count,
                      const int* active, const int* n_active, int* queue_head, float4* out_rgba, DevStats* st,
                      int num_sms, cudaStream_t s);

void launch_batch_pair(const BatchArgs& ba, int tiles16, int npix, const float4* frag_tp, const unsigned* frag_meta,
                       const int* frag_count, float4* pair_in, float4* pair_out, int* pair_block, int* pair_count,
                       int* active, int* n_active, DevStats* st, cudaStream_t s);
void launch_batch_face_project(const DevVolume& V, const BatchArgs& ba, int max_faces, const SurfaceWs& w,
                               cudaStream_t s);
// K2a warp tile tile_w x tile_h in {8x4, 4x8, 16x2}; tiles = the batch's
// count of such tiles (ba.tile0 holds their prefix); returns false for
// another shape.
bool launch_batch_intersect(const DevVolume& V, const BatchArgs& ba, int tiles, int tile_w, int tile_h, bool mixed,
                            bool stats, const SurfaceWs& w, size_t stride, DevStats* st, int num_sms,
                            cudaStream_t s);
void launch_batch_integrate(const DevVolume& V, const BatchArgs& ba, const IntegrateArgs& a, bool mixed, bool stats,
                            const float4* pin, const float4* pout, const int* pblk, const int* pcnt,
                            const int* active, const int* n_active, int* queue_head, DevStats* st, int grid,
                            cudaStream_t s);
int batch_integrate_max_ctas_per_sm(int P, bool mixed, bool stats);
// Split stage 3 of a batch (k_integrate_batch.cu): counts into cnt, their
// scan into off (sums: scan scratch), trace and shading into the sample
// buffer sp of cap samples, the fused integrator over the pixels that do not
// fit (list: npix ints of scratch).  counters: the render's counters block.
void launch_batch_count(const BatchArgs& ba, const float4* pin, const float4* pout, const int* pcnt, const int* active,
                        const int* n_active, int npix, int* cnt, int num_sms, cudaStream_t s);
void launch_batch_split(const DevVolume& V, const BatchArgs& ba, const IntegrateArgs& a, bool mixed, bool stats,
                        const float4* pin, const float4* pout, const int* pblk, const int* pcnt, const int* active,
                        int* counters, int* off, int* cnt, int* sums, float4* sp, int cap, int* list, int grid,
                        int num_sms, DevStats* st, cudaStream_t s);

// Explicit Runge-Kutta tableau of the fixed-step integrators, at most
// kRkStagesMax stages (a strictly lower triangular).
constexpr int kRkStagesMax = 6;
struct RkTableau {
  int s;
  float a[kRkStagesMax][kRkStagesMax];
  float b[kRkStagesMax];
};

template <int P>
void launch_fixed_p(const DevVolume& V, const DevCamera<float>& cam, const DevTF& tf, const IntegrateArgs& a,
                    const RkTableau& T, bool mixed, bool stats, const float4* pin, const float4* pout,
                    const int* pblk, const int* pcnt, const int* active, const int* n_active, int* queue_head,
                    float4* out, DevStats* st, int num_sms, cudaStream_t s);
// Implicit Euler (k_irk1.cuh).
template <int P>
void launch_irk1_p(const DevVolume& V, const DevCamera<float>& cam, const DevTF& tf, const IntegrateArgs& a,
                   bool mixed, bool stats, const float4* pin, const float4* pout, const int* pblk, const int* pcnt,
                   const int* active, const int* n_active, int* queue_head, float4* out, DevStats* st, int num_sms,
                   cudaStream_t s);

void launch_eval_points(const DevVolume& V, int block, int n, const float* p, float* phi, float* jac,
                        float* rho, cudaStream_t s);

void launch_fill_center(float4* p, int n, cudaStream_t s);
void launch_rf_count(const float4* pin, const float4* pout, const int* pblk, const int* pcnt, const int* active,
                     const int* n_active, int npix, float ds, float tail_eps, int* cnt, int num_sms, cudaStream_t s);
void launch_rf_scan(const int* cnt, const int* n_active, int npix, int* off, int* sums, int cap, int* total,
                    cudaStream_t s);
void launch_rf_expand(const DevCamera<float>& cam, const float4* pin, const float4* pout, const int* pblk,
                      const int* pcnt, const int* active, const int* n_active, const int* off, int npix, float ds,
                      float tail_eps, int guess, int cap, float4* sg, int* sblk, float4* sp, int num_sms,
                      cudaStream_t s);
// perm (optional): the order in which the samples are solved.
void launch_rf_newton(const DevVolume& V, const DevCamera<float>& cam, float rf_tol, float abs_tol, const int* n_ptr,
                      const float4* sg, const int* sblk, const float4* sp, float* srho, float4* p_out, int* it_out,
                      DevStats* st, bool stats, bool mixed, int num_sms, cudaStream_t s, const int* perm = nullptr);
// key[i]: global index of the element holding sample i's start sp[i].
void launch_rf_elem_key(const DevVolume& V, const int* n_ptr, const int* sblk, const float4* sp, int* key, int num_sms,
                        cudaStream_t s);
void launch_rf_composite(const DevTF& tf, int K, float early, const float4* pin, const float4* pout, const int* pblk,
                         const int* pcnt, const int* active, const int* n_active, const int* off, int npix, float ds,
                         float tail_eps, int cap, const float* srho, float4* out, DevStats* st,
                         bool stats, int num_sms, cudaStream_t s);

// Split ODE integration (FP32 / MIXED, one frame): the trace kernel K5t
// writes every sample's parameter point (x, y, z, block as int bits) at its
// offset in the per-pixel sample list (rf_count / rf_scan); k_shade_composite
// evaluates the scalar at the samples and composites, one thread per pixel.
struct SplitArgs {
  const int* off;      // [active items] first sample of each pixel
  float4* sp;          // [cap] sample points
  int cap;
};
template <int P>
void launch_integrate_split_p(const DevVolume& V, const DevCamera<float>& cam, const IntegrateArgs& a,
                              const SplitArgs& sa, bool mixed, bool stats, const float4* pin, const float4* pout,
                              const int* pblk, const int* pcnt, const int* active, const int* n_active,
                              int* queue_head, DevStats* st, int num_sms, cudaStream_t s);
template <int P>
void launch_shade_composite_p(const DevVolume& V, const DevCamera<float>& cam, const DevTF& tf, int K, float early,
                              const float4* pin, const float4* pout, const int* pblk, const int* pcnt,
                              const int* active, const int* n_active, int* queue_head, const int* off, int npix,
                              float ds, float tail_eps, const SplitArgs& sa, float4* out, bool stats, DevStats* st,
                              int num_sms, cudaStream_t s);

}  // namespace ivv
