// Stage 2 (§4.2): per-pixel depth sorting of the fragment list and blockwise
// entry/exit pairing (Alg. 2).
//   K4 pair -- one thread per pixel: load the pixel's fragment slots (the
//              A-buffer written by K2), insertion-sort them by
//              (depth, block, facing), merge duplicates of one block with equal
//              facing (hits on edges shared by two patches or two faces), then
//              repeatedly take the nearest unused back-facing record and the
//              nearest unused front-facing record of the same block (Alg. 2).
//              Pairs are written in that order, which is front to back for
//              non-overlapping blocks.  Pixels with pairs are appended to the
//              work queue of the integrator; the others get a zero pixel.
#include <cuda_runtime.h>

#include "ivv_device.cuh"

namespace ivv {

namespace {

// Sorting and pairing of the fragments of pixel `pix` (slot index
// slot * stride + pix); returns the number of pairs written.  A pixel
// without pairs gets a zero RGBA in *zero_out (if not NULL).
template <typename R>
__device__ __forceinline__ int pair_pixel(size_t pix, size_t stride, R tau_dup,
                                          const typename Vec4T<R>::type* __restrict__ frag_tp,
                                          const unsigned* __restrict__ frag_meta, const int* __restrict__ frag_count,
                                          typename Vec4T<R>::type* __restrict__ pair_in,
                                          typename Vec4T<R>::type* __restrict__ pair_out, int* __restrict__ pair_block,
                                          int* __restrict__ pair_count, int max_pairs, float4* zero_out,
                                          unsigned& um, unsigned& pov) {
  typedef typename Vec4T<R>::type V4;
  int n = frag_count[pix];
  n = n < kMaxFrags ? n : kMaxFrags;
  R t[kMaxFrags], pp[kMaxFrags][3];
  unsigned m[kMaxFrags];
  for (int i = 0; i < n; ++i) {
    const V4 f = frag_tp[(size_t)i * stride + pix];
    t[i] = f.x;
    pp[i][0] = f.y;
    pp[i][1] = f.z;
    pp[i][2] = f.w;
    m[i] = frag_meta[(size_t)i * stride + pix];
  }
  int in_idx[kMaxPairs], out_idx[kMaxPairs];
  const int np = pair_fragments<R>(n, t, m, pp, tau_dup, max_pairs, in_idx, out_idx, um, pov);
  for (int q = 0; q < np; ++q) {
    const size_t o = (size_t)q * stride + pix;
    pair_in[o] = frag_tp[(size_t)in_idx[q] * stride + pix];
    pair_out[o] = frag_tp[(size_t)out_idx[q] * stride + pix];
    pair_block[o] = (int)(m[in_idx[q]] >> 4);
  }
  pair_count[pix] = np;
  if (np == 0 && zero_out) *zero_out = make_float4(0.f, 0.f, 0.f, 0.f);
  return np;
}

// Warp-aggregated append of the active pixels to the integrator's queue and
// the counters that every render keeps.
__device__ __forceinline__ void pair_epilogue(int pix, int np, unsigned um, unsigned pov, int* __restrict__ active,
                                              int* __restrict__ n_active, DevStats* __restrict__ st) {
  const int lane = threadIdx.x & 31;
  const bool act = np > 0;
  const unsigned bal = __ballot_sync(0xffffffffu, act);
  int base = 0;
  if (lane == 0 && bal) base = atomicAdd(n_active, __popc(bal));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (act) active[base + __popc(bal & ((1u << lane) - 1u))] = pix;
  unsigned long long cu = um, cp = pov, cr = act ? 1 : 0, cpairs = np;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cu += __shfl_down_sync(0xffffffffu, cu, o);
    cp += __shfl_down_sync(0xffffffffu, cp, o);
    cr += __shfl_down_sync(0xffffffffu, cr, o);
    cpairs += __shfl_down_sync(0xffffffffu, cpairs, o);
  }
  if (lane == 0) {
    if (cu) atomicAdd(&st->unmatched, cu);
    if (cp) atomicAdd(&st->pair_overflow, cp);
    if (cr) atomicAdd(&st->rays, cr);
    if (cpairs) atomicAdd(&st->pairs, cpairs);
  }
}

// Pixel of thread threadIdx.x of 16x16 tile (tx, ty): warp w covers the 8x4
// block at (8 (w & 1), 4 (w >> 1)) of the tile.  Pixels are queued in this
// order, so the 32 lanes of an integrator warp start on a compact pixel block
// whose rays cross the same elements (shared control-point loads).
__device__ __forceinline__ void tile_pixel(int tx, int ty, int& x, int& y) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  x = tx * 16 + (warp & 1) * 8 + (lane & 7);
  y = ty * 16 + (warp >> 1) * 4 + (lane >> 3);
}

template <typename R>
__global__ void __launch_bounds__(256) k4_pair(int w, int npix, R tau_dup, const typename Vec4T<R>::type* __restrict__ frag_tp,
                                               const unsigned* __restrict__ frag_meta,
                                               const int* __restrict__ frag_count,
                                               typename Vec4T<R>::type* __restrict__ pair_in,
                                               typename Vec4T<R>::type* __restrict__ pair_out,
                                               int* __restrict__ pair_block, int* __restrict__ pair_count,
                                               int max_pairs, int* __restrict__ active, int* __restrict__ n_active,
                                               float4* __restrict__ out_rgba, DevStats* __restrict__ st) {
  const int tiles_x = (w + 15) / 16;
  int x, y;
  tile_pixel(blockIdx.x % tiles_x, blockIdx.x / tiles_x, x, y);
  const int pix = y * w + x;
  int np = 0;
  unsigned um = 0, pov = 0;
  if (x < w && pix < npix)
    np = pair_pixel<R>(pix, npix, tau_dup, frag_tp, frag_meta, frag_count, pair_in, pair_out, pair_block,
                       pair_count, max_pairs, out_rgba ? out_rgba + pix : nullptr, um, pov);
  pair_epilogue(pix, np, um, pov, active, n_active, st);
}

// Batched form: pixel `pix` of the batch's pixel space belongs to request
// rq with pix0[rq] <= pix < pix0[rq + 1]; its duplicate tolerance follows
// the request's volume and its empty-pixel zero goes to the request's image.
__global__ void __launch_bounds__(256) kb4_pair(BatchArgs ba, int npix, const float4* __restrict__ frag_tp,
                                                const unsigned* __restrict__ frag_meta,
                                                const int* __restrict__ frag_count, float4* __restrict__ pair_in,
                                                float4* __restrict__ pair_out, int* __restrict__ pair_block,
                                                int* __restrict__ pair_count, int* __restrict__ active,
                                                int* __restrict__ n_active, DevStats* __restrict__ st) {
  const int rq = batch_find(ba.tile16, ba.nreq, blockIdx.x);
  const DevRequest& q = ba.req[rq];
  const int t = blockIdx.x - __ldg(ba.tile16 + rq);
  const int tiles_x = (q.cam.w + 15) / 16;
  int x, y;
  tile_pixel(t % tiles_x, t / tiles_x, x, y);
  const int pix = __ldg(ba.pix0 + rq) + y * q.cam.w + x;
  int np = 0;
  unsigned um = 0, pov = 0;
  if (x < q.cam.w && y < q.cam.h) {
    const float tau = 1e-5f * q.diag;
    np = pair_pixel<float>(pix, npix, tau, frag_tp, frag_meta, frag_count, pair_in, pair_out, pair_block,
                           pair_count, kMaxPairs, q.out + (pix - __ldg(ba.pix0 + rq)), um, pov);
  }
  pair_epilogue(pix, np, um, pov, active, n_active, st);
}

}  // namespace

template <typename R>
void launch_pair(const DevVolume& V, int w, int npix, float diag, const typename Vec4T<R>::type* frag_tp,
                 const unsigned* frag_meta, const int* frag_count, typename Vec4T<R>::type* pair_in,
                 typename Vec4T<R>::type* pair_out, int* pair_block, int* pair_count, int max_pairs, int* active,
                 int* n_active, float4* out_rgba_zero, Dbl4* /*unused*/, DevStats* st, cudaStream_t s) {
  (void)V;
  if (npix <= 0) return;
  const R tau = sizeof(R) == 4 ? R(1e-5) * R(diag) : R(1e-9) * R(diag);
  if (w <= 0) return;
  const int h = npix / w;
  k4_pair<R><<<((w + 15) / 16) * ((h + 15) / 16), 256, 0, s>>>(w, npix, tau, frag_tp, frag_meta, frag_count, pair_in, pair_out,
                                                pair_block, pair_count, max_pairs, active, n_active, out_rgba_zero, st);
}

void launch_batch_pair(const BatchArgs& ba, int tiles16, int npix, const float4* frag_tp, const unsigned* frag_meta,
                       const int* frag_count, float4* pair_in, float4* pair_out, int* pair_block, int* pair_count,
                       int* active, int* n_active, DevStats* st, cudaStream_t s) {
  if (npix <= 0 || tiles16 <= 0) return;
  kb4_pair<<<tiles16, 256, 0, s>>>(ba, npix, frag_tp, frag_meta, frag_count, pair_in, pair_out,
                                             pair_block, pair_count, active, n_active, st);
}

template void launch_pair<float>(const DevVolume&, int, int, float, const float4*, const unsigned*, const int*, float4*,
                                 float4*, int*, int*, int, int*, int*, float4*, Dbl4*, DevStats*, cudaStream_t);
template void launch_pair<double>(const DevVolume&, int, int, float, const Dbl4*, const unsigned*, const int*,
                                  Dbl4*, Dbl4*, int*, int*, int, int*, int*, float4*, Dbl4*, DevStats*,
                                  cudaStream_t);

}  // namespace ivv

namespace ivv {
namespace {

__global__ void k_export_pairs(int npix, int max_pairs, const float4* __restrict__ pin, const float4* __restrict__ pout,
                               const int* __restrict__ pblk, const int* __restrict__ pcnt, int* __restrict__ out_count,
                               float* __restrict__ out_pairs, int* __restrict__ out_block) {
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  int n = pcnt[pix];
  n = n < max_pairs ? n : max_pairs;
  out_count[pix] = n;
  for (int q = 0; q < n; ++q) {
    const size_t s = (size_t)q * npix + pix;
    const float4 a = pin[s], b = pout[s];
    float* o = out_pairs + s * 8;
    o[0] = a.y; o[1] = a.z; o[2] = a.w; o[3] = a.x;
    o[4] = b.y; o[5] = b.z; o[6] = b.w; o[7] = b.x;
    out_block[s] = pblk[s];
  }
}

}  // namespace

void launch_export_pairs(int npix, int max_pairs, bool fp64, const void* pin, const void* pout, const int* pblk,
                         const int* pcnt, int* out_count, float* out_pairs, int* out_block, cudaStream_t s) {
  (void)fp64;
  if (npix <= 0) return;
  k_export_pairs<<<(npix + 255) / 256, 256, 0, s>>>(npix, max_pairs, (const float4*)pin, (const float4*)pout, pblk,
                                                    pcnt, out_count, out_pairs, out_block);
}

}  // namespace ivv
