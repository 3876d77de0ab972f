// Batched stage 1 (§4.1): one K0 launch over every (request, face patch), one
// K2a launch over every warp tile of every request and one K2b launch over
// the items of all requests.  A K2a warp finds its request from the batch's
// tile table and tags its items with it (high bits of the patch word); both
// then run the single-frame bodies (k_surface.cuh) on that request's camera,
// patches and slice of the batch's pixel space.
#include <cuda_runtime.h>

#include "k_surface.cuh"

namespace ivv {

namespace {

constexpr int kCullWarps = 8;
constexpr int kRootsThreads = 128;

template <int P>
__global__ void kb0_face_project(DevVolume V, BatchArgs ba, int4* __restrict__ boxes, int4* __restrict__ gboxes) {
  const DevRequest& q = ba.req[blockIdx.y];
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x * blockDim.x >= q.n_faces) return;    // whole CTA
  project_faces<P>(V, q.cam, f, q.n_faces, q.face0, q.diag, boxes + q.box0, gboxes + q.gbox0);
}

template <int TW, int TH>
__global__ void __launch_bounds__(32 * kCullWarps) kb2a_cull(DevVolume V, BatchArgs ba, int tiles,
                                                             const int4* __restrict__ boxes,
                                                             const int4* __restrict__ gboxes,
                                                             int2* __restrict__ items, int cap,
                                                             int* __restrict__ n_items, int* __restrict__ frag_count,
                                                             DevStats* __restrict__ st) {
  const int t = blockIdx.x * kCullWarps + (threadIdx.x >> 5);
  if (t >= tiles) return;                      // whole warps
  const int rq = batch_find(ba.tile0, ba.nreq, t);
  const DevRequest& q = ba.req[rq];
  const DevCamera<float> cam = q.cam;
  const int tiles_x = (cam.w + TW - 1) / TW;
  const int tl = t - __ldg(ba.tile0 + rq);
  cull_warp_tile<float, TW, TH>(V, cam, tl % tiles_x, tl / tiles_x, q.face0, q.n_faces, boxes + q.box0,
                                gboxes + q.gbox0, q.diag, __ldg(ba.pix0 + rq), rq << kBatchFaceBits, items, cap,
                                n_items, frag_count, st);
}

template <int P, bool MIXED, bool STATS>
__global__ void __launch_bounds__(kRootsThreads, 4) kb2b_roots(DevVolume V, BatchArgs ba,
                                                               const int2* __restrict__ items,
                                                               int* __restrict__ slow, int* __restrict__ n_items,
                                                               int cap, float4* __restrict__ frag_tp,
                                                               unsigned* __restrict__ frag_meta,
                                                               int* __restrict__ frag_count, size_t stride,
                                                               DevStats* __restrict__ st) {
  const int n = min(n_items[0], cap);
  unsigned long long c_tests = 0, c_fp64 = 0, c_frag = 0;
  int c_newton = 0;
  for (;;) {                                   // warps take 32 consecutive items at a time
    const int base = take_items(n_items, n);
    if (base >= n) break;
    const int i = base + (int)(threadIdx.x & 31);
    if (i >= n) continue;
    const int2 it = __ldg(items + i);
    const int rq = (int)((unsigned)it.y >> kBatchFaceBits);
    const int fi = it.y & ((1 << kBatchFaceBits) - 1);
    const DevRequest& q = ba.req[rq];
    const int loc = it.x - __ldg(ba.pix0 + rq);
    const int xw = loc % q.cam.w, yw = loc / q.cam.w;
    const int px = q.cam.x0 + xw, py = q.cam.y0 + yw;
    float o[3], d[3];
    make_ray<float>(q.cam, px, py, o, d);
    if (!roots_item<P, float, MIXED, STATS>(V, q.cam64, it.x, fi, px, py, o, d, q.diag, stride, frag_tp,
                                                   frag_meta, frag_count, st, c_tests, c_newton, c_fp64, c_frag))
      defer_item(i, slow, cap, n_items);
  }
  roots_counters<STATS, false>(c_tests, c_newton, c_fp64, c_frag, n, st);
}

template <int P, bool MIXED, bool STATS>
__global__ void __launch_bounds__(kRootsThreads) kb2c_split(DevVolume V, BatchArgs ba, const int2* __restrict__ items,
                                                            const int* __restrict__ slow, int* __restrict__ n_items,
                                                            int cap, int warp_max, float4* __restrict__ frag_tp,
                                                            unsigned* __restrict__ frag_meta,
                                                            int* __restrict__ frag_count, size_t stride,
                                                            DevStats* __restrict__ st) {
  __shared__ SplitSmem<float> s_split[kRootsThreads / 32];
  SplitSmem<float>& sm = s_split[threadIdx.x >> 5];
  const int n = min(n_items[kSlowCounter - kItemCounter], cap);
  if (n > warp_max) return;
  unsigned long long c_fp64 = 0, c_frag = 0;
  int c_newton = 0;
  unsigned dropped = 0;
  for (;;) {
    int k = 0;
    if ((threadIdx.x & 31) == 0) k = atomicAdd(n_items + (kSlowHead - kItemCounter), 1);
    k = __shfl_sync(0xffffffffu, k, 0);
    if (k >= n) break;
    const int2 it = __ldg(items + __ldg(slow + k));
    const int rq = (int)((unsigned)it.y >> kBatchFaceBits);
    const int fi = it.y & ((1 << kBatchFaceBits) - 1);
    const DevRequest& q = ba.req[rq];
    const int loc = it.x - __ldg(ba.pix0 + rq);
    const int xw = loc % q.cam.w, yw = loc / q.cam.w;
    const int px = q.cam.x0 + xw, py = q.cam.y0 + yw;
    float o[3], d[3];
    make_ray<float>(q.cam, px, py, o, d);
    split_item_warp<P, float, MIXED, STATS>(V, q.cam64, it.x, fi, px, py, o, d, q.diag, stride, frag_tp, frag_meta,
                                            frag_count, st, sm, c_newton, c_fp64, c_frag, dropped);
  }
  if (dropped) atomicAdd(&st->abuf_overflow, (unsigned long long)dropped);
  roots_counters<STATS, true>(0, c_newton, c_fp64, c_frag, n, st);
}

template <int P, bool MIXED, bool STATS>
__global__ void __launch_bounds__(kRootsThreads, 4) kb2c_thread(DevVolume V, BatchArgs ba,
                                                                const int2* __restrict__ items,
                                                                const int* __restrict__ slow,
                                                                int* __restrict__ n_items, int cap, int warp_max,
                                                                float4* __restrict__ frag_tp,
                                                                unsigned* __restrict__ frag_meta,
                                                                int* __restrict__ frag_count, size_t stride,
                                                                DevStats* __restrict__ st) {
  const int n = min(n_items[kSlowCounter - kItemCounter], cap);
  if (n <= warp_max) return;
  unsigned long long c_fp64 = 0, c_frag = 0;
  int c_newton = 0;
  __shared__ ThreadDeepSmem<P> s_deep[kRootsThreads / 32];
  ThreadDeepSmem<P>& dm = s_deep[threadIdx.x >> 5];
  for (;;) {
    const int base = take_items(n_items, n, kSlowHead);
    if (base >= n) break;
    const int k = base + (int)(threadIdx.x & 31);
    const bool have = k < n;
    int pix = 0, fi = 0, px = 0, py = 0, rq = 0;
    float o[3] = {0, 0, 0}, d[3] = {0, 0, 1}, diag = 1.f;
    if (have) {
      const int2 it = __ldg(items + __ldg(slow + k));
      rq = (int)((unsigned)it.y >> kBatchFaceBits);
      fi = it.y & ((1 << kBatchFaceBits) - 1);
      pix = it.x;
      const DevRequest& q = ba.req[rq];
      const int loc = it.x - __ldg(ba.pix0 + rq);
      px = q.cam.x0 + loc % q.cam.w;
      py = q.cam.y0 + loc / q.cam.w;
      diag = q.diag;
      make_ray<float>(q.cam, px, py, o, d);
    }
    split_round_thread<P, MIXED, STATS>(V, ba.req[rq].cam64, have, pix, fi, px, py, o, d, diag, stride, frag_tp,
                                        frag_meta, frag_count, st, dm, c_newton, c_fp64, c_frag);
  }
  roots_counters<STATS, true>(0, c_newton, c_fp64, c_frag, n, st);
}

template <int P, bool MIXED, bool STATS>
void launch_kb2b(const DevVolume& V, const BatchArgs& ba, const SurfaceWs& w, size_t stride, DevStats* st,
                 int num_sms, cudaStream_t s) {
  static int per_sm[3] = {-1, -1, -1};
  if (per_sm[0] < 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], kb2b_roots<P, MIXED, STATS>, kRootsThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], kb2c_split<P, MIXED, STATS>, kRootsThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[2], kb2c_thread<P, MIXED, STATS>, kRootsThreads, 0);
    for (int& x : per_sm) x = x < 1 ? 1 : x;
  }
  const int warp_max = kSplitWaves * num_sms * per_sm[1] * (kRootsThreads / 32);
  kb2b_roots<P, MIXED, STATS><<<num_sms * per_sm[0], kRootsThreads, 0, s>>>(
      V, ba, w.items, w.slow, w.n_items, w.cap, (float4*)w.frag_tp, w.frag_meta, w.frag_count, stride, st);
  kb2c_split<P, MIXED, STATS><<<num_sms * per_sm[1], kRootsThreads, 0, s>>>(
      V, ba, w.items, w.slow, w.n_items, w.cap, warp_max, (float4*)w.frag_tp, w.frag_meta, w.frag_count, stride, st);
  kb2c_thread<P, MIXED, STATS><<<num_sms * per_sm[2], kRootsThreads, 0, s>>>(
      V, ba, w.items, w.slow, w.n_items, w.cap, warp_max, (float4*)w.frag_tp, w.frag_meta, w.frag_count, stride, st);
}

template <int TW, int TH>
void launch_kb2a(const DevVolume& V, const BatchArgs& ba, int tiles, const SurfaceWs& w, DevStats* st,
                 cudaStream_t s) {
  kb2a_cull<TW, TH><<<(tiles + kCullWarps - 1) / kCullWarps, 32 * kCullWarps, 0, s>>>(
      V, ba, tiles, w.boxes, w.gboxes, w.items, w.cap, w.n_items, w.frag_count, st);
}

}  // namespace

void launch_batch_face_project(const DevVolume& V, const BatchArgs& ba, int max_faces, const SurfaceWs& w,
                               cudaStream_t s) {
  if (max_faces <= 0 || ba.nreq <= 0) return;
  const dim3 grid((max_faces + 127) / 128, ba.nreq);
  if (V.P == 2)
    kb0_face_project<2><<<grid, 128, 0, s>>>(V, ba, w.boxes, w.gboxes);
  else
    kb0_face_project<3><<<grid, 128, 0, s>>>(V, ba, w.boxes, w.gboxes);
}

bool launch_batch_intersect(const DevVolume& V, const BatchArgs& ba, int tiles, int tile_w, int tile_h, bool mixed,
                            bool stats, const SurfaceWs& w, size_t stride, DevStats* st, int num_sms,
                            cudaStream_t s) {
  if (tiles <= 0) return true;
  if (tile_w == 8 && tile_h == 4)
    launch_kb2a<8, 4>(V, ba, tiles, w, st, s);
  else if (tile_w == 4 && tile_h == 8)
    launch_kb2a<4, 8>(V, ba, tiles, w, st, s);
  else if (tile_w == 16 && tile_h == 2)
    launch_kb2a<16, 2>(V, ba, tiles, w, st, s);
  else
    return false;
#define IVV_KB2B(PP, MM, SS) launch_kb2b<PP, MM, SS>(V, ba, w, stride, st, num_sms, s)
  if (V.P == 2) {
    if (mixed) { if (stats) IVV_KB2B(2, true, true); else IVV_KB2B(2, true, false); }
    else { if (stats) IVV_KB2B(2, false, true); else IVV_KB2B(2, false, false); }
  } else {
    if (mixed) { if (stats) IVV_KB2B(3, true, true); else IVV_KB2B(3, true, false); }
    else { if (stats) IVV_KB2B(3, false, true); else IVV_KB2B(3, false, false); }
  }
#undef IVV_KB2B
  return true;
}

}  // namespace ivv
