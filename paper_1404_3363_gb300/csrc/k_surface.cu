// Stage 1 (§4.1) of a single frame: intersections of every pixel ray with the
// boundary surfaces of every block (device bodies in k_surface.cuh):
//   K0  k0_face_project -- screen boxes of the face patches and of groups of
//       32 patches.
//   K2a k2a_cull        -- one warp per 8x4 tile: culling and per-pixel
//       bounding-box tests; (pixel, patch) items to a global list.
//   K2b k2b_roots       -- one thread per item: hull test, roots of the
//       certified one-to-one patches, fragments into the pixel's A-buffer
//       slots (§4.2); items whose patch needs the subdivision search are
//       deferred to
//   K2c k2c_split / k2c_thread -- the subdivision search of the deferred
//       items: a warp per item, level by level across its lanes, while they
//       fit a few waves of warps; a thread per item beyond that.
#include <cuda_runtime.h>

#include "k_surface.cuh"

namespace ivv {

namespace {

constexpr int kCullWarps = 8;        // warps (8x4 tiles) per K2a CTA
constexpr int kRootsThreads = 128;

template <int P>
__global__ void k0_face_project(DevVolume V, DevCamera<float> cam, int4* __restrict__ boxes,
                                int4* __restrict__ gboxes) {
  pdl_wait();
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  project_faces<P>(V, cam, f, V.n_faces, 0, V.diag, boxes, gboxes);
}

template <typename R>
__global__ void __launch_bounds__(32 * kCullWarps) k2a_cull(DevVolume V, DevCamera<R> cam,
                                                            const int4* __restrict__ boxes,
                                                            const int4* __restrict__ gboxes, int2* __restrict__ items,
                                                            int cap, int* __restrict__ n_items,
                                                            int* __restrict__ frag_count, int* __restrict__ tile_flag,
                                                            int* __restrict__ pair_count,
                                                            float4* __restrict__ zero_out, DevStats* __restrict__ st) {
  pdl_wait();
  const int tiles_x = (cam.w + 7) / 8;
  const int tiles = tiles_x * ((cam.h + 3) / 4);
  const int t = blockIdx.x * kCullWarps + (threadIdx.x >> 5);
  if (t >= tiles) return;                      // whole warps
  const int tx = t % tiles_x, ty = t / tiles_x;
  const bool any = cull_warp_tile<R, 8, 4>(V, cam, tx, ty, 0, V.n_faces, boxes, gboxes, V.diag, 0, 0, items, cap,
                                           n_items, frag_count, st);
  if (tile_flag == nullptr) return;
  const int lane = threadIdx.x & 31;
  if (any) {
    // the 16 x 16 tile of K4 that holds this 8 x 4 warp tile
    if (lane == 0) tile_flag[(ty >> 2) * ((cam.w + 15) >> 4) + (tx >> 1)] = 1;
  } else {
    // no candidate: no fragments, no pairs, a zero pixel (K4 may skip it)
    const int xw = tx * 8 + (lane & 7), yw = ty * 4 + (lane >> 3);
    if (xw < cam.w && yw < cam.h) {
      const int pix = yw * cam.w + xw;
      pair_count[pix] = 0;
      if (zero_out) zero_out[pix] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

// K2b: every item on the certified fast path, the others deferred to the
// list `slow`.  Warps take 32 consecutive items at a time.
template <int P, typename R, bool MIXED, bool STATS>
__global__ void __launch_bounds__(kRootsThreads, 4) k2b_roots(DevVolume V, DevCamera<R> cam,
                                                              DevCamera<double> cam64,
                                                              const int2* __restrict__ items,
                                                              int* __restrict__ slow, int* __restrict__ n_items,
                                                              int cap, typename Vec4T<R>::type* __restrict__ frag_tp,
                                                              unsigned* __restrict__ frag_meta,
                                                              int* __restrict__ frag_count,
                                                              DevStats* __restrict__ st) {
  pdl_wait();
  const int n = min(n_items[0], cap);
  const size_t stride = (size_t)cam.w * cam.h;
  unsigned long long c_tests = 0, c_fp64 = 0, c_frag = 0;
  int c_newton = 0;
  for (;;) {
    const int base = take_items(n_items, n);
    if (base >= n) break;
    const int i = base + (int)(threadIdx.x & 31);
    if (i >= n) continue;
    const int2 it = __ldg(items + i);
    const int xw = it.x % cam.w, yw = it.x / cam.w;
    const int px = cam.x0 + xw, py = cam.y0 + yw;
    R o[3], d[3];
    make_ray<R>(cam, px, py, o, d);
    if (!roots_item<P, R, MIXED, STATS>(V, cam64, it.x, it.y, px, py, o, d, V.diag, stride, frag_tp,
                                               frag_meta, frag_count, st, c_tests, c_newton, c_fp64, c_frag))
      defer_item(i, slow, cap, n_items);
  }
  roots_counters<STATS, false>(c_tests, c_newton, c_fp64, c_frag, n, st);
}

// K2c: the deferred items' subdivision search.  With at most `warp_max`
// deferred items (they fit a few waves of warps) each gets a whole warp
// (split_item_warp, short latency); with more, one thread each
// (k2c_thread, throughput).  Both kernels are launched; the one whose case
// does not hold returns at once.
template <int P, typename R, bool MIXED, bool STATS>
__global__ void __launch_bounds__(kRootsThreads) k2c_split(DevVolume V, DevCamera<R> cam, DevCamera<double> cam64,
                                                           const int2* __restrict__ items,
                                                           const int* __restrict__ slow, int* __restrict__ n_items,
                                                           int cap, int warp_max,
                                                           typename Vec4T<R>::type* __restrict__ frag_tp,
                                                           unsigned* __restrict__ frag_meta,
                                                           int* __restrict__ frag_count, DevStats* __restrict__ st) {
  __shared__ SplitSmem<R> s_split[kRootsThreads / 32];
  SplitSmem<R>& sm = s_split[threadIdx.x >> 5];
  pdl_wait();
  const int n = min(n_items[kSlowCounter - kItemCounter], cap);
  if (n > warp_max) return;
  const size_t stride = (size_t)cam.w * cam.h;
  unsigned long long c_fp64 = 0, c_frag = 0;
  int c_newton = 0;
  unsigned dropped = 0;
  for (;;) {
    int k = 0;
    if ((threadIdx.x & 31) == 0) k = atomicAdd(n_items + (kSlowHead - kItemCounter), 1);
    k = __shfl_sync(0xffffffffu, k, 0);
    if (k >= n) break;
    const int2 it = __ldg(items + __ldg(slow + k));
    const int xw = it.x % cam.w, yw = it.x / cam.w;
    const int px = cam.x0 + xw, py = cam.y0 + yw;
    R o[3], d[3];
    make_ray<R>(cam, px, py, o, d);
    split_item_warp<P, R, MIXED, STATS>(V, cam64, it.x, it.y, px, py, o, d, V.diag, stride, frag_tp, frag_meta,
                                        frag_count, st, sm, c_newton, c_fp64, c_frag, dropped);
  }
  if (dropped) atomicAdd(&st->abuf_overflow, (unsigned long long)dropped);
  roots_counters<STATS, true>(0, c_newton, c_fp64, c_frag, n, st);
}

template <int P, typename R, bool MIXED, bool STATS>
__global__ void __launch_bounds__(kRootsThreads, 4) k2c_thread(DevVolume V, DevCamera<R> cam,
                                                               DevCamera<double> cam64,
                                                               const int2* __restrict__ items,
                                                               const int* __restrict__ slow,
                                                               int* __restrict__ n_items, int cap, int warp_max,
                                                               typename Vec4T<R>::type* __restrict__ frag_tp,
                                                               unsigned* __restrict__ frag_meta,
                                                               int* __restrict__ frag_count,
                                                               DevStats* __restrict__ st) {
  pdl_wait();
  const int n = min(n_items[kSlowCounter - kItemCounter], cap);
  if (n <= warp_max) return;
  const size_t stride = (size_t)cam.w * cam.h;
  unsigned long long c_fp64 = 0, c_frag = 0;
  int c_newton = 0;
  if constexpr (sizeof(R) == 4) {
    __shared__ ThreadDeepSmem<P> s_deep[kRootsThreads / 32];
    ThreadDeepSmem<P>& dm = s_deep[threadIdx.x >> 5];
    for (;;) {
      const int base = take_items(n_items, n, kSlowHead);
      if (base >= n) break;
      const int k = base + (int)(threadIdx.x & 31);
      const bool have = k < n;
      int2 it = make_int2(0, 0);
      int px = 0, py = 0;
      R o[3] = {0, 0, 0}, d[3] = {0, 0, 1};
      if (have) {
        it = __ldg(items + __ldg(slow + k));
        px = cam.x0 + it.x % cam.w;
        py = cam.y0 + it.x / cam.w;
        make_ray<R>(cam, px, py, o, d);
      }
      split_round_thread<P, MIXED, STATS>(V, cam64, have, it.x, it.y, px, py, o, d, V.diag, stride, frag_tp,
                                          frag_meta, frag_count, st, dm, c_newton, c_fp64, c_frag);
    }
  } else {
    for (;;) {
      const int base = take_items(n_items, n, kSlowHead);
      if (base >= n) break;
      const int k = base + (int)(threadIdx.x & 31);
      if (k >= n) continue;
      const int2 it = __ldg(items + __ldg(slow + k));
      const int xw = it.x % cam.w, yw = it.x / cam.w;
      const int px = cam.x0 + xw, py = cam.y0 + yw;
      R o[3], d[3];
      make_ray<R>(cam, px, py, o, d);
      split_item_thread<P, R, MIXED, STATS>(V, cam64, it.x, it.y, px, py, o, d, V.diag, stride, frag_tp, frag_meta,
                                            frag_count, st, c_newton, c_fp64, c_frag);
    }
  }
  roots_counters<STATS, true>(0, c_newton, c_fp64, c_frag, n, st);
}

// K2p: the deferred FP64 polish of the grazing hits listed by K2b / K2c
// (mixed precision), one thread per hit.
template <int P, bool STATS>
__global__ void __launch_bounds__(128) k2p_polish(DevVolume V, DevCamera<double> cam64, float4* __restrict__ frag_tp,
                                                  DevStats* __restrict__ st) {
  pdl_wait();
  const int n = min(*V.n_polish, V.polish_cap);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    polish_hit<P>(V, cam64, k, frag_tp);
  if (STATS && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&st->fp64_solves, (unsigned long long)n);
}

template <int P, typename R, bool MIXED, bool STATS>
void launch_k2b(const DevVolume& V, const DevCamera<R>& cam, const DevCamera<double>& cam64, const SurfaceWs& w,
                DevStats* st, int num_sms, cudaStream_t s) {
  typedef typename Vec4T<R>::type V4;
  static int per_sm[3] = {-1, -1, -1};
  if (per_sm[0] < 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], k2b_roots<P, R, MIXED, STATS>, kRootsThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], k2c_split<P, R, MIXED, STATS>, kRootsThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[2], k2c_thread<P, R, MIXED, STATS>, kRootsThreads, 0);
    for (int& x : per_sm) x = x < 1 ? 1 : x;
  }
  const int warp_max = kSplitWaves * num_sms * per_sm[1] * (kRootsThreads / 32);
  launch_pdl(k2b_roots<P, R, MIXED, STATS>, dim3(num_sms * per_sm[0]), dim3(kRootsThreads), s, V, cam, cam64,
             w.items, w.slow, w.n_items, w.cap, (V4*)w.frag_tp, w.frag_meta, w.frag_count, st);
  launch_pdl(k2c_split<P, R, MIXED, STATS>, dim3(num_sms * per_sm[1]), dim3(kRootsThreads), s, V, cam, cam64,
             (const int2*)w.items, (const int*)w.slow, w.n_items, w.cap, warp_max, (V4*)w.frag_tp, w.frag_meta,
             w.frag_count, st);
  launch_pdl(k2c_thread<P, R, MIXED, STATS>, dim3(num_sms * per_sm[2]), dim3(kRootsThreads), s, V, cam, cam64,
             (const int2*)w.items, (const int*)w.slow, w.n_items, w.cap, warp_max, (V4*)w.frag_tp, w.frag_meta,
             w.frag_count, st);
  if constexpr (MIXED && sizeof(R) == 4) {
    if (V.polish != nullptr)
      launch_pdl(k2p_polish<P, STATS>, dim3(num_sms * 4), dim3(128), s, V, cam64, (float4*)w.frag_tp, st);
  }
}

}  // namespace

void launch_face_project(const DevVolume& V, const DevCamera<float>& cam, int4* boxes, int4* gboxes,
                         cudaStream_t s) {
  if (V.n_faces <= 0) return;
  if (V.P == 2)
    launch_pdl(k0_face_project<2>, dim3((V.n_faces + 127) / 128), dim3(128), s, V, cam, boxes, gboxes);
  else
    launch_pdl(k0_face_project<3>, dim3((V.n_faces + 127) / 128), dim3(128), s, V, cam, boxes, gboxes);
}

template <typename R>
void launch_intersect(const DevVolume& V, const DevCamera<R>& cam, const DevCamera<double>& cam64, bool mixed,
                      bool stats, const SurfaceWs& w, DevStats* st, int num_sms, cudaStream_t s) {
  const int tiles = ((cam.w + 7) / 8) * ((cam.h + 3) / 4);
  if (tiles <= 0) return;
  launch_pdl(k2a_cull<R>, dim3((tiles + kCullWarps - 1) / kCullWarps), dim3(32 * kCullWarps), s, V, cam,
             (const int4*)w.boxes, (const int4*)w.gboxes, w.items, w.cap, w.n_items, w.frag_count, w.tile_flag,
             w.pair_count, w.zero_out, st);
#define IVV_K2B(PP, MM, SS) launch_k2b<PP, R, MM, SS>(V, cam, cam64, w, st, num_sms, s)
  if constexpr (sizeof(R) == 4) {
    if (V.P == 2) {
      if (mixed) { if (stats) IVV_K2B(2, true, true); else IVV_K2B(2, true, false); }
      else { if (stats) IVV_K2B(2, false, true); else IVV_K2B(2, false, false); }
    } else {
      if (mixed) { if (stats) IVV_K2B(3, true, true); else IVV_K2B(3, true, false); }
      else { if (stats) IVV_K2B(3, false, true); else IVV_K2B(3, false, false); }
    }
  } else {
    (void)mixed;
    if (V.P == 2) { if (stats) IVV_K2B(2, false, true); else IVV_K2B(2, false, false); }
    else { if (stats) IVV_K2B(3, false, true); else IVV_K2B(3, false, false); }
  }
#undef IVV_K2B
}

template void launch_intersect<float>(const DevVolume&, const DevCamera<float>&, const DevCamera<double>&, bool,
                                      bool, const SurfaceWs&, DevStats*, int, cudaStream_t);
template void launch_intersect<double>(const DevVolume&, const DevCamera<double>&, const DevCamera<double>&, bool,
                                       bool, const SurfaceWs&, DevStats*, int, cudaStream_t);

}  // namespace ivv
