// Batched stage 1 (§4.1) and the launchers of the batched stages: one K0
// launch over every (request, face) and one K2 launch over every screen tile
// of every request of a batch.  A CTA of K2 finds its request from the
// batch's tile table and runs the same tile body as the single-frame kernel
// (k_surface.cuh) on that request's camera, faces and slice of the pixel
// space.
#include <cuda_runtime.h>

#include "k_surface.cuh"

namespace ivv {

namespace {

template <int P>
__global__ void kb0_face_project(DevVolume V, BatchArgs ba, int4* __restrict__ boxes) {
  const DevRequest& q = ba.req[blockIdx.y];
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= q.n_faces) return;
  boxes[q.box0 + f] = face_box<P>(V, q.cam, q.face0 + f, q.diag);
}

template <int P, bool MIXED, bool STATS, int TW, int TH>
__global__ void __launch_bounds__(TW * TH, 512 / (TW * TH))
    kb2_intersect(DevVolume V, BatchArgs ba, const int4* __restrict__ boxes, float4* __restrict__ frag_tp,
                  unsigned* __restrict__ frag_meta, int* __restrict__ frag_count, size_t stride,
                  DevStats* __restrict__ st) {
  const int tile = blockIdx.x;
  const int rq = batch_find(ba.tile0, ba.nreq, tile);
  const DevRequest& q = ba.req[rq];
  const DevCamera<float> cam = q.cam;
  const int tiles_x = (cam.w + TW - 1) / TW;
  const int t = tile - __ldg(ba.tile0 + rq);
  k2_tile<P, float, MIXED, STATS, TW, TH>(V, cam, q.cam64, t % tiles_x, t / tiles_x, q.face0, q.n_faces,
                                          boxes + q.box0, q.diag, (size_t)__ldg(ba.pix0 + rq), stride, frag_tp,
                                          frag_meta, frag_count, st);
}

template <int P, int TW, int TH>
void launch_kb2(const DevVolume& V, const BatchArgs& ba, int tiles, bool mixed, bool stats, const int4* boxes,
                float4* frag_tp, unsigned* frag_meta, int* frag_count, size_t stride, DevStats* st, cudaStream_t s) {
#define IVV_KB2(MM, SS) \
  kb2_intersect<P, MM, SS, TW, TH><<<tiles, TW * TH, 0, s>>>(V, ba, boxes, frag_tp, frag_meta, frag_count, stride, st)
  if (mixed) {
    if (stats) IVV_KB2(true, true); else IVV_KB2(true, false);
  } else {
    if (stats) IVV_KB2(false, true); else IVV_KB2(false, false);
  }
#undef IVV_KB2
}

template <int P>
bool launch_kb2_shape(const DevVolume& V, const BatchArgs& ba, int tiles, int tw, int th, bool mixed, bool stats,
                      const int4* boxes, float4* frag_tp, unsigned* frag_meta, int* frag_count, size_t stride,
                      DevStats* st, cudaStream_t s) {
  if (tw == 16 && th == 8)
    launch_kb2<P, 16, 8>(V, ba, tiles, mixed, stats, boxes, frag_tp, frag_meta, frag_count, stride, st, s);
  else if (tw == 8 && th == 8)
    launch_kb2<P, 8, 8>(V, ba, tiles, mixed, stats, boxes, frag_tp, frag_meta, frag_count, stride, st, s);
  else if (tw == 16 && th == 16)
    launch_kb2<P, 16, 16>(V, ba, tiles, mixed, stats, boxes, frag_tp, frag_meta, frag_count, stride, st, s);
  else
    return false;
  return true;
}

}  // namespace

void launch_batch_face_project(const DevVolume& V, const BatchArgs& ba, int max_faces, int4* boxes, cudaStream_t s) {
  if (max_faces <= 0 || ba.nreq <= 0) return;
  const dim3 grid((max_faces + 127) / 128, ba.nreq);
  if (V.P == 2)
    kb0_face_project<2><<<grid, 128, 0, s>>>(V, ba, boxes);
  else
    kb0_face_project<3><<<grid, 128, 0, s>>>(V, ba, boxes);
}

bool launch_batch_intersect(const DevVolume& V, const BatchArgs& ba, int tiles, int tile_w, int tile_h, bool mixed,
                            bool stats, const int4* boxes, float4* frag_tp, unsigned* frag_meta, int* frag_count,
                            size_t stride, DevStats* st, cudaStream_t s) {
  if (tiles <= 0) return true;
  if (V.P == 2)
    return launch_kb2_shape<2>(V, ba, tiles, tile_w, tile_h, mixed, stats, boxes, frag_tp, frag_meta, frag_count,
                               stride, st, s);
  return launch_kb2_shape<3>(V, ba, tiles, tile_w, tile_h, mixed, stats, boxes, frag_tp, frag_meta, frag_count,
                             stride, st, s);
}

}  // namespace ivv
