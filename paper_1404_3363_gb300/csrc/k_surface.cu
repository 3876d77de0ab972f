// Stage 1 (§4.1): intersections of every pixel ray with the boundary surfaces
// of every block.  The paper rasterises a view-dependent pixel-accurate
// tessellation; here every ray is intersected with the Bezier face patches
// directly (device bodies in k_surface.cuh):
//   K0 face_project  -- conservative screen box of each face patch.
//   K2 intersect     -- one CTA per 16x8 screen tile; fragments go to the
//                       pixel's A-buffer slots (§4.2).
#include <cuda_runtime.h>

#include "k_surface.cuh"

namespace ivv {

namespace {

template <int P>
__global__ void k0_face_project(DevVolume V, DevCamera<float> cam, int4* __restrict__ boxes) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= V.n_faces) return;
  boxes[f] = face_box<P>(V, cam, f, V.diag);
}

template <int P, typename R, bool MIXED, bool STATS>
__global__ void __launch_bounds__(kTileW * kTileH, 4) k2_intersect(DevVolume V, DevCamera<R> cam, DevCamera<double> cam64,
                                                       const int4* __restrict__ boxes,
                                                       typename Vec4T<R>::type* __restrict__ frag_tp,
                                                       unsigned* __restrict__ frag_meta, int* __restrict__ frag_count,
                                                       DevStats* __restrict__ st) {
  const int tiles_x = (cam.w + kTileW - 1) / kTileW;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  k2_tile<P, R, MIXED, STATS, kTileW, kTileH>(V, cam, cam64, tx, ty, 0, V.n_faces, boxes, V.diag, 0,
                                              (size_t)cam.w * cam.h, frag_tp, frag_meta, frag_count, st);
}

}  // namespace

void launch_face_project(const DevVolume& V, const DevCamera<float>& cam, int4* boxes, cudaStream_t s) {
  if (V.n_faces <= 0) return;
  if (V.P == 2)
    k0_face_project<2><<<(V.n_faces + 127) / 128, 128, 0, s>>>(V, cam, boxes);
  else
    k0_face_project<3><<<(V.n_faces + 127) / 128, 128, 0, s>>>(V, cam, boxes);
}

template <typename R>
void launch_intersect(const DevVolume& V, const DevCamera<R>& cam, const DevCamera<double>& cam64, bool mixed,
                      bool stats, const int4* boxes, typename Vec4T<R>::type* frag_tp, unsigned* frag_meta,
                      int* frag_count, DevStats* st, cudaStream_t s) {
  const int tiles = ((cam.w + kTileW - 1) / kTileW) * ((cam.h + kTileH - 1) / kTileH);
  if (tiles <= 0) return;
#define IVV_K2(PP, MM, SS) \
  k2_intersect<PP, R, MM, SS><<<tiles, kTileW * kTileH, 0, s>>>(V, cam, cam64, boxes, frag_tp, frag_meta, frag_count, st)
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
