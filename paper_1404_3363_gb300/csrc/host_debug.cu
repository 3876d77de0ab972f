// Host execution of the stage 1-2 code (isect.cuh) that the device kernels
// run, for inspection and CPU testing of a volume description.  ivv_render
// never uses it: rendering needs the GPU.
#include <cmath>
#include <string>
#include <vector>

#include "ivv_device.cuh"
#include "ivv_internal.h"

namespace ivv {
std::string& last_error_ref();
ivv_status resolve_params_host(double diag, const ivv_render_params* in, ivv_render_params& p);
ivv_status frame_cameras(const ivv_camera* c, const ivv_render_params& p, int width, int height,
                         DevCamera<float>& c32, DevCamera<double>& c64);
}  // namespace ivv

namespace {

template <int P, typename R>
ivv_status host_pairs(const ivv::HostVolume& hv, const ivv::DevCamera<float>& c32, const ivv::DevCamera<double>& c64,
                      bool mixed, int max_pairs, int* pair_count, double* pairs, int* pair_block) {
  using namespace ivv;
  constexpr int NN = (P + 1) * (P + 1);
  const int F = hv.n_faces();
  const int w = c32.w, h = c32.h, npix = w * h;
  std::vector<float4> face32(hv.face_cp.size() / 4);
  std::vector<Dbl4> face64(hv.face_cp.size() / 4);
  for (size_t i = 0; i < face32.size(); ++i) {
    face32[i] = make_float4((float)hv.face_cp[4 * i], (float)hv.face_cp[4 * i + 1], (float)hv.face_cp[4 * i + 2], 0.f);
    face64[i].x = hv.face_cp[4 * i];
    face64[i].y = hv.face_cp[4 * i + 1];
    face64[i].z = hv.face_cp[4 * i + 2];
    face64[i].w = 0.0;
  }
  std::vector<int4> boxes(F);
  for (int f = 0; f < F; ++f) boxes[f] = face_screen_box<NN>(c32, &face32[(size_t)f * NN], hv.faces[f].org, (float)hv.diag);
  DevCamera<R> cam;
  if constexpr (sizeof(R) == 4) cam = c32; else cam = c64;
  const R tau = sizeof(R) == 4 ? R(1e-5) * R(hv.diag) : R(1e-9) * R(hv.diag);
  const R hull_pad = R(1e-6) * R((float)hv.diag);
  for (int yw = 0; yw < h; ++yw)
    for (int xw = 0; xw < w; ++xw) {
      const int px = c32.x0 + xw, py = c32.y0 + yw, pix = yw * w + xw;
      const int tx = xw / kTileW, ty = yw / kTileH;
      const int rx0 = c32.x0 + tx * kTileW, ry0 = c32.y0 + ty * kTileH;
      const int rx1 = std::min(rx0 + kTileW - 1, c32.x0 + w - 1), ry1 = std::min(ry0 + kTileH - 1, c32.y0 + h - 1);
      R o[3], d[3], e1[3], e2[3], inv_d[3];
      make_ray<R>(cam, px, py, o, d);
      ray_frame<R>(d, e1, e2);
      for (int r = 0; r < 3; ++r) inv_d[r] = R(1) / d[r];
      R tt[kMaxFrags], pp_all[kMaxFrags][3];
      unsigned mm[kMaxFrags];
      int n = 0, iters = 0;
      for (int f = 0; f < F; ++f) {
        const int4 b = boxes[f];
        if (!(b.x <= rx1 && b.z >= rx0 && b.y <= ry1 && b.w >= ry0)) continue;
        const FaceMeta& m = hv.faces[f];
        if (!ray_box<R>(o, inv_d, m.lo, m.hi, hull_pad) || !ray_obb<R>(o, d, m, R(4) * hull_pad)) continue;
        const FaceMeta64& m64 = hv.faces64[f];
        R org[3], pa0, pa1, pb0, pb1;
        if constexpr (sizeof(R) == 8) {
          for (int r = 0; r < 3; ++r) org[r] = m64.org[r];
          pa0 = m64.a0; pa1 = m64.a1; pb0 = m64.b0; pb1 = m64.b1;
        } else {
          for (int r = 0; r < 3; ++r) org[r] = m.org[r];
          pa0 = m.a0; pa1 = m.a1; pb0 = m.b0; pb1 = m.b1;
        }
        Patch2<P, R> pq;
        R ra[kMaxPatchRoots], rb[kMaxPatchRoots];
        int nr;
        if constexpr (sizeof(R) == 8) {
          const Dbl4* cp = &face64[(size_t)f * NN];
          project_patch<P, R, Dbl4>(cp, org, o, e1, e2, pq);
          if (!hull_has_origin<P, R>(pq, hull_pad)) continue;
          nr = patch_roots<P, R>(pq, hull_pad, ra, rb, iters);
        } else {
          const float4* cp = &face32[(size_t)f * NN];
          project_patch<P, R, float4>(cp, org, o, e1, e2, pq);
          if (!hull_has_origin<P, R>(pq, hull_pad)) continue;
          nr = patch_roots<P, R>(pq, hull_pad, ra, rb, iters);
        }
        for (int k = 0; k < nr; ++k) {
          const R a = ra[k], b2 = rb[k];     // within the acceptance tolerance of the patch
          R t, pp[3], cosang;
          bool front;
          if constexpr (sizeof(R) == 8)
            make_fragment<P, R, Dbl4>(&face64[(size_t)f * NN], org, m, pa0, pa1, pb0, pb1, o, d, a, b2, t, front, pp, cosang);
          else
            make_fragment<P, R, float4>(&face32[(size_t)f * NN], org, m, pa0, pa1, pb0, pb1, o, d, a, b2, t, front, pp,
                                        cosang);
          if (sizeof(R) == 4 && mixed && cosang < R(kPolishCos)) {
            double a64 = a, b64 = b2, t64 = t, o64[3], d64[3];
            make_ray<double>(c64, px, py, o64, d64);
            refine_hit_mixed<P>(&face64[(size_t)f * NN], &face32[(size_t)f * NN], m64.org, o64, d64, a64, b64, t64);
            t = R(t64);
            const int nd = m.face >> 1, ad = (nd + 1) % 3, bd = (nd + 2) % 3;
            pp[ad] = R(std::fmin(std::fmax(m64.a0 + a64 * (m64.a1 - m64.a0), 0.0), 1.0));
            pp[bd] = R(std::fmin(std::fmax(m64.b0 + b64 * (m64.b1 - m64.b0), 0.0), 1.0));
          }
          if (!(t > R(0)) || n >= kMaxFrags) continue;
          tt[n] = t;
          for (int r = 0; r < 3; ++r) pp_all[n][r] = pp[r];
          mm[n] = ((unsigned)m.block << 4) | ((unsigned)m.face << 1) | (front ? 1u : 0u);
          ++n;
        }
      }
      int in_idx[kMaxPairs], out_idx[kMaxPairs];
      unsigned um = 0, pov = 0;
      const int np = pair_fragments<R>(n, tt, mm, pp_all, tau, std::min(max_pairs, (int)kMaxPairs), in_idx, out_idx, um, pov);
      pair_count[pix] = np;
      for (int q = 0; q < np; ++q) {
        double* o8 = pairs + ((size_t)q * npix + pix) * 8;
        const int a = in_idx[q], b = out_idx[q];
        o8[0] = pp_all[a][0]; o8[1] = pp_all[a][1]; o8[2] = pp_all[a][2]; o8[3] = tt[a];
        o8[4] = pp_all[b][0]; o8[5] = pp_all[b][1]; o8[6] = pp_all[b][2]; o8[7] = tt[b];
        pair_block[(size_t)q * npix + pix] = (int)(mm[a] >> 4);
      }
    }
  return IVV_OK;
}

}  // namespace

extern "C" ivv_status ivv_host_render_pairs(const ivv_block_desc* blocks, int n_blocks, int scalar_mode,
                                            const ivv_camera* cam, const ivv_render_params* params, int width,
                                            int height, int max_pairs, int* pair_count, double* pairs,
                                            int* pair_block) {
  if (!pair_count || !pairs || !pair_block || max_pairs < 1) {
    ivv::last_error_ref() = "NULL output or max_pairs < 1";
    return IVV_ERR_INVALID_ARG;
  }
  ivv::HostVolume hv;
  std::string err;
  ivv_status st = ivv::prepare_volume(blocks, n_blocks, scalar_mode, hv, err);
  if (st != IVV_OK) {
    ivv::last_error_ref() = err;
    return st;
  }
  ivv_render_params p;
  st = ivv::resolve_params_host(hv.diag, params, p);
  if (st != IVV_OK) return st;
  ivv::DevCamera<float> c32;
  ivv::DevCamera<double> c64;
  st = ivv::frame_cameras(cam, p, width, height, c32, c64);
  if (st != IVV_OK) return st;
  const bool mixed = p.precision == IVV_PREC_MIXED;
  if (p.precision == IVV_PREC_FP64)
    return hv.P == 2 ? host_pairs<2, double>(hv, c32, c64, false, max_pairs, pair_count, pairs, pair_block)
                     : host_pairs<3, double>(hv, c32, c64, false, max_pairs, pair_count, pairs, pair_block);
  return hv.P == 2 ? host_pairs<2, float>(hv, c32, c64, mixed, max_pairs, pair_count, pairs, pair_block)
                   : host_pairs<3, float>(hv, c32, c64, mixed, max_pairs, pair_count, pairs, pair_block);
}
