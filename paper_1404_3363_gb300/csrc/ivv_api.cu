// C ABI of the isogeometric volume ray integrator (include/ivv.h): volume
// upload, per-frame workspace layout, stage launches and status plumbing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "ivv_device.cuh"
#include "ivv_internal.h"
#include "mlp.cuh"
#include "volume.h"
#include <random>

namespace ivv {
template <int P>
void launch_integrate_p(const DevVolume& V, const DevCamera<float>* cam32, const DevCamera<double>* cam64,
                        const DevTF& tf, const IntegrateArgs& a, bool mixed, bool stats, const void* pin,
                        const void* pout, const int* pblk, const int* pcnt, const int* active, const int* n_active,
                        int* queue_head, float4* out, DevStats* st, int num_sms, cudaStream_t s);
void launch_export_pairs(int npix, int max_pairs, bool fp64, const void* pin, const void* pout, const int* pblk,
                         const int* pcnt, int* out_count, float* out_pairs, int* out_block, cudaStream_t s);
void stats_to_public(const DevStats& d, ivv_stats* out);
}  // namespace ivv

namespace {

thread_local std::string g_err;

ivv_status fail(ivv_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

ivv_status cuda_fail(cudaError_t e, const char* what) {
  return fail(IVV_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define IVV_CUDA(call)                                    \
  do {                                                    \
    cudaError_t e__ = (call);                             \
    if (e__ != cudaSuccess) return cuda_fail(e__, #call); \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct WsLayout {
  size_t boxes, gboxes, items, slow, frag_tp, frag_meta, frag_count, pair_in, pair_out, pair_block, pair_count, active,
      tile_flag, polish, counters, total;
};

// Grazing hits per frame whose FP64 polish (mixed precision) runs in its own
// pass: one per pixel of the window (beyond it, hits are polished inline).
// Volumes with at most this many Bezier elements solve the RF method's
// samples in element order (a counting sort over the element index whose
// histogram fits shared memory; beyond it the sort's global-atomic form cost
// more than the ordered Newton saved: 1080p bar and beam +7 to +10 %, the
// 8904-element 4K step -9 %).
constexpr int kElemSortMax = 4096;

size_t polish_cap(size_t npix) { return std::max<size_t>(npix, 1024); }

WsLayout layout(int n_faces, size_t npix, size_t v4) {
  WsLayout L;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o += align256(bytes); return at; };
  L.boxes = take(sizeof(int4) * (size_t)std::max(n_faces, 1));
  L.gboxes = take(sizeof(int4) * (size_t)std::max((n_faces + 31) / 32, 1));
  L.items = take(sizeof(int2) * ivv::kItemsPerPixel * npix);
  L.slow = take(sizeof(int) * ivv::kItemsPerPixel * npix);
  L.frag_tp = take(v4 * ivv::kMaxFrags * npix);
  L.frag_meta = take(sizeof(unsigned) * ivv::kMaxFrags * npix);
  L.frag_count = take(sizeof(int) * npix);
  L.pair_in = take(v4 * ivv::kMaxPairs * npix);
  L.pair_out = take(v4 * ivv::kMaxPairs * npix);
  L.pair_block = take(sizeof(int) * ivv::kMaxPairs * npix);
  L.pair_count = take(sizeof(int) * npix);
  L.active = take(sizeof(int) * npix);
  // one flag per 16 x 16 tile: ceil(w/16) ceil(h/16) <= npix/256 + (w+h)/16 + 1 <= npix/8 + 3
  L.tile_flag = take(sizeof(int) * (npix / 8 + 64));
  L.polish = take(2 * sizeof(float4) * polish_cap(npix));
  L.counters = take(ivv::kCountersBytes);
  L.total = o;
  return L;
}

}  // namespace


namespace {

void free_volume(ivv_volume* v) {
  if (!v) return;
  if (v->copy_stream) {
    cudaStreamSynchronize(v->copy_stream);
    cudaStreamDestroy(v->copy_stream);
  }
  for (int k = 0; k < 2; ++k) {
    if (v->own_out2[k]) cudaFree(v->own_out2[k]);
    if (v->ev_rendered[k]) cudaEventDestroy(v->ev_rendered[k]);
    if (v->ev_copied[k]) cudaEventDestroy(v->ev_copied[k]);
  }
  void* ptrs[] = {v->d_blocks, v->d_brk32, v->d_brk64, v->d_elem32, v->d_elem64, v->d_org32, v->d_rho32, v->d_org64,
                  v->d_disp32, v->d_dorg32, v->d_disp64, v->d_dorg64, v->d_count, v->d_face32, v->d_face64,
                  v->d_faces, v->d_faces64, v->d_tf_r, v->d_tf_rgba, v->d_stats, v->own_ws, v->own_out};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (cudaEvent_t e : v->ev)
    if (e) cudaEventDestroy(e);
  void* g[] = {v->d_theta, v->d_adam_m, v->d_adam_v, v->d_theta16, v->d_norms, v->rf_buf, v->ode_buf};
  for (void* p : g)
    if (p) cudaFree(p);
  delete v;
}

template <typename T>
ivv_status upload(T** dst, const T* src, size_t n, cudaStream_t s) {
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)dst, sizeof(T) * n);
  if (e != cudaSuccess) return fail(IVV_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  if (src) {
    e = cudaMemcpyAsync(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
  }
  return IVV_OK;
}

ivv::DevVolume dev_volume(const ivv_volume* v) {
  ivv::DevVolume V;
  V.P = v->hv.P;
  V.mode = v->hv.mode;
  V.n_blocks = v->hv.n_blocks;
  V.n_faces = v->hv.n_faces();
  V.blocks = v->d_blocks;
  V.brk32 = v->d_brk32;
  V.brk64 = v->d_brk64;
  V.elem32 = v->d_elem32;
  V.elem64 = v->d_elem64;
  V.org32 = v->d_org32;
  V.rho32 = v->d_rho32;
  V.org64 = v->d_org64;
  V.disp32 = v->d_disp32;
  V.dorg32 = v->d_dorg32;
  V.disp64 = v->d_disp64;
  V.dorg64 = v->d_dorg64;
  V.face32 = v->d_face32;
  V.face64 = v->d_face64;
  V.faces = v->d_faces;
  V.faces64 = v->d_faces64;
  V.diag = (float)v->hv.diag;
  V.max_frags = v->lim_frags;
  V.max_newton = v->lim_newton;
  V.polish = nullptr;
  V.polish_cap = 0;
  V.n_polish = nullptr;
  return V;
}

// Largest window of one render: pixel, item and slot indices stay in int.
constexpr long long kMaxWindowPixels = 1ll << 27;

struct Frame {
  double eye[3], f[3], r[3], u[3], sx, sy;
  int ortho, W, H, x0, y0, w, h;
};

ivv_status make_frame(const ivv_camera* c, const ivv_render_params& p, int width, int height, Frame& F) {
  if (!c) return fail(IVV_ERR_INVALID_ARG, "camera is NULL");
  if (width <= 0 || height <= 0) return fail(IVV_ERR_INVALID_ARG, "width and height must be positive");
  if ((long long)width * height > kMaxWindowPixels)
    return fail(IVV_ERR_INVALID_ARG, "window larger than 2^27 pixels");
  F.W = p.full_width > 0 ? p.full_width : width;
  F.H = p.full_height > 0 ? p.full_height : height;
  F.x0 = p.x0;
  F.y0 = p.y0;
  F.w = width;
  F.h = height;
  if (F.x0 < 0 || F.y0 < 0 || F.x0 + width > F.W || F.y0 + height > F.H)
    return fail(IVV_ERR_INVALID_ARG, "window outside the full image");
  double f[3], n = 0;
  for (int i = 0; i < 3; ++i) {
    if (!std::isfinite(c->eye[i]) || !std::isfinite(c->target[i]) || !std::isfinite(c->up[i]))
      return fail(IVV_ERR_INVALID_ARG, "non-finite camera");
    f[i] = c->target[i] - c->eye[i];
    n += f[i] * f[i];
  }
  n = std::sqrt(n);
  if (!(n > 0)) return fail(IVV_ERR_INVALID_ARG, "camera target equals eye");
  for (int i = 0; i < 3; ++i) f[i] /= n;
  double r[3] = {f[1] * c->up[2] - f[2] * c->up[1], f[2] * c->up[0] - f[0] * c->up[2],
                 f[0] * c->up[1] - f[1] * c->up[0]};
  const double nr = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  if (!(nr > 1e-12)) return fail(IVV_ERR_INVALID_ARG, "camera up is parallel to the view direction");
  for (int i = 0; i < 3; ++i) r[i] /= nr;
  double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
  const double aspect = (double)F.W / F.H;
  if (c->ortho) {
    if (!(c->ortho_height > 0)) return fail(IVV_ERR_INVALID_ARG, "ortho_height must be positive");
    F.sy = 0.5 * c->ortho_height;
    F.sx = F.sy * aspect;
  } else {
    if (!(c->fovy_deg > 0 && c->fovy_deg < 180)) return fail(IVV_ERR_INVALID_ARG, "fovy_deg must be in (0,180)");
    F.sy = std::tan(0.5 * c->fovy_deg * M_PI / 180.0);
    F.sx = F.sy * aspect;
  }
  F.ortho = c->ortho ? 1 : 0;
  for (int i = 0; i < 3; ++i) {
    F.eye[i] = c->eye[i];
    F.f[i] = f[i];
    F.r[i] = r[i];
    F.u[i] = u[i];
  }
  return IVV_OK;
}

template <typename R>
ivv::DevCamera<R> dev_camera(const Frame& F) {
  ivv::DevCamera<R> c;
  for (int i = 0; i < 3; ++i) {
    c.eye[i] = (R)F.eye[i];
    c.f[i] = (R)F.f[i];
    c.r[i] = (R)F.r[i];
    c.u[i] = (R)F.u[i];
  }
  c.sx = (R)F.sx;
  c.sy = (R)F.sy;
  c.ortho = F.ortho;
  c.W = F.W;
  c.H = F.H;
  c.x0 = F.x0;
  c.y0 = F.y0;
  c.w = F.w;
  c.h = F.h;
  return c;
}

ivv_status resolve_params_diag(double diag, const ivv_render_params* in, ivv_render_params& p) {
  if (in) {
    p = *in;
  } else {
    std::memset(&p, 0, sizeof(p));
    p.rk_tol = 1e-5;
    p.supersample_k = 4;
    p.c = 1.0;
    p.early_alpha = 1.0 - 1e-4;
  }
  if (!(p.rf_tol > 0)) p.rf_tol = 0.05;
  if (!(p.ds > 0)) p.ds = diag / 128.0;
  if (!(p.rk_tol > 0) || !std::isfinite(p.rk_tol)) return fail(IVV_ERR_INVALID_ARG, "rk_tol must be positive");
  if (p.supersample_k < 1 || p.supersample_k > 64) return fail(IVV_ERR_INVALID_ARG, "supersample_k must be in 1..64");
  if (!(p.c >= 0) || !std::isfinite(p.c)) return fail(IVV_ERR_INVALID_ARG, "c must be non-negative");
  if (!(p.early_alpha > 0)) return fail(IVV_ERR_INVALID_ARG, "early_alpha must be positive");
  if (p.precision < IVV_PREC_FP32 || p.precision > IVV_PREC_FP64) return fail(IVV_ERR_INVALID_ARG, "bad precision");
  if (p.method != IVV_METHOD_ODE && p.method != IVV_METHOD_RF) return fail(IVV_ERR_INVALID_ARG, "bad method");
  if (p.use_mlp_guess < IVV_GUESS_CENTER || p.use_mlp_guess > IVV_GUESS_CHORD)
    return fail(IVV_ERR_INVALID_ARG, "bad initial-guess mode");
  if (p.method == IVV_METHOD_ODE && p.use_mlp_guess == IVV_GUESS_CHORD)
    return fail(IVV_ERR_INVALID_ARG, "the chord guess applies to the RF method");
  if (p.method == IVV_METHOD_RF && p.precision == IVV_PREC_FP64)
    return fail(IVV_ERR_UNSUPPORTED, "the RF method runs in FP32 or MIXED precision");
  if (p.rk_method < IVV_RK_BS32 || p.rk_method > IVV_RK_IMPLICIT_EULER) return fail(IVV_ERR_INVALID_ARG, "bad rk_method");
  if (p.rk_method != IVV_RK_BS32 && p.method != IVV_METHOD_ODE)
    return fail(IVV_ERR_INVALID_ARG, "rk_method applies to the ODE method");
  if (p.rk_method != IVV_RK_BS32 && p.precision == IVV_PREC_FP64)
    return fail(IVV_ERR_UNSUPPORTED, "the fixed-step integrators run in FP32 or MIXED precision");
  if (!(p.near_clip >= 0) || !std::isfinite(p.near_clip)) return fail(IVV_ERR_INVALID_ARG, "near_clip must be >= 0");
  if (p.n_cut_planes < 0 || p.n_cut_planes > IVV_MAX_CUT_PLANES)
    return fail(IVV_ERR_INVALID_ARG, "n_cut_planes must be in 0..IVV_MAX_CUT_PLANES");
  for (int k = 0; k < p.n_cut_planes; ++k) {
    const double* c = p.cut_planes[k];
    if (!(std::isfinite(c[0]) && std::isfinite(c[1]) && std::isfinite(c[2]) && std::isfinite(c[3])))
      return fail(IVV_ERR_INVALID_ARG, "non-finite cutting plane");
    if (!(c[0] * c[0] + c[1] * c[1] + c[2] * c[2] > 0)) return fail(IVV_ERR_INVALID_ARG, "cutting plane normal is zero");
  }
  return IVV_OK;
}

ivv_status resolve_params(const ivv_volume* v, const ivv_render_params* in, ivv_render_params& p) {
  return resolve_params_diag(v->hv.diag, in, p);
}

// Tableaux of the fixed-step family (published coefficients: Euler;
// explicit midpoint; Kutta 1901 third order; classic RK4; Kutta's 3/8 rule;
// Fehlberg 1969 4(5) nodes with the fifth-order weights).
ivv::RkTableau rk_tableau(int method) {
  ivv::RkTableau T;
  std::memset(&T, 0, sizeof(T));
  switch (method) {
    case IVV_RK_EULER:
      T.s = 1; T.b[0] = 1.f;
      break;
    case IVV_RK_MIDPOINT:
      T.s = 2; T.a[1][0] = 0.5f; T.b[1] = 1.f;
      break;
    case IVV_RK_KUTTA3:
      T.s = 3; T.a[1][0] = 0.5f; T.a[2][0] = -1.f; T.a[2][1] = 2.f;
      T.b[0] = 1.f / 6; T.b[1] = 2.f / 3; T.b[2] = 1.f / 6;
      break;
    case IVV_RK_RK4:
      T.s = 4; T.a[1][0] = 0.5f; T.a[2][1] = 0.5f; T.a[3][2] = 1.f;
      T.b[0] = 1.f / 6; T.b[1] = 1.f / 3; T.b[2] = 1.f / 3; T.b[3] = 1.f / 6;
      break;
    case IVV_RK_RK4_38:
      T.s = 4; T.a[1][0] = 1.f / 3; T.a[2][0] = -1.f / 3; T.a[2][1] = 1.f;
      T.a[3][0] = 1.f; T.a[3][1] = -1.f; T.a[3][2] = 1.f;
      T.b[0] = 1.f / 8; T.b[1] = 3.f / 8; T.b[2] = 3.f / 8; T.b[3] = 1.f / 8;
      break;
    case IVV_RK_FEHLBERG5: {
      T.s = 6;
      const double a[6][5] = {{0, 0, 0, 0, 0},
                              {1.0 / 4, 0, 0, 0, 0},
                              {3.0 / 32, 9.0 / 32, 0, 0, 0},
                              {1932.0 / 2197, -7200.0 / 2197, 7296.0 / 2197, 0, 0},
                              {439.0 / 216, -8.0, 3680.0 / 513, -845.0 / 4104, 0},
                              {-8.0 / 27, 2.0, -3544.0 / 2565, 1859.0 / 4104, -11.0 / 40}};
      const double b[6] = {16.0 / 135, 0, 6656.0 / 12825, 28561.0 / 56430, -9.0 / 50, 2.0 / 55};
      for (int i = 0; i < 6; ++i) {
        for (int j = 0; j < 5; ++j) T.a[i][j] = (float)a[i][j];
        T.b[i] = (float)b[i];
      }
      break;
    }
    default:
      T.s = 0;
  }
  return T;
}

ivv_status ensure_own(void** buf, size_t* have, size_t need, cudaStream_t s) {
  if (*have >= need) return IVV_OK;
  cudaStreamCaptureStatus cs;
  if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
    return fail(IVV_ERR_WORKSPACE, "library workspace must grow, but a stream capture is active");
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc(buf, need);
  if (e != cudaSuccess) return fail(IVV_ERR_OOM, std::string("cudaMalloc workspace: ") + cudaGetErrorString(e));
  *have = need;
  return IVV_OK;
}

// Stages 1-2 into the workspace.  out_zero receives zero pixels for rays
// without pairs (may be NULL).
template <typename R>
// count (optional): K4 also counts the pixels' samples into the sample
// lists when no fix-up solve moves a pair end after it; *counted tells.
ivv_status run_surface_pairs(ivv_volume* v, const Frame& F, const ivv_render_params& p, char* ws, const WsLayout& L,
                             int max_pairs, float4* out_zero, cudaStream_t s, const ivv::SampleCount* count = nullptr,
                             bool* counted = nullptr) {
  typedef typename ivv::Vec4T<R>::type V4;
  ivv::DevVolume V = dev_volume(v);
  const int npix = F.w * F.h;
  const bool stats = (p.flags & IVV_FLAG_STATS) != 0;
  const bool mixed = p.precision == IVV_PREC_MIXED;
  if (mixed && sizeof(R) == 4) {
    V.polish = (float4*)(ws + L.polish);
    V.polish_cap = (int)std::min<size_t>(polish_cap((size_t)npix), 0x7fffffff);
    V.n_polish = (int*)(ws + L.counters) + ivv::kPolishCounter;
  }
  const bool timing = (p.flags & IVV_FLAG_TIMING) != 0;
  IVV_CUDA(cudaMemsetAsync(ws + L.counters, 0, ivv::kCountersBytes, s));
  ivv::SurfaceWs sw;
  sw.boxes = (int4*)(ws + L.boxes);
  sw.gboxes = (int4*)(ws + L.gboxes);
  sw.items = (int2*)(ws + L.items);
  sw.slow = (int*)(ws + L.slow);
  sw.cap = (int)std::min<size_t>((size_t)v->lim_items * npix, 0x7fffffff);
  sw.n_items = (int*)(ws + L.counters) + ivv::kItemCounter;
  sw.frag_tp = ws + L.frag_tp;
  sw.frag_meta = (unsigned*)(ws + L.frag_meta);
  sw.frag_count = (int*)(ws + L.frag_count);
  sw.tile_flag = (int*)(ws + L.tile_flag);
  sw.pair_count = (int*)(ws + L.pair_count);
  sw.zero_out = out_zero;
  if (timing) IVV_CUDA(cudaEventRecord(v->ev[0], s));
  ivv::launch_face_project(V, dev_camera<float>(F), sw.boxes, sw.gboxes, s);
  if (timing) IVV_CUDA(cudaEventRecord(v->ev[1], s));
  ivv::launch_intersect<R>(V, dev_camera<R>(F), dev_camera<double>(F), mixed, stats, sw, v->d_stats, v->num_sms, s);
  if (timing) IVV_CUDA(cudaEventRecord(v->ev[2], s));
  ivv::ClipArgs<R> clip;
  std::memset(&clip, 0, sizeof(clip));
  clip.on = (p.near_clip > 0 || p.n_cut_planes > 0) ? 1 : 0;
  clip.near = (R)p.near_clip;
  for (int r = 0; r < 3; ++r) clip.f[r] = (R)F.f[r];
  clip.n_cut = p.n_cut_planes;
  for (int k = 0; k < p.n_cut_planes; ++k)
    for (int c = 0; c < 4; ++c) clip.cut[k][c] = (R)p.cut_planes[k][c];
  clip.cam = dev_camera<R>(F);
  const bool count_here = count != nullptr && sizeof(R) == 4 && !clip.on && !v->hv.any_singular;
  if (counted) *counted = count_here;
  ivv::launch_pair<R>(V, F.w, npix, (float)v->hv.diag, (const V4*)(ws + L.frag_tp), (const unsigned*)(ws + L.frag_meta),
                      (const int*)(ws + L.frag_count), (V4*)(ws + L.pair_in), (V4*)(ws + L.pair_out),
                      (int*)(ws + L.pair_block), (int*)(ws + L.pair_count), max_pairs, (int*)(ws + L.active),
                      (int*)(ws + L.counters), out_zero, clip, sw.tile_flag, v->d_stats, s,
                      count_here ? count : nullptr);
  // fix-up solves of stage 2: ends moved onto cutting or near-clip planes
  // (§5.5) and entries with a singular Jacobian (§5.4), the entries without
  // chord context from the learned guess when it is asked for
  const bool learned = p.use_mlp_guess == IVV_GUESS_MLP && v->guess_ready && (clip.on || v->hv.any_singular);
  if (learned) {
    ivv::GuessList gl;
    gl.g = (float4*)(ws + L.frag_tp);                 // the fragment lists are dead after K4
    gl.p = gl.g + (size_t)ivv::kMaxPairs * npix;
    gl.gidx = (int*)(ws + L.frag_meta);
    gl.blk = gl.gidx + (size_t)ivv::kMaxPairs * npix;
    gl.n = (int*)(ws + L.counters) + ivv::kGuessCounter;
    ivv::launch_guess_mark<R>(V, clip.cam, npix, (V4*)(ws + L.pair_in), (V4*)(ws + L.pair_out),
                              (int*)(ws + L.pair_block), (const int*)(ws + L.pair_count), (const int*)(ws + L.active),
                              (const int*)(ws + L.counters), v->hv.any_singular, mixed, gl, v->d_stats, v->num_sms,
                              s);
    ivv::launch_mlp_infer(v->d_theta16, v->d_norms, gl.g, gl.blk, gl.n, 0, gl.p, v->d_stats, v->num_sms, s);
    ivv::launch_clip_solve<R>(V, clip.cam, npix, (V4*)(ws + L.pair_in), (V4*)(ws + L.pair_out),
                              (int*)(ws + L.pair_block), (const int*)(ws + L.pair_count), (const int*)(ws + L.active),
                              (const int*)(ws + L.counters), mixed, &gl, v->d_stats, v->num_sms, s);
  } else if (clip.on) {
    ivv::launch_clip_solve<R>(V, clip.cam, npix, (V4*)(ws + L.pair_in), (V4*)(ws + L.pair_out),
                              (int*)(ws + L.pair_block), (const int*)(ws + L.pair_count), (const int*)(ws + L.active),
                              (const int*)(ws + L.counters), mixed, nullptr, v->d_stats, v->num_sms, s);
  }
  if (v->hv.any_singular)
    ivv::launch_entry_fix<R>(V, clip.cam, npix, (V4*)(ws + L.pair_in), (V4*)(ws + L.pair_out),
                             (const int*)(ws + L.pair_block), (const int*)(ws + L.pair_count),
                             (const int*)(ws + L.active), (const int*)(ws + L.counters), mixed, v->d_stats, v->num_sms,
                             s);
  if (timing) IVV_CUDA(cudaEventRecord(v->ev[3], s));
  IVV_CUDA(cudaGetLastError());
  return IVV_OK;
}

// Sample-list capacity per pixel of the split integration: the pairs of a
// ray lie in disjoint blocks inside the control-point box, so their lengths
// add up to at most its diagonal; each pair adds at most two partial samples.
// Up to kSplitBoundBytes the sample list is sized by this bound (no host
// round trip); above it the render reads the exact sample total back first
// (not inside a stream capture), and above kSplitMaxBytes of samples it keeps
// the fused integrator.
constexpr double kSplitBoundBytes = 4.0 * (1ull << 30);
constexpr double kSplitMaxBytes = 64.0 * (1ull << 30);
size_t split_bound(const ivv_volume* v, const ivv_render_params& p) {
  return (size_t)std::ceil(v->hv.diag / p.ds) + 2 * ivv::kMaxPairs + 2;
}
double split_bytes(const ivv_volume* v, const ivv_render_params& p, size_t npix) {
  return (double)split_bound(v, p) * (double)npix * (double)sizeof(float4);
}

ivv_status render_impl(ivv_volume* v, const ivv_camera* cam, const ivv_render_params* params, int width, int height,
                       float* out, void* workspace, size_t workspace_bytes, cudaStream_t s,
                       bool ws_is_scratch = false) {
  if (!v) return fail(IVV_ERR_INVALID_ARG, "volume is NULL");
  if (!out) return fail(IVV_ERR_INVALID_ARG, "out_rgba is NULL");
  if (((uintptr_t)out) % 16) return fail(IVV_ERR_INVALID_ARG, "out_rgba must be 16-byte aligned");
  if (!v->tf_set) return fail(IVV_ERR_INVALID_ARG, "no transfer function set");
  ivv_render_params p;
  ivv_status st = resolve_params(v, params, p);
  if (st != IVV_OK) return st;
  Frame F;
  st = make_frame(cam, p, width, height, F);
  if (st != IVV_OK) return st;
  const bool fp64 = p.precision == IVV_PREC_FP64;
  const size_t npix = (size_t)width * height;
  const WsLayout L = layout(v->hv.n_faces(), npix, fp64 ? sizeof(ivv::Dbl4) : sizeof(float4));
  char* ws = (char*)workspace;
  if (ws) {
    if (workspace_bytes < L.total) return fail(IVV_ERR_WORKSPACE, "workspace smaller than ivv_workspace_size");
    if (((uintptr_t)ws) % 256) return fail(IVV_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  } else {
    st = ensure_own(&v->own_ws, &v->own_ws_bytes, L.total, s);
    if (st != IVV_OK) return st;
    ws = (char*)v->own_ws;
  }
  v->last_stream = s;
  const ivv::DevVolume V = dev_volume(v);
  ivv::DevTF tf;
  tf.n = v->tf_n;
  tf.sigma = v->sigma;
  tf.lo = (float)v->lo;
  tf.inv_range = (float)(1.0 / (v->hi - v->lo));
  tf.r = v->d_tf_r;
  tf.rgba = v->d_tf_rgba;
  ivv::IntegrateArgs a;
  a.rk_tol = (float)p.rk_tol;
  a.ds = (float)p.ds;
  a.c = (float)p.c;
  a.early_alpha = (float)p.early_alpha;
  a.K = p.supersample_k;
  a.max_steps = v->lim_rk_steps;
  a.max_step_samples = 8;
  a.npix = (int)npix;
  const bool stats = (p.flags & IVV_FLAG_STATS) != 0;
  const bool mixed = p.precision == IVV_PREC_MIXED;
  if (p.use_mlp_guess == IVV_GUESS_MLP && !v->guess_ready)
    return fail(IVV_ERR_INVALID_ARG, "IVV_GUESS_MLP needs ivv_train_guess or ivv_set_guess_weights first");
  if (p.method == IVV_METHOD_RF) {
    int* counters = (int*)(ws + L.counters);
    const float tail_eps = (float)(1e-12 * v->hv.diag);
    // sample lists counted by K4 where no fix-up follows it (their arrays in
    // the stage-1 item list, dead after K2c), else by the count and scan
    // kernels over the fragment lists, dead after stage 2
    ivv::SampleCount sc{(float)p.ds, tail_eps, (int*)(ws + L.items), (int*)(ws + L.items) + npix, counters + 2};
    bool counted = false;
    st = run_surface_pairs<float>(v, F, p, ws, L, v->lim_pairs, (float4*)out, s, &sc, &counted);
    if (st != IVV_OK) return st;
    const float4* pin = (const float4*)(ws + L.pair_in);
    const float4* pout = (const float4*)(ws + L.pair_out);
    const int* pblk = (const int*)(ws + L.pair_block);
    const int* pcnt = (const int*)(ws + L.pair_count);
    const int* act = (const int*)(ws + L.active);
    int* cnt = counted ? sc.cnt : (int*)(ws + L.frag_count);
    int* off = counted ? sc.off : (int*)(ws + L.frag_meta);
    int* sums = (int*)(ws + L.frag_meta) + npix;
    if (!counted) {
      ivv::launch_rf_count(pin, pout, pblk, pcnt, act, counters, (int)npix, (float)p.ds, tail_eps, cnt, v->num_sms,
                           s);
      ivv::launch_rf_scan(cnt, counters, (int)npix, off, sums, 0x7fffffff, counters + 2, s);
    }
    int totals[2] = {0, 0};
    IVV_CUDA(cudaMemcpyAsync(totals, counters + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    IVV_CUDA(cudaStreamSynchronize(s));
    if (totals[1] != 0) return fail(IVV_ERR_UNSUPPORTED, "the frame's sample count exceeds INT_MAX");
    const int total = totals[0];
    // per sample: world point, guess, block, scalar, the sorted order (by
    // block for the learned guess's inference, then by element for Newton)
    // and the element key; then the sort's histogram
    const size_t per = 2 * sizeof(float4) + 4 * sizeof(int);
    const size_t cap_n = (size_t)std::max(total, 1);
    const int nb = v->hv.n_blocks;
    const int ne = v->hv.n_elems();
    const bool esort = ne <= kElemSortMax;
    st = ensure_own(&v->rf_buf, &v->rf_bytes, cap_n * per + sizeof(int) * ((size_t)std::max(nb, ne) + 1) + 1024, s);
    if (st != IVV_OK) return st;
    char* rb = (char*)v->rf_buf;
    float4* sg = (float4*)rb;
    float4* sp = sg + cap_n;
    int* sblk = (int*)(sp + cap_n);
    float* srho = (float*)(sblk + cap_n);
    int* sperm = (int*)(srho + cap_n);
    int* skey = sperm + cap_n;
    int* shist = skey + cap_n;
    ivv::DevCamera<float> c32 = dev_camera<float>(F);
    ivv::launch_rf_expand(c32, pin, pout, pblk, pcnt, act, counters, off, (int)npix, (float)p.ds, tail_eps,
                          p.use_mlp_guess, total, sg, sblk, sp, v->num_sms, s);
    // Newton in the order of the elements of the samples' chord points: a
    // warp's control-point loads then meet one or two elements instead of
    // the several that consecutive samples of neighbouring rays cross.  The
    // element order is also block order, so the inference reads it too.
    if (esort) {
      ivv::launch_rf_elem_key(V, counters + 2, sblk, sp, skey, v->num_sms, s);
      ivv::launch_block_sort(skey, counters + 2, ne, shist, sperm, v->num_sms, s);
    }
    if (p.use_mlp_guess == IVV_GUESS_MLP) {
      // with many blocks a tile of consecutive samples spans many of them
      // (one inference pass each): read them in block order; with few, the
      // scattered reads of the sorted order cost more than the passes
      const bool sort = nb >= 8;
      if (sort && !esort) ivv::launch_block_sort(sblk, counters + 2, nb, shist, sperm, v->num_sms, s);
      ivv::launch_mlp_infer(v->d_theta16, v->d_norms, sg, sblk, counters + 2, 0, sp, v->d_stats, v->num_sms, s,
                            sort ? sperm : nullptr);
    }
    if (p.flags & IVV_FLAG_TIMING) IVV_CUDA(cudaEventRecord(v->ev[3], s));
    ivv::launch_rf_newton(V, c32, (float)p.rf_tol, 0.f, counters + 2, sg, sblk, sp, srho, nullptr, nullptr, v->d_stats,
                          stats, mixed, v->num_sms, s, esort ? sperm : nullptr);
    ivv::launch_rf_composite(tf, p.supersample_k, (float)p.early_alpha, pin, pout, pblk, pcnt, act, counters, off,
                             (int)npix, (float)p.ds, tail_eps, total, srho, (float4*)out, v->d_stats, stats,
                             v->num_sms, s);
    if (p.flags & IVV_FLAG_TIMING) {
      IVV_CUDA(cudaEventRecord(v->ev[4], s));
      v->timed = true;
    }
    IVV_CUDA(cudaGetLastError());
    return IVV_OK;
  }
  if (fp64) {
    st = run_surface_pairs<double>(v, F, p, ws, L, v->lim_pairs, (float4*)out, s);
    if (st != IVV_OK) return st;
    ivv::DevCamera<double> c64 = dev_camera<double>(F);
    if (V.P == 2)
      ivv::launch_integrate_p<2>(V, nullptr, &c64, tf, a, false, stats, ws + L.pair_in, ws + L.pair_out,
                                 (const int*)(ws + L.pair_block), (const int*)(ws + L.pair_count),
                                 (const int*)(ws + L.active), (const int*)(ws + L.counters),
                                 (int*)(ws + L.counters) + ivv::kQueueHeadOff, (float4*)out, v->d_stats, v->num_sms, s);
    else
      ivv::launch_integrate_p<3>(V, nullptr, &c64, tf, a, false, stats, ws + L.pair_in, ws + L.pair_out,
                                 (const int*)(ws + L.pair_block), (const int*)(ws + L.pair_count),
                                 (const int*)(ws + L.active), (const int*)(ws + L.counters),
                                 (int*)(ws + L.counters) + ivv::kQueueHeadOff, (float4*)out, v->d_stats, v->num_sms, s);
  } else if (p.rk_method == IVV_RK_IMPLICIT_EULER) {
    st = run_surface_pairs<float>(v, F, p, ws, L, v->lim_pairs, (float4*)out, s);
    if (st != IVV_OK) return st;
    const ivv::DevCamera<float> c32 = dev_camera<float>(F);
    const float4* pin = (const float4*)(ws + L.pair_in);
    const float4* pout = (const float4*)(ws + L.pair_out);
    if (V.P == 2)
      ivv::launch_irk1_p<2>(V, c32, tf, a, mixed, stats, pin, pout, (const int*)(ws + L.pair_block),
                            (const int*)(ws + L.pair_count), (const int*)(ws + L.active),
                            (const int*)(ws + L.counters), (int*)(ws + L.counters) + ivv::kQueueHeadOff,
                            (float4*)out, v->d_stats, v->num_sms, s);
    else
      ivv::launch_irk1_p<3>(V, c32, tf, a, mixed, stats, pin, pout, (const int*)(ws + L.pair_block),
                            (const int*)(ws + L.pair_count), (const int*)(ws + L.active),
                            (const int*)(ws + L.counters), (int*)(ws + L.counters) + ivv::kQueueHeadOff,
                            (float4*)out, v->d_stats, v->num_sms, s);
  } else if (p.rk_method != IVV_RK_BS32) {
    st = run_surface_pairs<float>(v, F, p, ws, L, v->lim_pairs, (float4*)out, s);
    if (st != IVV_OK) return st;
    const ivv::DevCamera<float> c32 = dev_camera<float>(F);
    const ivv::RkTableau T = rk_tableau(p.rk_method);
    const float4* pin = (const float4*)(ws + L.pair_in);
    const float4* pout = (const float4*)(ws + L.pair_out);
    if (V.P == 2)
      ivv::launch_fixed_p<2>(V, c32, tf, a, T, mixed, stats, pin, pout, (const int*)(ws + L.pair_block),
                             (const int*)(ws + L.pair_count), (const int*)(ws + L.active),
                             (const int*)(ws + L.counters), (int*)(ws + L.counters) + ivv::kQueueHeadOff,
                             (float4*)out, v->d_stats, v->num_sms, s);
    else
      ivv::launch_fixed_p<3>(V, c32, tf, a, T, mixed, stats, pin, pout, (const int*)(ws + L.pair_block),
                             (const int*)(ws + L.pair_count), (const int*)(ws + L.active),
                             (const int*)(ws + L.counters), (int*)(ws + L.counters) + ivv::kQueueHeadOff,
                             (float4*)out, v->d_stats, v->num_sms, s);
  } else {
    // split integration: sample lists (counted by K4, or count and scan),
    // trace kernel writing the sample points, scalar at every sample and
    // per-pixel compositing
    const bool by_bound = split_bytes(v, p, npix) <= kSplitBoundBytes;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool capturing = cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
    bool split = !ws_is_scratch && (by_bound || !capturing);
    int* counters = (int*)(ws + L.counters);
    const float tail_eps = 1e-12f * (float)v->hv.diag;  // as the integrator computes it
    ivv::SampleCount sc{(float)p.ds, tail_eps, (int*)(ws + L.items), (int*)(ws + L.items) + npix, counters + 2};
    bool counted = false;
    st = run_surface_pairs<float>(v, F, p, ws, L, v->lim_pairs, (float4*)out, s, split ? &sc : nullptr, &counted);
    if (st != IVV_OK) return st;
    const ivv::DevCamera<float> c32 = dev_camera<float>(F);
    const float4* pin = (const float4*)(ws + L.pair_in);
    const float4* pout = (const float4*)(ws + L.pair_out);
    const int* pblk = (const int*)(ws + L.pair_block);
    const int* pcnt = (const int*)(ws + L.pair_count);
    const int* act = (const int*)(ws + L.active);
    size_t cap = 0;
    int* cnt = counted ? sc.cnt : (int*)(ws + L.frag_count);   // fragment lists are dead after stage 2
    int* off = counted ? sc.off : (int*)(ws + L.frag_meta);
    int* sums = (int*)(ws + L.frag_meta) + npix;
    if (split) {
      if (!counted) {
        ivv::launch_rf_count(pin, pout, pblk, pcnt, act, counters, (int)npix, (float)p.ds, tail_eps, cnt,
                             v->num_sms, s);
        ivv::launch_rf_scan(cnt, counters, (int)npix, off, sums, 0x7fffffff, counters + 2, s);
      }
      if (by_bound) {
        cap = split_bound(v, p) * npix;
      } else {
        int total[2] = {0, 0};          // the sample total and its excess over INT_MAX
        IVV_CUDA(cudaMemcpyAsync(total, counters + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        IVV_CUDA(cudaStreamSynchronize(s));
        cap = (size_t)std::max(total[0], 1);
        split = total[1] == 0 && (double)cap * sizeof(float4) <= kSplitMaxBytes;
      }
    }
    if (split) {
      st = ensure_own(&v->ode_buf, &v->ode_bytes, cap * sizeof(float4), s);
      if (st != IVV_OK) return st;
      ivv::SplitArgs sa;
      sa.off = off;
      sa.sp = (float4*)v->ode_buf;
      sa.cap = (int)cap;
      if (V.P == 2) {
        ivv::launch_integrate_split_p<2>(V, c32, a, sa, mixed, stats, pin, pout, pblk, pcnt, act, counters,
                                         counters + ivv::kQueueHeadOff, v->d_stats, v->num_sms, s);
        ivv::launch_shade_composite_p<2>(V, c32, tf, p.supersample_k, (float)p.early_alpha, pin, pout, pblk, pcnt,
                                         act, counters, counters + ivv::kShadeHead, off, (int)npix, (float)p.ds,
                                         tail_eps, sa, (float4*)out, stats, v->d_stats, v->num_sms, s);
      } else {
        ivv::launch_integrate_split_p<3>(V, c32, a, sa, mixed, stats, pin, pout, pblk, pcnt, act, counters,
                                         counters + ivv::kQueueHeadOff, v->d_stats, v->num_sms, s);
        ivv::launch_shade_composite_p<3>(V, c32, tf, p.supersample_k, (float)p.early_alpha, pin, pout, pblk, pcnt,
                                         act, counters, counters + ivv::kShadeHead, off, (int)npix, (float)p.ds,
                                         tail_eps, sa, (float4*)out, stats, v->d_stats, v->num_sms, s);
      }
    } else {
      ivv::DevCamera<float> cf = c32;
      if (V.P == 2)
        ivv::launch_integrate_p<2>(V, &cf, nullptr, tf, a, mixed, stats, pin, pout, pblk, pcnt, act, counters,
                                   counters + ivv::kQueueHeadOff, (float4*)out, v->d_stats, v->num_sms, s);
      else
        ivv::launch_integrate_p<3>(V, &cf, nullptr, tf, a, mixed, stats, pin, pout, pblk, pcnt, act, counters,
                                   counters + ivv::kQueueHeadOff, (float4*)out, v->d_stats, v->num_sms, s);
    }
  }
  if (p.flags & IVV_FLAG_TIMING) {
    IVV_CUDA(cudaEventRecord(v->ev[4], s));
    v->timed = true;
  }
  IVV_CUDA(cudaGetLastError());
  return IVV_OK;
}

}  // namespace

namespace ivv {
std::string& last_error_ref() { return g_err; }
ivv_status resolve_params_host(double diag, const ivv_render_params* in, ivv_render_params& p) {
  return resolve_params_diag(diag, in, p);
}
ivv_status frame_cameras(const ivv_camera* c, const ivv_render_params& p, int width, int height,
                         DevCamera<float>& c32, DevCamera<double>& c64) {
  Frame F;
  ivv_status st = make_frame(c, p, width, height, F);
  if (st != IVV_OK) return st;
  c32 = dev_camera<float>(F);
  c64 = dev_camera<double>(F);
  return IVV_OK;
}
}  // namespace ivv

extern "C" {

const char* ivv_last_error(void) { return g_err.c_str(); }

ivv_status ivv_create_volume(const ivv_block_desc* blocks, int n_blocks, int scalar_mode, void* stream,
                             ivv_volume** out) {
  if (!out) return fail(IVV_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  ivv_volume* v = new ivv_volume();
  std::string err;
  ivv_status st = ivv::prepare_volume(blocks, n_blocks, scalar_mode, v->hv, err);
  if (st != IVV_OK) {
    delete v;
    return fail(st, err);
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&v->device);
  if (e != cudaSuccess) {
    delete v;
    return cuda_fail(e, "cudaGetDevice");
  }
  e = cudaDeviceGetAttribute(&v->num_sms, cudaDevAttrMultiProcessorCount, v->device);
  if (e != cudaSuccess) {
    delete v;
    return cuda_fail(e, "cudaDeviceGetAttribute");
  }
  const ivv::HostVolume& hv = v->hv;
  std::vector<float> brk32(hv.brk.begin(), hv.brk.end());
  std::vector<float4> elem32(hv.elem.size() / 4), face32(hv.face_cp.size() / 4), org32(hv.elem_org.size() / 4);
  for (size_t i = 0; i < org32.size(); ++i)
    org32[i] = make_float4((float)hv.elem_org[4 * i], (float)hv.elem_org[4 * i + 1], (float)hv.elem_org[4 * i + 2], 0.f);
  for (size_t i = 0; i < elem32.size(); ++i)
    elem32[i] = make_float4((float)hv.elem[4 * i], (float)hv.elem[4 * i + 1], (float)hv.elem[4 * i + 2],
                            (float)hv.elem[4 * i + 3]);
  for (size_t i = 0; i < face32.size(); ++i)
    face32[i] = make_float4((float)hv.face_cp[4 * i], (float)hv.face_cp[4 * i + 1], (float)hv.face_cp[4 * i + 2], 0.f);
  const size_t nnn = (size_t)(hv.P + 1) * (hv.P + 1) * (hv.P + 1), rs = (size_t)ivv::rho_stride32(hv.P);
  std::vector<float> rho32((size_t)hv.n_elems() * rs, 0.f);
  for (size_t i = 0; i < hv.elem.size() / 4; ++i) rho32[(i / nnn) * rs + i % nnn] = (float)hv.elem[4 * i + 3];
  if ((st = upload(&v->d_blocks, hv.blocks.data(), hv.blocks.size(), s)) != IVV_OK ||
      (st = upload(&v->d_brk32, brk32.data(), brk32.size(), s)) != IVV_OK ||
      (st = upload(&v->d_brk64, hv.brk.data(), hv.brk.size(), s)) != IVV_OK ||
      (st = upload(&v->d_elem32, elem32.data(), elem32.size(), s)) != IVV_OK ||
      (st = upload(&v->d_elem64, (const ivv::Dbl4*)hv.elem.data(), hv.elem.size() / 4, s)) != IVV_OK ||
      (st = upload(&v->d_org32, org32.data(), org32.size(), s)) != IVV_OK ||
      (st = upload(&v->d_rho32, rho32.data(), rho32.size(), s)) != IVV_OK ||
      (st = upload(&v->d_org64, (const ivv::Dbl4*)hv.elem_org.data(), hv.elem_org.size() / 4, s)) != IVV_OK ||
      (st = upload(&v->d_face32, face32.data(), face32.size(), s)) != IVV_OK ||
      (st = upload(&v->d_face64, (const ivv::Dbl4*)hv.face_cp.data(), hv.face_cp.size() / 4, s)) != IVV_OK ||
      (st = upload(&v->d_faces, hv.faces.data(), hv.faces.size(), s)) != IVV_OK ||
      (st = upload(&v->d_faces64, hv.faces64.data(), hv.faces64.size(), s)) != IVV_OK ||
      (st = upload<float>(&v->d_tf_r, nullptr, 256, s)) != IVV_OK ||
      (st = upload<float4>(&v->d_tf_rgba, nullptr, 256, s)) != IVV_OK ||
      (st = upload<ivv::DevStats>(&v->d_stats, nullptr, 1, s)) != IVV_OK ||
      (st = upload<int>(&v->d_count, nullptr, 4, s)) != IVV_OK) {
    std::string m = g_err;
    free_volume(v);
    return fail(st, m);
  }
  if (!hv.disp.empty()) {
    std::vector<float4> disp32(hv.disp.size() / 4), dorg32(hv.disp_org.size() / 4);
    for (size_t i = 0; i < disp32.size(); ++i)
      disp32[i] = make_float4((float)hv.disp[4 * i], (float)hv.disp[4 * i + 1], (float)hv.disp[4 * i + 2], 0.f);
    for (size_t i = 0; i < dorg32.size(); ++i)
      dorg32[i] = make_float4((float)hv.disp_org[4 * i], (float)hv.disp_org[4 * i + 1], (float)hv.disp_org[4 * i + 2],
                              0.f);
    if ((st = upload(&v->d_disp32, disp32.data(), disp32.size(), s)) != IVV_OK ||
        (st = upload(&v->d_dorg32, dorg32.data(), dorg32.size(), s)) != IVV_OK ||
        (st = upload(&v->d_disp64, (const ivv::Dbl4*)hv.disp.data(), hv.disp.size() / 4, s)) != IVV_OK ||
        (st = upload(&v->d_dorg64, (const ivv::Dbl4*)hv.disp_org.data(), hv.disp_org.size() / 4, s)) != IVV_OK) {
      std::string m = g_err;
      free_volume(v);
      return fail(st, m);
    }
    // the host vectors die with this scope: the copies must be done
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      free_volume(v);
      return cuda_fail(e, "displacement upload");
    }
  }
  for (int i = 0; i <= IVV_N_STAGES && e == cudaSuccess; ++i) e = cudaEventCreate(&v->ev[i]);
  if (e != cudaSuccess) {
    free_volume(v);
    return cuda_fail(e, "cudaEventCreate");
  }
  e = cudaMemsetAsync(v->d_stats, 0, sizeof(ivv::DevStats), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    free_volume(v);
    return cuda_fail(e, "volume upload");
  }
  v->lo = hv.def_lo;
  v->hi = hv.def_hi;
  // per-block input normalisation of the guess network: control-point box
  for (int b = 0; b < n_blocks; ++b) {
    const ivv_block_desc& d = blocks[b];
    const size_t ncp = (size_t)d.n_cp[0] * d.n_cp[1] * d.n_cp[2];
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (size_t q = 0; q < ncp; ++q)
      for (int r = 0; r < 3; ++r) {
        lo[r] = std::min(lo[r], d.geom_cp[3 * q + r]);
        hi[r] = std::max(hi[r], d.geom_cp[3 * q + r]);
      }
    ivv::MlpNorm nm;
    double hmax = 0;
    for (int r = 0; r < 3; ++r) hmax = std::max(hmax, 0.5 * (hi[r] - lo[r]));
    for (int r = 0; r < 3; ++r) {
      nm.c[r] = (float)(0.5 * (lo[r] + hi[r]));
      const double hw = std::max(0.5 * (hi[r] - lo[r]), 1e-6 * hmax);
      nm.inv_h[r] = (float)(1.0 / (hw > 0 ? hw : 1.0));
    }
    v->norms.push_back(nm);
  }
  {
    const size_t np = (size_t)n_blocks * ivv::kMlpStride;
    if ((st = upload<float>(&v->d_theta, nullptr, np, s)) != IVV_OK ||
        (st = upload<float>(&v->d_adam_m, nullptr, np, s)) != IVV_OK ||
        (st = upload<float>(&v->d_adam_v, nullptr, np, s)) != IVV_OK ||
        (st = upload<__half>(&v->d_theta16, nullptr, np, s)) != IVV_OK ||
        (st = upload(&v->d_norms, v->norms.data(), v->norms.size(), s)) != IVV_OK) {
      std::string m = g_err;
      free_volume(v);
      return fail(st, m);
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      free_volume(v);
      return cuda_fail(e, "guess buffers");
    }
  }
  *out = v;
  return IVV_OK;
}

void ivv_destroy_volume(ivv_volume* vol) {
  if (!vol) return;
  cudaDeviceSynchronize();
  free_volume(vol);
}

ivv_status ivv_set_transfer_function(ivv_volume* v, int n, const float* r, const float* rgba, float sigma, float lo,
                                     float hi) {
  if (!v) return fail(IVV_ERR_INVALID_ARG, "volume is NULL");
  if (n < 2 || n > 256) return fail(IVV_ERR_INVALID_ARG, "n_knots must be in 2..256");
  if (!r || !rgba) return fail(IVV_ERR_INVALID_ARG, "NULL transfer function array");
  if (r[0] != 0.f || r[n - 1] != 1.f) return fail(IVV_ERR_INVALID_ARG, "r[0] must be 0 and r[n-1] must be 1");
  for (int i = 1; i < n; ++i)
    if (!(r[i] >= r[i - 1])) return fail(IVV_ERR_INVALID_ARG, "knots r must be ascending");
  for (int i = 0; i < 4 * n; ++i)
    if (!std::isfinite(rgba[i])) return fail(IVV_ERR_INVALID_ARG, "non-finite rgba");
  if (!(sigma >= 0) || !std::isfinite(sigma)) return fail(IVV_ERR_INVALID_ARG, "sigma must be non-negative");
  cudaError_t e = cudaMemcpy(v->d_tf_r, r, sizeof(float) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(v->d_tf_rgba, rgba, sizeof(float4) * n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "transfer function upload");
  v->tf_n = n;
  v->tf_r_host.assign(r, r + n);
  v->tf_rgba_host.assign(rgba, rgba + 4 * n);
  v->sigma = sigma;
  if (std::isfinite(lo) && std::isfinite(hi) && hi > lo) {
    v->lo = lo;
    v->hi = hi;
  } else {
    v->lo = v->hv.def_lo;
    v->hi = v->hv.def_hi;
  }
  v->tf_set = true;
  return IVV_OK;
}

ivv_status ivv_get_scalar_range(const ivv_volume* v, double* lo, double* hi) {
  if (!v || !lo || !hi) return fail(IVV_ERR_INVALID_ARG, "NULL argument");
  *lo = v->lo;
  *hi = v->hi;
  return IVV_OK;
}

ivv_status ivv_workspace_size(const ivv_volume* v, int width, int height, int precision, size_t* bytes) {
  if (!v || !bytes) return fail(IVV_ERR_INVALID_ARG, "NULL argument");
  if (width <= 0 || height <= 0) return fail(IVV_ERR_INVALID_ARG, "width and height must be positive");
  if ((long long)width * height > kMaxWindowPixels)
    return fail(IVV_ERR_INVALID_ARG, "window larger than 2^27 pixels");
  const bool fp64 = precision == IVV_PREC_FP64;
  *bytes = layout(v->hv.n_faces(), (size_t)width * height, fp64 ? sizeof(ivv::Dbl4) : sizeof(float4)).total;
  return IVV_OK;
}

ivv_status ivv_render(ivv_volume* v, const ivv_camera* cam, const ivv_render_params* params, int width, int height,
                      float* out_rgba, void* workspace, size_t workspace_bytes, void* stream) {
  return render_impl(v, cam, params, width, height, out_rgba, workspace, workspace_bytes, (cudaStream_t)stream);
}

ivv_status ivv_render_to_host(ivv_volume* v, const ivv_camera* cam, const ivv_render_params* params, int width,
                              int height, float* out_host, void* stream) {
  if (!v || !out_host) return fail(IVV_ERR_INVALID_ARG, "NULL argument");
  if (width <= 0 || height <= 0) return fail(IVV_ERR_INVALID_ARG, "width and height must be positive");
  const size_t bytes = sizeof(float4) * (size_t)width * height;
  cudaStream_t s = (cudaStream_t)stream;
  ivv_status st = ensure_own((void**)&v->own_out, &v->own_out_bytes, bytes, s);
  if (st != IVV_OK) return st;
  st = render_impl(v, cam, params, width, height, v->own_out, nullptr, 0, s);
  if (st != IVV_OK) return st;
  IVV_CUDA(cudaMemcpyAsync(out_host, v->own_out, bytes, cudaMemcpyDeviceToHost, s));
  IVV_CUDA(cudaStreamSynchronize(s));
  return IVV_OK;
}

ivv_status ivv_render_to_host_async(ivv_volume* v, const ivv_camera* cam, const ivv_render_params* params,
                                    int width, int height, float* out_host, void* stream) {
  if (!v || !out_host) return fail(IVV_ERR_INVALID_ARG, "NULL argument");
  if (width <= 0 || height <= 0) return fail(IVV_ERR_INVALID_ARG, "width and height must be positive");
  const size_t bytes = sizeof(float4) * (size_t)width * height;
  cudaStream_t s = (cudaStream_t)stream;
  if (!v->copy_stream) {
    IVV_CUDA(cudaStreamCreateWithFlags(&v->copy_stream, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
      IVV_CUDA(cudaEventCreateWithFlags(&v->ev_rendered[k], cudaEventDisableTiming));
      IVV_CUDA(cudaEventCreateWithFlags(&v->ev_copied[k], cudaEventDisableTiming));
      IVV_CUDA(cudaEventRecord(v->ev_copied[k], v->copy_stream));
    }
  }
  const int slot = v->next_slot;
  if (v->own_out2_bytes[slot] < bytes) {
    // the slot's earlier copy must be done before its image is reallocated
    IVV_CUDA(cudaStreamSynchronize(v->copy_stream));
    ivv_status st = ensure_own((void**)&v->own_out2[slot], &v->own_out2_bytes[slot], bytes, s);
    if (st != IVV_OK) return st;
  }
  // the slot's image is overwritten only after its previous copy finished
  IVV_CUDA(cudaStreamWaitEvent(s, v->ev_copied[slot], 0));
  ivv_status st = render_impl(v, cam, params, width, height, v->own_out2[slot], nullptr, 0, s);
  if (st != IVV_OK) return st;
  IVV_CUDA(cudaEventRecord(v->ev_rendered[slot], s));
  IVV_CUDA(cudaStreamWaitEvent(v->copy_stream, v->ev_rendered[slot], 0));
  IVV_CUDA(cudaMemcpyAsync(out_host, v->own_out2[slot], bytes, cudaMemcpyDeviceToHost, v->copy_stream));
  IVV_CUDA(cudaEventRecord(v->ev_copied[slot], v->copy_stream));
  v->next_slot = slot ^ 1;
  return IVV_OK;
}

ivv_status ivv_render_to_host_wait(ivv_volume* v) {
  if (!v) return fail(IVV_ERR_INVALID_ARG, "NULL argument");
  if (v->copy_stream) IVV_CUDA(cudaStreamSynchronize(v->copy_stream));
  return IVV_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- no-alloc
// Fixed scratch for ivv_render_noalloc: the per-frame workspace (fragment
// lists, pairs, queue, counters) of a small window lives in this file-scope
// device array instead of memory the caller or the library allocates.  Each
// GPU that loads the library holds it until the process exits.
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(12) << 20;   // 12 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array in the current device's context.  In
// host code the array's name only stands for it, so the address is looked up
// with that device current.  The lookup is repeated on every call (it is a
// table read once the module is loaded): a cached address would outlive a
// cudaDeviceReset or a re-created primary context.  The first call on a
// device may load the library's device code, so it belongs before any stream
// capture.
ivv_status noalloc_scratch(void** out) {
  void* ptr = nullptr;
  IVV_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
  *out = ptr;
  return IVV_OK;
}

}  // namespace

extern "C" {

ivv_status ivv_render_noalloc(ivv_volume* v, const ivv_camera* cam, const ivv_render_params* params, int width,
                              int height, float* out_rgba, void* stream) {
  if (!v) return fail(IVV_ERR_INVALID_ARG, "volume is NULL");
  if (width <= 0 || height <= 0) return fail(IVV_ERR_INVALID_ARG, "width and height must be positive");
  const int precision = params ? params->precision : IVV_PREC_FP32;
  if (params && params->method == IVV_METHOD_RF)
    return fail(IVV_ERR_UNSUPPORTED, "ivv_render_noalloc renders with the ODE method only (the RF method sizes its "
                                     "sample buffers from a read-back and allocates them)");
  const size_t need = layout(v->hv.n_faces(), (size_t)width * height,
                             precision == IVV_PREC_FP64 ? sizeof(ivv::Dbl4) : sizeof(float4)).total;
  if (need > kNoAllocScratchBytes)
    return fail(IVV_ERR_WORKSPACE, "window needs " + std::to_string(need) + " bytes of scratch; ivv_render_noalloc has " +
                                       std::to_string(kNoAllocScratchBytes) + " (use ivv_render for larger windows)");
  void* scratch = nullptr;
  ivv_status st = noalloc_scratch(&scratch);
  if (st != IVV_OK) return st;
  return render_impl(v, cam, params, width, height, out_rgba, scratch, kNoAllocScratchBytes, (cudaStream_t)stream,
                     true);
}

ivv_status ivv_render_pairs(ivv_volume* v, const ivv_camera* cam, const ivv_render_params* params, int width,
                            int height, int max_pairs, int* pair_count, float* pairs, int* pair_block, void* workspace,
                            size_t workspace_bytes, void* stream) {
  if (!v || !pair_count || !pairs || !pair_block) return fail(IVV_ERR_INVALID_ARG, "NULL argument");
  if (max_pairs < 1) return fail(IVV_ERR_INVALID_ARG, "max_pairs must be >= 1");
  ivv_render_params p;
  ivv_status st = resolve_params(v, params, p);
  if (st != IVV_OK) return st;
  if (p.precision == IVV_PREC_FP64) return fail(IVV_ERR_INVALID_ARG, "ivv_render_pairs supports FP32 and MIXED");
  Frame F;
  st = make_frame(cam, p, width, height, F);
  if (st != IVV_OK) return st;
  const size_t npix = (size_t)width * height;
  const WsLayout L = layout(v->hv.n_faces(), npix, sizeof(float4));
  cudaStream_t s = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  if (ws) {
    if (workspace_bytes < L.total) return fail(IVV_ERR_WORKSPACE, "workspace smaller than ivv_workspace_size");
    if (((uintptr_t)ws) % 256) return fail(IVV_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  } else {
    st = ensure_own(&v->own_ws, &v->own_ws_bytes, L.total, s);
    if (st != IVV_OK) return st;
    ws = (char*)v->own_ws;
  }
  v->last_stream = s;
  const int mp = std::min(max_pairs, v->lim_pairs);
  st = run_surface_pairs<float>(v, F, p, ws, L, mp, nullptr, s);
  if (st != IVV_OK) return st;
  ivv::launch_export_pairs((int)npix, max_pairs, false, ws + L.pair_in, ws + L.pair_out,
                           (const int*)(ws + L.pair_block), (const int*)(ws + L.pair_count), pair_count, pairs,
                           pair_block, s);
  IVV_CUDA(cudaGetLastError());
  return IVV_OK;
}

ivv_status ivv_eval_points(ivv_volume* v, int block, int n, const float* p, float* phi, float* jac, float* rho,
                           void* stream) {
  if (!v || (!p && n > 0)) return fail(IVV_ERR_INVALID_ARG, "NULL argument");
  if (block < 0 || block >= v->hv.n_blocks) return fail(IVV_ERR_INVALID_ARG, "block out of range");
  if (n < 0) return fail(IVV_ERR_INVALID_ARG, "n must be >= 0");
  ivv::launch_eval_points(dev_volume(v), block, n, p, phi, jac, rho, (cudaStream_t)stream);
  IVV_CUDA(cudaGetLastError());
  return IVV_OK;
}

// ---------------------------------------------------------------- guess
ivv_status ivv_train_guess(ivv_volume* v, const ivv_guess_train_params* in, float* final_loss, void* stream) {
  if (!v) return fail(IVV_ERR_INVALID_ARG, "volume is NULL");
  ivv_guess_train_params p;
  if (in) {
    p = *in;
  } else {
    p.samples_per_block = 1 << 20;
    p.epochs = 8;
    p.batch = 4096;
    p.lr = 3e-3f;
    p.seed = 1;
  }
  if (p.samples_per_block < 128 || p.epochs < 1 || p.batch < 128 || p.batch % 128 || !(p.lr > 0))
    return fail(IVV_ERR_INVALID_ARG, "bad training parameters");
  cudaStream_t s = (cudaStream_t)stream;
  const int S = p.samples_per_block;
  const int nb = v->hv.n_blocks;
  const int ctas = ivv::mlp_train_ctas(std::max(p.batch, std::min(S, 65536)));
  float4 *xs = nullptr, *ps = nullptr;
  float *partial = nullptr, *partial_loss = nullptr, *grad = nullptr, *loss = nullptr;
  auto cleanup = [&]() {
    void* q[] = {xs, ps, partial, partial_loss, grad, loss};
    for (void* x : q)
      if (x) cudaFree(x);
  };
  cudaError_t e = cudaMalloc(&xs, sizeof(float4) * S);
  if (e == cudaSuccess) e = cudaMalloc(&ps, sizeof(float4) * S);
  if (e == cudaSuccess) e = cudaMalloc(&partial, sizeof(float) * (size_t)ctas * ivv::kMlpParams);
  if (e == cudaSuccess) e = cudaMalloc(&partial_loss, sizeof(float) * ctas);
  if (e == cudaSuccess) e = cudaMalloc(&grad, sizeof(float) * ivv::kMlpParams);
  if (e == cudaSuccess) e = cudaMalloc(&loss, sizeof(float));
  if (e != cudaSuccess) {
    cleanup();
    return fail(IVV_ERR_OOM, std::string("training buffers: ") + cudaGetErrorString(e));
  }
  const ivv::DevVolume V = dev_volume(v);
  const long steps = (long)p.epochs * std::max(1, S / p.batch);
  for (int b = 0; b < nb; ++b) {
    // He-style initialisation, seeded per block
    std::mt19937_64 rng(p.seed * 1000003ull + (unsigned long long)b);
    std::normal_distribution<double> nd(0.0, 1.0);
    std::vector<float> th(ivv::kMlpParams, 0.f);
    for (int i = 0; i < ivv::kMlpH * 3; ++i) th[ivv::kOffW1 + i] = (float)(nd(rng) * std::sqrt(2.0 / 3.0));
    for (int i = 0; i < ivv::kMlpH * ivv::kMlpH; ++i) th[ivv::kOffW2 + i] = (float)(nd(rng) * std::sqrt(2.0 / ivv::kMlpH));
    for (int i = 0; i < 3 * ivv::kMlpH; ++i) th[ivv::kOffW3 + i] = (float)(nd(rng) * std::sqrt(1.0 / ivv::kMlpH));
    for (int i = 0; i < 3; ++i) th[ivv::kOffB3 + i] = 0.5f;
    float* tb = v->d_theta + (size_t)b * ivv::kMlpStride;
    float* mb = v->d_adam_m + (size_t)b * ivv::kMlpStride;
    float* vb = v->d_adam_v + (size_t)b * ivv::kMlpStride;
    __half* hb = v->d_theta16 + (size_t)b * ivv::kMlpStride;
    e = cudaMemcpyAsync(tb, th.data(), sizeof(float) * ivv::kMlpParams, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(mb, 0, sizeof(float) * ivv::kMlpParams, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(vb, 0, sizeof(float) * ivv::kMlpParams, s);
    if (e != cudaSuccess) {
      cleanup();
      return cuda_fail(e, "guess init");
    }
    ivv::launch_mlp_samples(V, v->norms[b], b, S, p.seed, xs, ps, s);
    for (long k = 1; k <= steps; ++k) {
      const int first = (int)(((k - 1) * (long)p.batch) % S);
      const double frac = (double)k / steps;
      const float lr = (float)(p.lr * (0.1 + 0.9 * 0.5 * (1.0 + std::cos(M_PI * frac))));
      e = ivv::launch_mlp_fwd_bwd(tb, xs, ps, S, first, p.batch, 1.f / p.batch, partial, partial_loss, s);
      if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "mlp_fwd_bwd");
      }
      ivv::launch_mlp_reduce(partial, partial_loss, ivv::mlp_train_ctas(p.batch), grad, loss, s);
      ivv::launch_mlp_adam(tb, mb, vb, grad, lr, (int)k, hb, s);
    }
    if (final_loss) {
      const int n = std::min(S, 65536);
      e = ivv::launch_mlp_fwd_bwd(tb, xs, ps, S, 0, n, 1.f / n, partial, partial_loss, s);
      if (e == cudaSuccess) {
        ivv::launch_mlp_reduce(partial, partial_loss, ivv::mlp_train_ctas(n), grad, loss, s);
        e = cudaMemcpyAsync(final_loss + b, loss, sizeof(float), cudaMemcpyDeviceToHost, s);
      }
      if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "final loss");
      }
    }
  }
  e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  cleanup();
  if (e != cudaSuccess) return cuda_fail(e, "training");
  v->guess_ready = true;
  return IVV_OK;
}

ivv_status ivv_guess_points(ivv_volume* v, int n, const float* g, const int* block_of, float* p_out, void* stream) {
  if (!v || n < 0 || (n > 0 && (!g || !block_of || !p_out))) return fail(IVV_ERR_INVALID_ARG, "bad argument");
  if (!v->guess_ready) return fail(IVV_ERR_INVALID_ARG, "the guess network is neither trained nor set");
  if (((uintptr_t)g) % 16 || ((uintptr_t)p_out) % 16) return fail(IVV_ERR_INVALID_ARG, "g and p_out must be 16-byte aligned");
  if (n == 0) return IVV_OK;
  ivv::launch_mlp_infer(v->d_theta16, v->d_norms, (const float4*)g, block_of, nullptr, n, (float4*)p_out, v->d_stats,
                        v->num_sms, (cudaStream_t)stream);
  IVV_CUDA(cudaGetLastError());
  return IVV_OK;
}

ivv_status ivv_invert_points(ivv_volume* v, int n, const float* g, const int* block_of, int guess, float tol,
                             float* p_out, int* iters, void* stream) {
  if (!v || n < 0 || (n > 0 && (!g || !block_of || !p_out))) return fail(IVV_ERR_INVALID_ARG, "bad argument");
  if (guess != IVV_GUESS_CENTER && guess != IVV_GUESS_MLP) return fail(IVV_ERR_INVALID_ARG, "bad guess mode");
  if (guess == IVV_GUESS_MLP && !v->guess_ready) return fail(IVV_ERR_INVALID_ARG, "the guess network is not trained");
  if (!(tol > 0)) return fail(IVV_ERR_INVALID_ARG, "tol must be positive");
  if (((uintptr_t)g) % 16 || ((uintptr_t)p_out) % 16) return fail(IVV_ERR_INVALID_ARG, "g and p_out must be 16-byte aligned");
  if (n == 0) return IVV_OK;
  cudaStream_t s = (cudaStream_t)stream;
  IVV_CUDA(cudaMemcpyAsync(v->d_count, &n, sizeof(int), cudaMemcpyHostToDevice, s));
  if (guess == IVV_GUESS_MLP)
    ivv::launch_mlp_infer(v->d_theta16, v->d_norms, (const float4*)g, block_of, nullptr, n, (float4*)p_out,
                          v->d_stats, v->num_sms, s);
  else
    ivv::launch_fill_center((float4*)p_out, n, s);
  ivv::DevCamera<float> cam{};
  cam.H = 1;
  cam.ortho = 1;
  ivv::launch_rf_newton(dev_volume(v), cam, 0.f, tol, v->d_count, (const float4*)g, block_of, (const float4*)p_out,
                        nullptr, (float4*)p_out, iters, v->d_stats, false, false, v->num_sms, s);
  IVV_CUDA(cudaGetLastError());
  return IVV_OK;
}

ivv_status ivv_guess_loss_grad(ivv_volume* v, int block, int n, const float* x_hat, const float* p, float* grad,
                               float* loss, void* stream) {
  if (!v || !x_hat || !p || !grad || !loss || n <= 0) return fail(IVV_ERR_INVALID_ARG, "bad argument");
  if (block < 0 || block >= v->hv.n_blocks) return fail(IVV_ERR_INVALID_ARG, "block out of range");
  cudaStream_t s = (cudaStream_t)stream;
  const int ctas = ivv::mlp_train_ctas(n);
  float *partial = nullptr, *partial_loss = nullptr, *dgrad = nullptr, *dloss = nullptr;
  cudaError_t e = cudaMalloc(&partial, sizeof(float) * (size_t)ctas * ivv::kMlpParams);
  if (e == cudaSuccess) e = cudaMalloc(&partial_loss, sizeof(float) * ctas);
  if (e == cudaSuccess) e = cudaMalloc(&dgrad, sizeof(float) * ivv::kMlpParams);
  if (e == cudaSuccess) e = cudaMalloc(&dloss, sizeof(float));
  if (e == cudaSuccess)
    e = ivv::launch_mlp_fwd_bwd(v->d_theta + (size_t)block * ivv::kMlpStride, (const float4*)x_hat, (const float4*)p,
                                n, 0, n, 1.f / n, partial, partial_loss, s);
  if (e == cudaSuccess) {
    ivv::launch_mlp_reduce(partial, partial_loss, ctas, dgrad, dloss, s);
    e = cudaMemcpyAsync(grad, dgrad, sizeof(float) * ivv::kMlpParams, cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(loss, dloss, sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  void* q[] = {partial, partial_loss, dgrad, dloss};
  for (void* x : q)
    if (x) cudaFree(x);
  if (e != cudaSuccess) return cuda_fail(e, "guess loss/grad");
  return IVV_OK;
}

ivv_status ivv_get_guess_weights(ivv_volume* v, int block, float* params, float* c, float* inv_h) {
  if (!v) return fail(IVV_ERR_INVALID_ARG, "volume is NULL");
  if (block < 0 || block >= v->hv.n_blocks) return fail(IVV_ERR_INVALID_ARG, "block out of range");
  if (params)
    IVV_CUDA(cudaMemcpy(params, v->d_theta + (size_t)block * ivv::kMlpStride, sizeof(float) * ivv::kMlpParams,
                        cudaMemcpyDeviceToHost));
  for (int r = 0; r < 3; ++r) {
    if (c) c[r] = v->norms[block].c[r];
    if (inv_h) inv_h[r] = v->norms[block].inv_h[r];
  }
  return IVV_OK;
}

ivv_status ivv_set_guess_weights(ivv_volume* v, int block, const float* params) {
  if (!v || !params) return fail(IVV_ERR_INVALID_ARG, "NULL argument");
  if (block < 0 || block >= v->hv.n_blocks) return fail(IVV_ERR_INVALID_ARG, "block out of range");
  float* tb = v->d_theta + (size_t)block * ivv::kMlpStride;
  IVV_CUDA(cudaMemcpy(tb, params, sizeof(float) * ivv::kMlpParams, cudaMemcpyHostToDevice));
  ivv::launch_mlp_to_half(tb, v->d_theta16 + (size_t)block * ivv::kMlpStride, ivv::kMlpParams, nullptr);
  IVV_CUDA(cudaDeviceSynchronize());
  v->guess_ready = true;
  return IVV_OK;
}

ivv_status ivv_host_eval(const ivv_block_desc* blocks, int n_blocks, int scalar_mode, int block, int n,
                         const double* p, double* phi, double* jac, double* rho) {
  if (n < 0 || (n > 0 && !p)) return fail(IVV_ERR_INVALID_ARG, "bad points");
  ivv::HostVolume hv;
  std::string err;
  ivv_status st = ivv::prepare_volume(blocks, n_blocks, scalar_mode, hv, err);
  if (st != IVV_OK) return fail(st, err);
  if (block < 0 || block >= hv.n_blocks) return fail(IVV_ERR_INVALID_ARG, "block out of range");
  for (int i = 0; i < n; ++i) {
    double f[3], J[3][3], rc;
    ivv::host_eval(hv, block, p + 3 * i, f, J, &rc);
    if (phi)
      for (int r = 0; r < 3; ++r) phi[3 * i + r] = f[r];
    if (jac)
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) jac[9 * i + 3 * r + c] = J[r][c];
    if (rho) rho[i] = ivv::host_scalar(hv, block, p + 3 * i, J, rc);
  }
  return IVV_OK;
}

ivv_status ivv_get_stage_times(ivv_volume* v, float* ms) {
  if (!v || !ms) return fail(IVV_ERR_INVALID_ARG, "NULL argument");
  if (!v->timed) return fail(IVV_ERR_INVALID_ARG, "no render with IVV_FLAG_TIMING was made");
  IVV_CUDA(cudaEventSynchronize(v->ev[IVV_N_STAGES]));
  for (int i = 0; i < IVV_N_STAGES; ++i) IVV_CUDA(cudaEventElapsedTime(&ms[i], v->ev[i], v->ev[i + 1]));
  return IVV_OK;
}

ivv_status ivv_get_stats(ivv_volume* v, ivv_stats* out) {
  if (!v || !out) return fail(IVV_ERR_INVALID_ARG, "NULL argument");
  IVV_CUDA(cudaStreamSynchronize(v->last_stream));
  ivv::DevStats d;
  IVV_CUDA(cudaMemcpy(&d, v->d_stats, sizeof(d), cudaMemcpyDeviceToHost));
  ivv::stats_to_public(d, out);
  return IVV_OK;
}

}  // extern "C"

namespace ivv {
void stats_to_public(const DevStats& d, ivv_stats* out) {
  out->rays = d.rays;
  out->pairs = d.pairs;
  out->fragments = d.fragments;
  out->samples = d.samples;
  out->rk_steps = d.rk_steps;
  out->rk_rejects = d.rk_rejects;
  out->rhs_evals = d.rhs_evals;
  out->isect_newton = d.isect_newton;
  out->isect_tests = d.isect_tests;
  out->fp64_solves = d.fp64_solves;
  out->abuf_overflow = d.abuf_overflow;
  out->pair_overflow = d.pair_overflow;
  out->unmatched = d.unmatched;
  out->step_cap = d.step_cap;
  out->rf_newton_iters = d.rf_newton_iters;
  out->rf_unconverged = d.rf_unconverged;
  out->isect_items = d.isect_items;
  out->isect_split = d.isect_split;
  out->rho_evals = d.rho_evals;
  out->entry_shrinks = d.entry_shrinks;
  out->entry_newton = d.entry_newton;
  out->async_timeouts = d.async_timeouts;
  float f;
  std::memcpy(&f, &d.max_delta_p_bits, sizeof(f));
  out->max_delta_p = f;
}
}  // namespace ivv

extern "C" {

ivv_status ivv_reset_stats(ivv_volume* v) {
  if (!v) return fail(IVV_ERR_INVALID_ARG, "volume is NULL");
  IVV_CUDA(cudaMemsetAsync(v->d_stats, 0, sizeof(ivv::DevStats), v->last_stream));
  IVV_CUDA(cudaStreamSynchronize(v->last_stream));
  v->seen_overflow = v->seen_cap = 0;
  return IVV_OK;
}

ivv_status ivv_set_limits(ivv_volume* v, const ivv_limits* in) {
  if (!v) return fail(IVV_ERR_INVALID_ARG, "volume is NULL");
  ivv_limits l = {ivv::kMaxFrags, ivv::kMaxPairs, ivv::kItemsPerPixel, 200000, 16};
  if (in) l = *in;
  if (l.max_frags < 1 || l.max_frags > ivv::kMaxFrags) return fail(IVV_ERR_INVALID_ARG, "max_frags must be in 1..32");
  if (l.max_pairs < 1 || l.max_pairs > ivv::kMaxPairs) return fail(IVV_ERR_INVALID_ARG, "max_pairs must be in 1..16");
  if (l.items_per_pixel < 1 || l.items_per_pixel > ivv::kItemsPerPixel)
    return fail(IVV_ERR_INVALID_ARG, "items_per_pixel must be in 1..16");
  if (l.max_rk_steps < 1) return fail(IVV_ERR_INVALID_ARG, "max_rk_steps must be >= 1");
  if (l.max_newton < 1 || l.max_newton > 64) return fail(IVV_ERR_INVALID_ARG, "max_newton must be in 1..64");
  v->lim_frags = l.max_frags;
  v->lim_pairs = l.max_pairs;
  v->lim_items = l.items_per_pixel;
  v->lim_rk_steps = l.max_rk_steps;
  v->lim_newton = l.max_newton;
  return IVV_OK;
}

ivv_status ivv_get_limits(const ivv_volume* v, ivv_limits* out) {
  if (!v || !out) return fail(IVV_ERR_INVALID_ARG, "volume or output is NULL");
  out->max_frags = v->lim_frags;
  out->max_pairs = v->lim_pairs;
  out->items_per_pixel = v->lim_items;
  out->max_rk_steps = v->lim_rk_steps;
  out->max_newton = v->lim_newton;
  return IVV_OK;
}

ivv_status ivv_check_frame(ivv_volume* v) {
  if (!v) return fail(IVV_ERR_INVALID_ARG, "volume is NULL");
  IVV_CUDA(cudaStreamSynchronize(v->last_stream));
  ivv::DevStats d;
  IVV_CUDA(cudaMemcpy(&d, v->d_stats, sizeof(d), cudaMemcpyDeviceToHost));
  if (d.async_timeouts)
    return fail(IVV_ERR_CUDA, std::to_string(d.async_timeouts) + " bounded waits for the tensor cores gave up");
  const unsigned long long ov = d.abuf_overflow + d.pair_overflow, cap = d.step_cap + d.rf_unconverged;
  const unsigned long long new_ov = ov - std::min(ov, v->seen_overflow), new_cap = cap - std::min(cap, v->seen_cap);
  v->seen_overflow = ov;
  v->seen_cap = cap;
  if (new_ov)
    return fail(IVV_ERR_ABUF_OVERFLOW, std::to_string(new_ov) + " fragments, candidates or pairs dropped (" +
                                           std::to_string(d.abuf_overflow) + " fragment/candidate and " +
                                           std::to_string(d.pair_overflow) + " pair drops since the last reset)");
  if (new_cap)
    return fail(IVV_ERR_NONCONVERGED, std::to_string(new_cap) + " capped iterations (" + std::to_string(d.step_cap) +
                                          " pairs at the RK step cap, " + std::to_string(d.rf_unconverged) +
                                          " RF samples off tolerance since the last reset)");
  return IVV_OK;
}

ivv_status ivv_volume_info(const ivv_volume* v, int* n_blocks, int* n_elements, int* n_faces, int* degree) {
  if (!v) return fail(IVV_ERR_INVALID_ARG, "volume is NULL");
  if (n_blocks) *n_blocks = v->hv.n_blocks;
  if (n_elements) *n_elements = v->hv.n_elems();
  if (n_faces) *n_faces = v->hv.n_faces();
  if (degree) *degree = v->hv.P;
  return IVV_OK;
}

}  // extern "C"
