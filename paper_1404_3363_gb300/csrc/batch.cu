// Batched rendering (ivv_batch_*): many views of several volumes, of uneven
// image sizes, rendered by one launch per stage and replayed from a captured
// CUDA graph.
//
// Creation merges every distinct volume of the batch into one device pool --
// block table, Bezier elements, face patches and breakpoints concatenated,
// with the block table's element and breakpoint offsets and the face
// records' block ids rebased -- so that fragments, pairs and the integrator
// address geometry through global block ids alone.  Per request the library
// keeps a record (cameras, pixel offset, face range, screen-box offset,
// volume diagonal, sample distance, output image) and a transfer-function
// slot; the pixel space of the batch is the requests' images one after the
// other.  The stages are K0 over every (request, face), K2 over every tile of
// every request, K4 over every pixel and one persistent K5 over a queue that
// spans all requests.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ivv_device.cuh"
#include "ivv_internal.h"
#include "volume.h"

namespace ivv {
std::string& last_error_ref();
ivv_status resolve_params_host(double diag, const ivv_render_params* in, ivv_render_params& p);
ivv_status frame_cameras(const ivv_camera* c, const ivv_render_params& p, int width, int height,
                         DevCamera<float>& c32, DevCamera<double>& c64);
void stats_to_public(const DevStats& d, ivv_stats* out);
}  // namespace ivv

namespace {

ivv_status bfail(ivv_status s, const std::string& msg) {
  ivv::last_error_ref() = msg;
  return s;
}

ivv_status bcuda(cudaError_t e, const char* what) {
  return bfail(IVV_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define IVV_BCUDA(call)                                   \
  do {                                                    \
    cudaError_t e__ = (call);                             \
    if (e__ != cudaSuccess) return bcuda(e__, #call);     \
  } while (0)

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// Tile shapes with a tile table: the K2a warp tiles the batch kernels are
// built for (the first kNumWarpShapes), then K4's 16x16 pixel order.
constexpr int kNumWarpShapes = 3;
constexpr int kNumShapes = 4;
constexpr int kShapes[kNumShapes][2] = {{8, 4}, {4, 8}, {16, 2}, {16, 16}};
constexpr int kShape16 = 3;
int shape_index(int tw, int th) {
  for (int i = 0; i < kNumWarpShapes; ++i)
    if (kShapes[i][0] == tw && kShapes[i][1] == th) return i;
  return -1;
}

struct BatchLayout {
  size_t boxes, gboxes, items, slow, frag_tp, frag_meta, frag_count, pair_in, pair_out, pair_block, pair_count, active,
      counters, total;
};

BatchLayout batch_layout(size_t n_boxes, size_t n_gboxes, size_t npix) {
  BatchLayout L;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o += a256(bytes); return at; };
  L.boxes = take(sizeof(int4) * std::max<size_t>(n_boxes, 1));
  L.gboxes = take(sizeof(int4) * std::max<size_t>(n_gboxes, 1));
  L.items = take(sizeof(int2) * ivv::kItemsPerPixel * npix);
  L.slow = take(sizeof(int) * ivv::kItemsPerPixel * npix);
  L.frag_tp = take(sizeof(float4) * ivv::kMaxFrags * npix);
  L.frag_meta = take(sizeof(unsigned) * ivv::kMaxFrags * npix);
  L.frag_count = take(sizeof(int) * npix);
  L.pair_in = take(sizeof(float4) * ivv::kMaxPairs * npix);
  L.pair_out = take(sizeof(float4) * ivv::kMaxPairs * npix);
  L.pair_block = take(sizeof(int) * ivv::kMaxPairs * npix);
  L.pair_count = take(sizeof(int) * npix);
  L.active = take(sizeof(int) * npix);
  L.counters = take(ivv::kCountersBytes);
  L.total = o;
  return L;
}

}  // namespace

struct ivv_batch {
  int device = 0, num_sms = 1, P = 3;
  ivv_render_params p{};
  int nreq = 0;
  long long npix = 0;
  std::vector<ivv::DevRequest> hreq;
  std::vector<ivv::BlockInfo> blocks;
  int n_faces = 0, max_faces = 0, n_boxes = 0, n_gboxes = 0;
  int tiles[kNumShapes] = {};               // tiles of the batch per shape
  // pool
  ivv::BlockInfo* d_blocks = nullptr;
  float* d_brk32 = nullptr;
  double* d_brk64 = nullptr;
  float4* d_elem32 = nullptr;
  float4* d_org32 = nullptr;
  float4* d_face32 = nullptr;
  ivv::Dbl4* d_face64 = nullptr;
  ivv::FaceMeta* d_faces = nullptr;
  ivv::FaceMeta64* d_faces64 = nullptr;
  // tables
  ivv::DevRequest* d_req = nullptr;
  int* d_pix0 = nullptr;
  int* d_tile0[kNumShapes] = {};
  ivv::DevTFSlot* d_tf = nullptr;
  ivv::DevStats* d_stats = nullptr;
  // workspace
  BatchLayout L{};
  char* ws = nullptr;
  // sample buffer of the split integration (sp_cap samples; NULL: fused K5)
  float4* d_sp = nullptr;
  long long sp_cap = 0;
  bool sp_sized = false;
  // launch shapes, graph, timing
  ivv_batch_tuning tune{8, 4, 4, 8};
  int k5_max_ctas[2] = {1, 1};              // occupancy limit without / with statistics
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev[IVV_N_STAGES + 1] = {};
  bool timed = false;
  cudaStream_t last_stream = nullptr;
};

namespace {

void drop_graph(ivv_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

void free_batch(ivv_batch* b) {
  if (!b) return;
  drop_graph(b);
  void* ptrs[] = {b->d_blocks, b->d_brk32, b->d_brk64, b->d_elem32, b->d_org32, b->d_face32, b->d_face64,
                  b->d_faces, b->d_faces64, b->d_req, b->d_pix0, b->d_tile0[0], b->d_tile0[1], b->d_tile0[2],
                  b->d_tile0[3], b->d_tf, b->d_stats, b->ws, b->d_sp};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (cudaEvent_t e : b->ev)
    if (e) cudaEventDestroy(e);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
}

template <typename T>
ivv_status balloc(T** dst, size_t n) {
  cudaError_t e = cudaMalloc((void**)dst, sizeof(T) * std::max<size_t>(n, 1));
  if (e != cudaSuccess) return bfail(IVV_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  return IVV_OK;
}

// The request's transfer function as a device slot (knots, colours and the
// segment lookup table of tf_eval).
ivv_status make_tf_slot(const ivv_request& r, ivv::DevTFSlot& slot) {
  const ivv_volume* v = r.volume;
  int n;
  const float *tr, *trgba;
  float sigma;
  double lo, hi;
  if (r.tf_r) {
    n = r.tf_n;
    tr = r.tf_r;
    trgba = r.tf_rgba;
    sigma = r.tf_sigma;
    lo = r.scalar_lo;
    hi = r.scalar_hi;
    if (!(std::isfinite(lo) && std::isfinite(hi) && hi > lo)) {
      lo = v->hv.def_lo;
      hi = v->hv.def_hi;
    }
    if (!trgba) return bfail(IVV_ERR_INVALID_ARG, "request tf_rgba is NULL");
  } else {
    if (!v->tf_set) return bfail(IVV_ERR_INVALID_ARG, "request has no transfer function and its volume has none");
    n = v->tf_n;
    tr = v->tf_r_host.data();
    trgba = v->tf_rgba_host.data();
    sigma = v->sigma;
    lo = v->lo;
    hi = v->hi;
  }
  if (n < 2 || n > ivv::kBatchTfMax) return bfail(IVV_ERR_INVALID_ARG, "request tf_n must be in 2..IVV_BATCH_TF_MAX");
  if (tr[0] != 0.f || tr[n - 1] != 1.f) return bfail(IVV_ERR_INVALID_ARG, "tf_r[0] must be 0 and tf_r[n-1] 1");
  for (int i = 1; i < n; ++i)
    if (!(tr[i] >= tr[i - 1])) return bfail(IVV_ERR_INVALID_ARG, "tf_r must be ascending");
  for (int i = 0; i < 4 * n; ++i)
    if (!std::isfinite(trgba[i])) return bfail(IVV_ERR_INVALID_ARG, "non-finite tf_rgba");
  if (!(sigma >= 0) || !std::isfinite(sigma)) return bfail(IVV_ERR_INVALID_ARG, "tf_sigma must be non-negative");
  std::memset(&slot, 0, sizeof(slot));
  for (int i = 0; i < n; ++i) {
    slot.r[i] = tr[i];
    slot.rgba[i] = make_float4(trgba[4 * i], trgba[4 * i + 1], trgba[4 * i + 2], trgba[4 * i + 3]);
  }
  for (int i = 0; i < ivv::kTfTable; ++i) {
    const float x = (float)i / (float)ivv::kTfTable;
    int k = 0;
    while (k < n - 2 && slot.r[k + 1] <= x) ++k;
    slot.seg[i] = (unsigned char)k;
  }
  slot.n = n;
  slot.sigma = sigma;
  slot.lo = (float)lo;
  slot.inv_range = (float)(1.0 / (hi - lo));
  return IVV_OK;
}

ivv::DevVolume pool_volume(const ivv_batch* b) {
  ivv::DevVolume V{};
  V.P = b->P;
  V.mode = -1;                       // per block (BlockInfo::mode)
  V.n_blocks = (int)b->blocks.size();
  V.n_faces = b->n_faces;
  V.blocks = b->d_blocks;
  V.brk32 = b->d_brk32;
  V.brk64 = b->d_brk64;
  V.elem32 = b->d_elem32;
  V.elem64 = nullptr;
  V.org32 = b->d_org32;
  V.rho32 = nullptr;
  V.org64 = nullptr;
  V.face32 = b->d_face32;
  V.face64 = b->d_face64;
  V.faces = b->d_faces;
  V.faces64 = b->d_faces64;
  V.diag = 0.f;
  V.max_frags = ivv::kMaxFrags;
  V.max_newton = 16;
  return V;
}

ivv::BatchArgs batch_args(const ivv_batch* b) {
  ivv::BatchArgs a;
  a.req = b->d_req;
  a.pix0 = b->d_pix0;
  a.tile0 = b->d_tile0[shape_index(b->tune.tile_w, b->tune.tile_h)];
  a.tile16 = b->d_tile0[kShape16];
  a.tf = b->d_tf;
  a.nreq = b->nreq;
  return a;
}

// Every stage of one batch render on stream s.  measure: stop after the
// sample counts and their scan (the total lands in counters[2]).
ivv_status enqueue(ivv_batch* b, bool stats, bool timing, cudaStream_t s, bool measure = false) {
  const ivv::DevVolume V = pool_volume(b);
  const ivv::BatchArgs ba = batch_args(b);
  const BatchLayout& L = b->L;
  char* ws = b->ws;
  const int npix = (int)b->npix;
  const bool mixed = b->p.precision == IVV_PREC_MIXED;
  IVV_BCUDA(cudaMemsetAsync(ws + L.counters, 0, ivv::kCountersBytes, s));
  ivv::SurfaceWs sw;
  sw.boxes = (int4*)(ws + L.boxes);
  sw.gboxes = (int4*)(ws + L.gboxes);
  sw.items = (int2*)(ws + L.items);
  sw.slow = (int*)(ws + L.slow);
  sw.cap = (int)std::min<long long>((long long)ivv::kItemsPerPixel * b->npix, 0x7fffffffll);
  sw.n_items = (int*)(ws + L.counters) + ivv::kItemCounter;
  sw.frag_tp = ws + L.frag_tp;
  sw.frag_meta = (unsigned*)(ws + L.frag_meta);
  sw.frag_count = (int*)(ws + L.frag_count);
  if (timing) IVV_BCUDA(cudaEventRecord(b->ev[0], s));
  ivv::launch_batch_face_project(V, ba, b->max_faces, sw, s);
  if (timing) IVV_BCUDA(cudaEventRecord(b->ev[1], s));
  const int si = shape_index(b->tune.tile_w, b->tune.tile_h);
  if (si < 0 || !ivv::launch_batch_intersect(V, ba, b->tiles[si], b->tune.tile_w, b->tune.tile_h, mixed, stats, sw,
                                             (size_t)npix, b->d_stats, b->num_sms, s))
    return bfail(IVV_ERR_INVALID_ARG, "unsupported K2 tile shape");
  if (timing) IVV_BCUDA(cudaEventRecord(b->ev[2], s));
  ivv::launch_batch_pair(ba, b->tiles[kShape16], npix, (const float4*)(ws + L.frag_tp), (const unsigned*)(ws + L.frag_meta),
                         (const int*)(ws + L.frag_count), (float4*)(ws + L.pair_in), (float4*)(ws + L.pair_out),
                         (int*)(ws + L.pair_block), (int*)(ws + L.pair_count), (int*)(ws + L.active),
                         (int*)(ws + L.counters), b->d_stats, s);
  if (timing) IVV_BCUDA(cudaEventRecord(b->ev[3], s));
  int* counters = (int*)(ws + L.counters);
  int* cnt = (int*)(ws + L.frag_count);            // fragment lists are dead after stage 2
  int* off = (int*)(ws + L.frag_meta);
  if (measure) {
    ivv::launch_batch_count(ba, (const float4*)(ws + L.pair_in), (const float4*)(ws + L.pair_out),
                            (const int*)(ws + L.pair_count), (const int*)(ws + L.active), counters, npix, cnt,
                            b->num_sms, s);
    ivv::launch_rf_scan(cnt, counters, npix, off, off + npix, 0x7fffffff, counters + 2, s);
    IVV_BCUDA(cudaGetLastError());
    return IVV_OK;
  }
  ivv::IntegrateArgs a;
  a.rk_tol = (float)b->p.rk_tol;
  a.ds = 0.f;                        // per request
  a.c = (float)b->p.c;
  a.early_alpha = (float)b->p.early_alpha;
  a.K = b->p.supersample_k;
  a.max_steps = 200000;
  a.max_step_samples = b->tune.step_samples;
  a.npix = npix;
  const int cps = std::min(b->tune.k5_ctas_per_sm, b->k5_max_ctas[stats ? 1 : 0]);
  int grid = b->num_sms * std::max(cps, 1);
  grid = std::min(grid, std::max(1, (npix + 127) / 128));
  if (b->d_sp)
    ivv::launch_batch_split(V, ba, a, mixed, stats, (const float4*)(ws + L.pair_in), (const float4*)(ws + L.pair_out),
                            (const int*)(ws + L.pair_block), (const int*)(ws + L.pair_count),
                            (const int*)(ws + L.active), counters, off, cnt, off + npix, b->d_sp, (int)b->sp_cap,
                            (int*)(ws + L.slow), grid, b->num_sms, b->d_stats, s);
  else
    ivv::launch_batch_integrate(V, ba, a, mixed, stats, (const float4*)(ws + L.pair_in),
                                (const float4*)(ws + L.pair_out), (const int*)(ws + L.pair_block),
                                (const int*)(ws + L.pair_count), (const int*)(ws + L.active), counters,
                                counters + ivv::kQueueHeadOff, b->d_stats, grid, s);
  if (timing) {
    IVV_BCUDA(cudaEventRecord(b->ev[4], s));
    b->timed = true;
  }
  IVV_BCUDA(cudaGetLastError());
  return IVV_OK;
}

// The split integration's sample buffer, sized once from the samples of the
// batch as it is (stages 1-2 and the counts run eagerly on s; the samples of
// later camera changes may differ: pixels beyond the buffer are rendered by
// the fused integrator).  Without room for it, stage 3 stays fused.
ivv_status ensure_samples(ivv_batch* b, cudaStream_t s) {
  if (b->sp_sized) return IVV_OK;
  ivv::DevStats saved;                 // the measuring pass leaves the statistics as they were
  IVV_BCUDA(cudaMemcpyAsync(&saved, b->d_stats, sizeof(saved), cudaMemcpyDeviceToHost, s));
  const ivv_status st = enqueue(b, false, false, s, true);
  if (st != IVV_OK) return st;
  int total[2] = {0, 0};               // the sample total and its excess over INT_MAX
  IVV_BCUDA(cudaMemcpyAsync(total, (int*)(b->ws + b->L.counters) + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  IVV_BCUDA(cudaMemcpyAsync(b->d_stats, &saved, sizeof(saved), cudaMemcpyHostToDevice, s));
  IVV_BCUDA(cudaStreamSynchronize(s));
  const long long cap = std::min<long long>((long long)total[0] + total[0] / 4 + 4096, 0x7fffffffll);
  if (total[1] == 0 && cudaMalloc((void**)&b->d_sp, sizeof(float4) * (size_t)cap) == cudaSuccess) {
    b->sp_cap = cap;
  } else {
    cudaGetLastError();
    b->d_sp = nullptr;
    b->sp_cap = 0;
  }
  b->sp_sized = true;
  return IVV_OK;
}

ivv_status capture(ivv_batch* b) {
  drop_graph(b);
  IVV_BCUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  const ivv_status st = enqueue(b, false, false, b->cap_stream);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
  if (st != IVV_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return bcuda(e, "cudaStreamEndCapture");
  b->graph = g;
  IVV_BCUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
  return IVV_OK;
}

bool tuning_ok(const ivv_batch_tuning& t) {
  return shape_index(t.tile_w, t.tile_h) >= 0 && t.k5_ctas_per_sm >= 1 && t.k5_ctas_per_sm <= 4 &&
         (t.step_samples == 4 || t.step_samples == 8 || t.step_samples == 16);
}

}  // namespace

extern "C" {

ivv_status ivv_batch_create(const ivv_request* req, int n, const ivv_render_params* params, void* stream,
                            ivv_batch** out) {
  if (!out) return bfail(IVV_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!req) return bfail(IVV_ERR_INVALID_ARG, "requests is NULL");
  if (n < 1 || n > IVV_BATCH_MAX_REQUESTS) return bfail(IVV_ERR_INVALID_ARG, "n must be in 1..IVV_BATCH_MAX_REQUESTS");
  for (int i = 0; i < n; ++i) {
    if (!req[i].volume) return bfail(IVV_ERR_INVALID_ARG, "request volume is NULL");
    if (!req[i].out_rgba) return bfail(IVV_ERR_INVALID_ARG, "request out_rgba is NULL");
    if (((uintptr_t)req[i].out_rgba) % 16) return bfail(IVV_ERR_INVALID_ARG, "request out_rgba must be 16-byte aligned");
    if (req[i].width <= 0 || req[i].height <= 0) return bfail(IVV_ERR_INVALID_ARG, "request size must be positive");
    if (req[i].volume->hv.P != req[0].volume->hv.P)
      return bfail(IVV_ERR_UNSUPPORTED, "the volumes of a batch must share one common degree P");
    if (req[i].volume->hv.any_singular)
      return bfail(IVV_ERR_UNSUPPORTED, "batches take volumes without singular faces (render those with ivv_render)");
    if (req[i].volume->hv.mode == IVV_SCALAR_VONMISES)
      return bfail(IVV_ERR_UNSUPPORTED, "batches do not take von Mises volumes (render those with ivv_render)");
  }
  // shared parameters (diag 1: ds is resolved per request below)
  ivv_render_params p;
  ivv_status st = ivv::resolve_params_host(1.0, params, p);
  if (st != IVV_OK) return st;
  const bool ds_given = params && params->ds > 0;
  if (p.method != IVV_METHOD_ODE) return bfail(IVV_ERR_UNSUPPORTED, "batches run the ODE method");
  if (p.precision == IVV_PREC_FP64) return bfail(IVV_ERR_UNSUPPORTED, "batches run in FP32 or MIXED precision");
  if (p.x0 || p.y0 || p.full_width || p.full_height)
    return bfail(IVV_ERR_INVALID_ARG, "batches render whole images (no window)");
  if (p.near_clip > 0 || p.n_cut_planes > 0)
    return bfail(IVV_ERR_UNSUPPORTED, "batches render without cutting or near-clip planes");
  if (p.rk_method != IVV_RK_BS32)
    return bfail(IVV_ERR_UNSUPPORTED, "batches integrate with the error-controlled BS3(2) pair (rk_method 0)");
  p.flags = 0;

  ivv_batch* b = new ivv_batch();
  b->p = p;
  b->nreq = n;
  b->P = req[0].volume->hv.P;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess) {
    free_batch(b);
    return bcuda(e, "device query");
  }

  // ---- distinct volumes, in order of first appearance, and their pool offsets
  std::vector<const ivv_volume*> vols;
  std::vector<int> vol_of(n);
  for (int i = 0; i < n; ++i) {
    auto it = std::find(vols.begin(), vols.end(), req[i].volume);
    vol_of[i] = (int)(it - vols.begin());
    if (it == vols.end()) vols.push_back(req[i].volume);
  }
  const int NNN = (b->P + 1) * (b->P + 1) * (b->P + 1), NN = (b->P + 1) * (b->P + 1);
  std::vector<int> face_base(vols.size()), elem_base(vols.size()), brk_base(vols.size());
  std::vector<ivv::FaceMeta> faces;
  size_t n_elem = 0, n_brk = 0;
  for (size_t u = 0; u < vols.size(); ++u) {
    const ivv::HostVolume& hv = vols[u]->hv;
    const int block_base = (int)b->blocks.size();
    face_base[u] = (int)faces.size();
    elem_base[u] = (int)n_elem;
    brk_base[u] = (int)n_brk;
    for (const ivv::BlockInfo& B0 : hv.blocks) {
      ivv::BlockInfo B = B0;
      B.elem_off += elem_base[u];
      for (int d = 0; d < 3; ++d) B.brk_off[d] += brk_base[u];
      B.mode = hv.mode;
      b->blocks.push_back(B);
    }
    for (const ivv::FaceMeta& m0 : hv.faces) {
      ivv::FaceMeta m = m0;
      m.block += block_base;
      faces.push_back(m);
    }
    n_elem += (size_t)hv.n_elems();
    n_brk += hv.brk.size();
  }
  if (b->blocks.size() >= (1u << 27) || faces.size() >= (1u << ivv::kBatchFaceBits)) {
    free_batch(b);
    return bfail(IVV_ERR_UNSUPPORTED, "a batch's volumes hold fewer than 2^27 blocks and 2^20 face patches");
  }
  b->n_faces = (int)faces.size();
  if ((st = balloc(&b->d_blocks, b->blocks.size())) != IVV_OK || (st = balloc(&b->d_brk32, n_brk)) != IVV_OK ||
      (st = balloc(&b->d_brk64, n_brk)) != IVV_OK || (st = balloc(&b->d_elem32, n_elem * NNN)) != IVV_OK ||
      (st = balloc(&b->d_org32, n_elem)) != IVV_OK ||
      (st = balloc(&b->d_face32, (size_t)b->n_faces * NN)) != IVV_OK ||
      (st = balloc(&b->d_face64, (size_t)b->n_faces * NN)) != IVV_OK ||
      (st = balloc(&b->d_faces, (size_t)b->n_faces)) != IVV_OK ||
      (st = balloc(&b->d_faces64, (size_t)b->n_faces)) != IVV_OK) {
    free_batch(b);
    return st;
  }
  e = cudaMemcpyAsync(b->d_blocks, b->blocks.data(), sizeof(ivv::BlockInfo) * b->blocks.size(),
                      cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_faces, faces.data(), sizeof(ivv::FaceMeta) * faces.size(), cudaMemcpyHostToDevice, s);
  for (size_t u = 0; u < vols.size() && e == cudaSuccess; ++u) {
    const ivv_volume* v = vols[u];
    const size_t ne = (size_t)v->hv.n_elems(), nb = v->hv.brk.size(), nf = (size_t)v->hv.n_faces();
    const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
    e = cudaMemcpyAsync(b->d_elem32 + (size_t)elem_base[u] * NNN, v->d_elem32, sizeof(float4) * ne * NNN, k, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_org32 + elem_base[u], v->d_org32, sizeof(float4) * ne, k, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_brk32 + brk_base[u], v->d_brk32, sizeof(float) * nb, k, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_brk64 + brk_base[u], v->d_brk64, sizeof(double) * nb, k, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->d_face32 + (size_t)face_base[u] * NN, v->d_face32, sizeof(float4) * nf * NN, k, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->d_face64 + (size_t)face_base[u] * NN, v->d_face64, sizeof(ivv::Dbl4) * nf * NN, k, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->d_faces64 + face_base[u], v->d_faces64, sizeof(ivv::FaceMeta64) * nf, k, s);
  }
  if (e != cudaSuccess) {
    free_batch(b);
    return bcuda(e, "batch pool upload");
  }

  // ---- request records, transfer-function slots, pixel and tile tables
  std::vector<ivv::DevTFSlot> slots(n);
  std::vector<int> pix0(n + 1), tile0[kNumShapes];
  for (int k = 0; k < kNumShapes; ++k) tile0[k].assign(n + 1, 0);
  b->hreq.resize(n);
  long long pix = 0, tl[kNumShapes] = {}, box = 0, gbox = 0;
  ivv_render_params pw = p;
  for (int i = 0; i < n; ++i) {
    const ivv_request& r = req[i];
    const ivv_volume* v = r.volume;
    ivv::DevRequest& q = b->hreq[i];
    std::memset(&q, 0, sizeof(q));
    if ((st = ivv::frame_cameras(&r.camera, pw, r.width, r.height, q.cam, q.cam64)) != IVV_OK ||
        (st = make_tf_slot(r, slots[i])) != IVV_OK) {
      free_batch(b);
      return st;
    }
    q.face0 = face_base[vol_of[i]];
    q.n_faces = v->hv.n_faces();
    q.box0 = (int)box;
    q.gbox0 = (int)gbox;
    q.diag = (float)v->hv.diag;
    q.ds = (float)(ds_given ? params->ds : v->hv.diag / 128.0);
    q.out = (float4*)r.out_rgba;
    b->max_faces = std::max(b->max_faces, q.n_faces);
    pix0[i] = (int)pix;
    for (int k = 0; k < kNumShapes; ++k) {
      tile0[k][i] = (int)tl[k];
      tl[k] += (long long)((r.width + kShapes[k][0] - 1) / kShapes[k][0]) * ((r.height + kShapes[k][1] - 1) / kShapes[k][1]);
    }
    pix += (long long)r.width * r.height;
    box += q.n_faces;
    gbox += (q.n_faces + ivv::kGroup - 1) / ivv::kGroup;
    if (pix * ivv::kItemsPerPixel >= (1ll << 31) || tl[1] >= (1ll << 31)) {
      free_batch(b);
      return bfail(IVV_ERR_UNSUPPORTED, "a batch holds fewer than 2^27 pixels");
    }
  }
  pix0[n] = (int)pix;
  for (int k = 0; k < kNumShapes; ++k) {
    tile0[k][n] = (int)tl[k];
    b->tiles[k] = (int)tl[k];
  }
  b->npix = pix;
  b->n_boxes = (int)box;
  b->n_gboxes = (int)gbox;
  b->L = batch_layout((size_t)box, (size_t)gbox, (size_t)pix);
  if ((st = balloc(&b->d_req, n)) != IVV_OK || (st = balloc(&b->d_pix0, n + 1)) != IVV_OK ||
      (st = balloc(&b->d_tile0[0], n + 1)) != IVV_OK || (st = balloc(&b->d_tile0[1], n + 1)) != IVV_OK ||
      (st = balloc(&b->d_tile0[2], n + 1)) != IVV_OK || (st = balloc(&b->d_tile0[3], n + 1)) != IVV_OK ||
      (st = balloc(&b->d_tf, n)) != IVV_OK ||
      (st = balloc(&b->d_stats, 1)) != IVV_OK || (st = balloc(&b->ws, b->L.total)) != IVV_OK) {
    free_batch(b);
    return st;
  }
  e = cudaMemcpyAsync(b->d_req, b->hreq.data(), sizeof(ivv::DevRequest) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_pix0, pix0.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s);
  for (int k = 0; k < kNumShapes && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(b->d_tile0[k], tile0[k].data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_tf, slots.data(), sizeof(ivv::DevTFSlot) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_stats, 0, sizeof(ivv::DevStats), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (int i = 0; i <= IVV_N_STAGES && e == cudaSuccess; ++i) e = cudaEventCreate(&b->ev[i]);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    free_batch(b);
    return bcuda(e, "batch tables");
  }
  b->k5_max_ctas[0] = ivv::batch_integrate_max_ctas_per_sm(b->P, p.precision == IVV_PREC_MIXED, false);
  b->k5_max_ctas[1] = ivv::batch_integrate_max_ctas_per_sm(b->P, p.precision == IVV_PREC_MIXED, true);
  b->tune.k5_ctas_per_sm = std::min(4, b->k5_max_ctas[0]);
  b->last_stream = s;
  *out = b;
  return IVV_OK;
}

ivv_status ivv_batch_render(ivv_batch* b, int flags, void* stream) {
  if (!b) return bfail(IVV_ERR_INVALID_ARG, "batch is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  b->last_stream = s;
  const bool stats = (flags & IVV_FLAG_STATS) != 0, timing = (flags & IVV_FLAG_TIMING) != 0;
  const ivv_status sst = ensure_samples(b, s);
  if (sst != IVV_OK) return sst;
  if (stats || timing) return enqueue(b, stats, timing, s);
  if (!b->exec) {
    const ivv_status st = capture(b);
    if (st != IVV_OK) return st;
  }
  IVV_BCUDA(cudaGraphLaunch(b->exec, s));
  return IVV_OK;
}

ivv_status ivv_batch_set_camera(ivv_batch* b, int i, const ivv_camera* camera, void* stream) {
  if (!b || !camera) return bfail(IVV_ERR_INVALID_ARG, "NULL argument");
  if (i < 0 || i >= b->nreq) return bfail(IVV_ERR_INVALID_ARG, "request index out of range");
  ivv::DevRequest q = b->hreq[i];
  const ivv_status st = ivv::frame_cameras(camera, b->p, q.cam.w, q.cam.h, q.cam, q.cam64);
  if (st != IVV_OK) return st;
  b->hreq[i] = q;
  IVV_BCUDA(cudaMemcpyAsync(b->d_req + i, &b->hreq[i], sizeof(q), cudaMemcpyHostToDevice, (cudaStream_t)stream));
  return IVV_OK;
}

ivv_status ivv_batch_set_tuning(ivv_batch* b, const ivv_batch_tuning* t) {
  if (!b || !t) return bfail(IVV_ERR_INVALID_ARG, "NULL argument");
  if (!tuning_ok(*t)) return bfail(IVV_ERR_INVALID_ARG, "unsupported tuning (see ivv_batch_tuning)");
  if (std::memcmp(t, &b->tune, sizeof(*t)) != 0) {
    b->tune = *t;
    drop_graph(b);
  }
  return IVV_OK;
}

ivv_status ivv_batch_get_tuning(const ivv_batch* b, ivv_batch_tuning* t) {
  if (!b || !t) return bfail(IVV_ERR_INVALID_ARG, "NULL argument");
  *t = b->tune;
  return IVV_OK;
}

ivv_status ivv_batch_autotune(ivv_batch* b, int reps, ivv_batch_tuning* best, float* best_ms, void* stream) {
  if (!b) return bfail(IVV_ERR_INVALID_ARG, "batch is NULL");
  if (reps < 1) reps = 3;
  cudaStream_t s = (cudaStream_t)stream;
  // mean time of stage range [s0, s1) over reps renders with tuning t
  auto stage_ms = [&](const ivv_batch_tuning& t, int s0, int s1, float& ms) -> ivv_status {
    b->tune = t;
    ivv_status st = enqueue(b, false, false, s);
    if (st != IVV_OK) return st;
    float sum = 0.f;
    for (int r = 0; r < reps; ++r) {
      if ((st = enqueue(b, false, true, s)) != IVV_OK) return st;
      IVV_BCUDA(cudaEventSynchronize(b->ev[IVV_N_STAGES]));
      float x = 0.f;
      IVV_BCUDA(cudaEventElapsedTime(&x, b->ev[s0], b->ev[s1]));
      sum += x;
    }
    ms = sum / reps;
    return IVV_OK;
  };
  drop_graph(b);
  {
    const ivv_status sst = ensure_samples(b, s);
    if (sst != IVV_OK) return sst;
  }
  ivv_batch_tuning cur = b->tune, win = cur;
  float best_t = 1e30f;
  for (int k = 0; k < kNumWarpShapes; ++k) {     // K2a warp tile by the surface stage
    ivv_batch_tuning t = cur;
    t.tile_w = kShapes[k][0];
    t.tile_h = kShapes[k][1];
    float ms;
    const ivv_status st = stage_ms(t, 1, 2, ms);
    if (st != IVV_OK) return st;
    if (ms < best_t) {
      best_t = ms;
      win = t;
    }
  }
  cur = win;
  best_t = 1e30f;
  for (int c = 1; c <= std::min(4, b->k5_max_ctas[0]); ++c) {   // K5 shape by the integration stage
    for (int ss : {4, 8, 16}) {
      ivv_batch_tuning t = cur;
      t.k5_ctas_per_sm = c;
      t.step_samples = ss;
      float ms;
      const ivv_status st = stage_ms(t, 3, 4, ms);
      if (st != IVV_OK) return st;
      if (ms < best_t) {
        best_t = ms;
        win = t;
      }
    }
  }
  b->tune = win;
  // frame time of the winner through the graph
  ivv_status st = capture(b);
  if (st != IVV_OK) return st;
  IVV_BCUDA(cudaGraphLaunch(b->exec, s));
  IVV_BCUDA(cudaEventRecord(b->ev[0], s));
  for (int r = 0; r < reps; ++r) IVV_BCUDA(cudaGraphLaunch(b->exec, s));
  IVV_BCUDA(cudaEventRecord(b->ev[1], s));
  IVV_BCUDA(cudaEventSynchronize(b->ev[1]));
  float ms = 0.f;
  IVV_BCUDA(cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]));
  b->timed = false;
  b->last_stream = s;
  if (best) *best = win;
  if (best_ms) *best_ms = ms / reps;
  return IVV_OK;
}

ivv_status ivv_batch_get_stats(ivv_batch* b, ivv_stats* out) {
  if (!b || !out) return bfail(IVV_ERR_INVALID_ARG, "NULL argument");
  IVV_BCUDA(cudaStreamSynchronize(b->last_stream));
  ivv::DevStats d;
  IVV_BCUDA(cudaMemcpy(&d, b->d_stats, sizeof(d), cudaMemcpyDeviceToHost));
  ivv::stats_to_public(d, out);
  return IVV_OK;
}

ivv_status ivv_batch_reset_stats(ivv_batch* b) {
  if (!b) return bfail(IVV_ERR_INVALID_ARG, "batch is NULL");
  IVV_BCUDA(cudaStreamSynchronize(b->last_stream));
  IVV_BCUDA(cudaMemset(b->d_stats, 0, sizeof(ivv::DevStats)));
  return IVV_OK;
}

ivv_status ivv_batch_get_stage_times(ivv_batch* b, float* ms) {
  if (!b || !ms) return bfail(IVV_ERR_INVALID_ARG, "NULL argument");
  if (!b->timed) return bfail(IVV_ERR_INVALID_ARG, "no batch render with IVV_FLAG_TIMING was made");
  IVV_BCUDA(cudaEventSynchronize(b->ev[IVV_N_STAGES]));
  for (int i = 0; i < IVV_N_STAGES; ++i) IVV_BCUDA(cudaEventElapsedTime(&ms[i], b->ev[i], b->ev[i + 1]));
  return IVV_OK;
}

ivv_status ivv_batch_info(const ivv_batch* b, int* n_requests, long long* n_pixels, size_t* workspace_bytes,
                          int* graph_ready) {
  if (!b) return bfail(IVV_ERR_INVALID_ARG, "batch is NULL");
  if (n_requests) *n_requests = b->nreq;
  if (n_pixels) *n_pixels = b->npix;
  if (workspace_bytes) *workspace_bytes = b->L.total;
  if (graph_ready) *graph_ready = b->exec ? 1 : 0;
  return IVV_OK;
}

void ivv_batch_destroy(ivv_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  free_batch(b);
}

}  // extern "C"
