// Batched stage 3.  The split integration of single frames over every
// request of a batch: per-pixel sample counts with each request's sample
// distance, their scan, the trace kernel K5t and the shading pass with
// BATCH = true (k_trace.cuh, k_integrate.cuh); pixels whose sample list does
// not fit the batch's sample buffer are compacted into a list and rendered by
// the fused integrator K5 (BATCH = true), which is also the whole of stage 3
// when the batch has no sample buffer.
#include "k_integrate.cuh"
#include "k_trace.cuh"

namespace ivv {

namespace {

template <int P, bool MIXED, bool STATS>
void launch_kb5(const DevVolume& V, const BatchArgs& ba, const IntegrateArgs& a, const float4* pin,
                const float4* pout, const int* pblk, const int* pcnt, const int* active, const int* n_active,
                int* queue_head, DevStats* st, int grid, cudaStream_t s) {
  DevCamera<float> cam{};
  DevTF tf{};
  k5_integrate<P, float, MIXED, STATS, true><<<grid, 128, 0, s>>>(V, cam, tf, a, ba, pin, pout, pblk, pcnt,
                                                                  active, n_active, queue_head, nullptr, st);
}

// Samples of each active pixel (the integrator's sample rule with its
// request's ds and diagonal).
__global__ void kb_count(BatchArgs ba, const float4* __restrict__ pair_in, const float4* __restrict__ pair_out,
                         const int* __restrict__ pair_count, const int* __restrict__ active,
                         const int* __restrict__ n_active, int npix, int* __restrict__ cnt) {
  const int nact = *n_active;
  for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < nact; item += gridDim.x * blockDim.x) {
    const int pix = __ldg(active + item);
    const DevRequest& rr = ba.req[batch_request(ba, pix)];
    const float ds = rr.ds, tail_eps = 1e-12f * rr.diag;
    const int np = __ldg(pair_count + pix);
    int c = 0;
    for (int q = 0; q < np; ++q) {
      const size_t slot = (size_t)q * npix + pix;
      const float L = pair_out[slot].x - pair_in[slot].x;
      if (!(L > 0.f)) continue;
      const float fl = floorf(L / ds);
      c += (int)fl + ((L - fl * ds > tail_eps) ? 1 : 0) + 1;
    }
    cnt[item] = c;
  }
}

// Active pixels whose sample list would end beyond cap (all of them when the
// scanned total did not fit an int: n_active[3] > 0), for the fused integrator.
__global__ void kb_overflow(const int* __restrict__ active, const int* __restrict__ n_active,
                            const int* __restrict__ off, const int* __restrict__ cnt, int cap, int* __restrict__ list,
                            int* __restrict__ n_list) {
  const int nact = *n_active;
  const bool excess = n_active[3] > 0;
  for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < nact; item += gridDim.x * blockDim.x) {
    const int o = __ldg(off + item);
    if (excess || o < 0 || o + __ldg(cnt + item) > cap) list[atomicAdd(n_list, 1)] = __ldg(active + item);
  }
}

template <int P, bool MIXED, bool STATS>
void launch_kb5t(const DevVolume& V, const BatchArgs& ba, const IntegrateArgs& a, const float4* pin, const float4* pout,
                 const int* pblk, const int* pcnt, const int* active, const int* n_active, int* queue_head,
                 const int* off, const int* cnt, float4* sp, int cap, DevStats* st, int grid, cudaStream_t s) {
  DevCamera<float> cam{};
  k5_trace<P, MIXED, STATS, true><<<grid, 128, 0, s>>>(V, cam, a, ba, cnt, pin, pout, pblk, pcnt, active, n_active,
                                                       queue_head, off, sp, cap, st);
}

template <int P, bool STATS>
void launch_kbshade(const DevVolume& V, const BatchArgs& ba, const IntegrateArgs& a, const float4* pin,
                    const float4* pout, const int* pblk, const int* pcnt, const int* active, const int* n_active,
                    int* queue_head, const int* off, const int* cnt, const float4* sp, int cap, DevStats* st,
                    int num_sms, cudaStream_t s) {
  DevCamera<float> cam{};
  DevTF tf{};
  static int per_sm = -1;
  if (per_sm < 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_shade_composite<P, STATS, false, true>, 128, 0);
    if (per_sm < 1) per_sm = 1;
  }
  int grid = num_sms * per_sm;                      // persistent: the lanes refill from the queue
  const int useful = (a.npix + 127) / 128;
  grid = grid < useful ? grid : (useful > 0 ? useful : 1);
  k_shade_composite<P, STATS, false, true><<<grid, 128, 0, s>>>(V, cam, tf, a.K, a.early_alpha, ba, cnt, pin, pout,
                                                                 pblk, pcnt, active, n_active, queue_head, off,
                                                                 a.npix, 0.f, 0.f, cap, sp, nullptr, st);
}

template <int P, bool MIXED, bool STATS>
int max_ctas() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k5_integrate<P, float, MIXED, STATS, true>, 128, 0);
  return n < 1 ? 1 : n;
}

}  // namespace

void launch_batch_integrate(const DevVolume& V, const BatchArgs& ba, const IntegrateArgs& a, bool mixed, bool stats,
                            const float4* pin, const float4* pout, const int* pblk, const int* pcnt,
                            const int* active, const int* n_active, int* queue_head, DevStats* st, int grid,
                            cudaStream_t s) {
  if (grid < 1) grid = 1;
#define IVV_KB5(PP, MM, SS) \
  launch_kb5<PP, MM, SS>(V, ba, a, pin, pout, pblk, pcnt, active, n_active, queue_head, st, grid, s)
  if (V.P == 2) {
    if (mixed) { if (stats) IVV_KB5(2, true, true); else IVV_KB5(2, true, false); }
    else { if (stats) IVV_KB5(2, false, true); else IVV_KB5(2, false, false); }
  } else {
    if (mixed) { if (stats) IVV_KB5(3, true, true); else IVV_KB5(3, true, false); }
    else { if (stats) IVV_KB5(3, false, true); else IVV_KB5(3, false, false); }
  }
#undef IVV_KB5
}

void launch_batch_count(const BatchArgs& ba, const float4* pin, const float4* pout, const int* pcnt, const int* active,
                        const int* n_active, int npix, int* cnt, int num_sms, cudaStream_t s) {
  kb_count<<<num_sms * 8, 256, 0, s>>>(ba, pin, pout, pcnt, active, n_active, npix, cnt);
}

void launch_batch_split(const DevVolume& V, const BatchArgs& ba, const IntegrateArgs& a, bool mixed, bool stats,
                        const float4* pin, const float4* pout, const int* pblk, const int* pcnt, const int* active,
                        int* counters, int* off, int* cnt, int* sums, float4* sp, int cap, int* list, int grid,
                        int num_sms, DevStats* st, cudaStream_t s) {
  if (grid < 1) grid = 1;
  const int npix = a.npix;
  launch_batch_count(ba, pin, pout, pcnt, active, counters, npix, cnt, num_sms, s);
  launch_rf_scan(cnt, counters, npix, off, sums, 0x7fffffff, counters + 2, s);
  int* qhead = counters + kQueueHeadOff;
  int* n_list = counters + kOverflowCounter;
#define IVV_KB5T(PP, MM, SS) \
  launch_kb5t<PP, MM, SS>(V, ba, a, pin, pout, pblk, pcnt, active, counters, qhead, off, cnt, sp, cap, st, grid, s)
#define IVV_KBS(PP, SS) \
  launch_kbshade<PP, SS>(V, ba, a, pin, pout, pblk, pcnt, active, counters, counters + kShadeHead, off, cnt, sp, cap, \
                         st, num_sms, s)
  if (V.P == 2) {
    if (mixed) { if (stats) IVV_KB5T(2, true, true); else IVV_KB5T(2, true, false); }
    else { if (stats) IVV_KB5T(2, false, true); else IVV_KB5T(2, false, false); }
    if (stats) IVV_KBS(2, true); else IVV_KBS(2, false);
  } else {
    if (mixed) { if (stats) IVV_KB5T(3, true, true); else IVV_KB5T(3, true, false); }
    else { if (stats) IVV_KB5T(3, false, true); else IVV_KB5T(3, false, false); }
    if (stats) IVV_KBS(3, true); else IVV_KBS(3, false);
  }
#undef IVV_KB5T
#undef IVV_KBS
  // pixels beyond the sample buffer: the fused integrator over their list
  kb_overflow<<<num_sms * 8, 256, 0, s>>>(active, counters, off, cnt, cap, list, n_list);
  launch_batch_integrate(V, ba, a, mixed, stats, pin, pout, pblk, pcnt, list, n_list, counters + kOverflowHead, st,
                         grid, s);
}

int batch_integrate_max_ctas_per_sm(int P, bool mixed, bool stats) {
  if (P == 2) {
    if (mixed) return stats ? max_ctas<2, true, true>() : max_ctas<2, true, false>();
    return stats ? max_ctas<2, false, true>() : max_ctas<2, false, false>();
  }
  if (mixed) return stats ? max_ctas<3, true, true>() : max_ctas<3, true, false>();
  return stats ? max_ctas<3, false, true>() : max_ctas<3, false, false>();
}

}  // namespace ivv
