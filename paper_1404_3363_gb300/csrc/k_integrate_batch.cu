// Batched stage 3: one persistent K5 launch whose work queue spans every
// request of a batch (k_integrate.cuh, BATCH = true).
#include "k_integrate.cuh"

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

int batch_integrate_max_ctas_per_sm(int P, bool mixed, bool stats) {
  if (P == 2) {
    if (mixed) return stats ? max_ctas<2, true, true>() : max_ctas<2, true, false>();
    return stats ? max_ctas<2, false, true>() : max_ctas<2, false, false>();
  }
  if (mixed) return stats ? max_ctas<3, true, true>() : max_ctas<3, true, false>();
  return stats ? max_ctas<3, false, true>() : max_ctas<3, false, false>();
}

}  // namespace ivv
