// Degree-2 instantiations of the fixed-step integrators (K5f, see k_fixed.cuh;
// implicit Euler K5i, see k_irk1.cuh).
#include "k_fixed.cuh"
#include "k_irk1.cuh"

namespace ivv {
template void launch_fixed_p<2>(const DevVolume&, const DevCamera<float>&, const DevTF&, const IntegrateArgs&,
                                  const RkTableau&, bool, bool, const float4*, const float4*, const int*, const int*,
                                  const int*, const int*, int*, float4*, DevStats*, int, cudaStream_t);
template void launch_irk1_p<2>(const DevVolume&, const DevCamera<float>&, const DevTF&, const IntegrateArgs&,
                                 bool, bool, const float4*, const float4*, const int*, const int*, const int*,
                                 const int*, int*, float4*, DevStats*, int, cudaStream_t);
}  // namespace ivv
