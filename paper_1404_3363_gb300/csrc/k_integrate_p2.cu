// Degree-2 instantiations of the ray integrator (K5, K5t and the shading
// pass); see k_integrate.cuh and k_trace.cuh.
#include "k_integrate.cuh"
#include "k_trace.cuh"

namespace ivv {
template void launch_integrate_p<2>(const DevVolume&, const DevCamera<float>*, const DevCamera<double>*,
                                     const DevTF&, const IntegrateArgs&, bool, bool, const void*, const void*,
                                     const int*, const int*, const int*, const int*, int*, float4*, DevStats*, int,
                                     cudaStream_t);
template void launch_integrate_split_p<2>(const DevVolume&, const DevCamera<float>&, const IntegrateArgs&,
                                           const SplitArgs&, bool, bool, const float4*, const float4*, const int*,
                                           const int*, const int*, const int*, int*, DevStats*, int, cudaStream_t);
template void launch_shade_composite_p<2>(const DevVolume&, const DevCamera<float>&, const DevTF&, int, float,
                                           const float4*, const float4*, const int*, const int*, const int*,
                                           const int*, int*, const int*, int, float, float, const SplitArgs&, float4*, bool,
                                           DevStats*, int, cudaStream_t);
}  // namespace ivv
