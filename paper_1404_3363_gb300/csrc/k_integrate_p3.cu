// Degree-3 instantiations of the ray integrator (K5); see k_integrate.cuh.
#include "k_integrate.cuh"

namespace ivv {
template void launch_integrate_p<3>(const DevVolume&, const DevCamera<float>*, const DevCamera<double>*,
                                     const DevTF&, const IntegrateArgs&, bool, bool, const void*, const void*,
                                     const int*, const int*, const int*, const int*, int*, float4*, DevStats*, int,
                                     cudaStream_t);
}  // namespace ivv
