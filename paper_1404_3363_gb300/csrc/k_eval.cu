// Spline evaluation at caller-given parameter points (Eq. 1 on the Bezier
// elements): the device evaluator K5 uses, exposed for testing and tools.
#include "ivv_device.cuh"

namespace ivv {
namespace {

template <int P>
__global__ void k_eval_points(DevVolume V, int block, int n, const float* __restrict__ p, float* __restrict__ phi,
                              float* __restrict__ jac, float* __restrict__ rho) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const BlockInfo B = V.blocks[block];
  const float q[3] = {p[3 * i], p[3 * i + 1], p[3 * i + 2]};
  float f[3], J[3][3], rc;
  eval_block<P, float, true>(V, B, q, f, J, rc);
  if (phi)
    for (int r = 0; r < 3; ++r) phi[3 * i + r] = f[r];
  if (jac)
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) jac[9 * i + 3 * r + c] = J[r][c];
  if (rho) rho[i] = scalar_at<P, float>(V, B, V.mode, q, J, rc);
}

}  // namespace

void launch_eval_points(const DevVolume& V, int block, int n, const float* p, float* phi, float* jac, float* rho,
                        cudaStream_t s) {
  if (n <= 0) return;
  if (V.P == 2)
    k_eval_points<2><<<(n + 127) / 128, 128, 0, s>>>(V, block, n, p, phi, jac, rho);
  else
    k_eval_points<3><<<(n + 127) / 128, 128, 0, s>>>(V, block, n, p, phi, jac, rho);
}

}  // namespace ivv
