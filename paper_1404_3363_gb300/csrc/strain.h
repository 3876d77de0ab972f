// Von Mises value of the strain of a displacement field (§6.2, Eq. 24),
// shared by the host preparation (FP64, default scalar range) and the
// kernels (FP32 / FP64, every sample of IVV_SCALAR_VONMISES).
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define IVV_HD __host__ __device__ __forceinline__
#else
#define IVV_HD inline
#endif

namespace ivv {

// J = J_phi(p), Ju = J_u(p) (J[r][c] = d f_r / d p_c).  The Jacobian of
// u o phi^-1 at phi(p) is A = J_u J_phi^-1 = J_u adj(J_phi) / det J_phi (its
// transpose is what J_phi^T X = J_u^T gives; the strain only uses the
// symmetric part, which is the same).  sigma = (A + A^T) / 2 and
// rho = sqrt(((s11-s22)^2 + (s22-s33)^2 + (s33-s11)^2 + 6 (s12^2 + s23^2 + s31^2)) / 2).
template <typename R>
IVV_HD R von_mises(const R J[3][3], const R Ju[3][3]) {
  R adj[3][3];
  adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  const R det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
  const R inv = R(1) / det;
  R A[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) A[r][c] = (Ju[r][0] * adj[0][c] + Ju[r][1] * adj[1][c] + Ju[r][2] * adj[2][c]) * inv;
  const R d01 = A[0][0] - A[1][1], d12 = A[1][1] - A[2][2], d20 = A[2][2] - A[0][0];
  const R s01 = R(0.5) * (A[0][1] + A[1][0]), s12 = R(0.5) * (A[1][2] + A[2][1]), s20 = R(0.5) * (A[2][0] + A[0][2]);
  const R q = d01 * d01 + d12 * d12 + d20 * d20 + R(6) * (s01 * s01 + s12 * s12 + s20 * s20);
  return sqrt(R(0.5) * q);
}

}  // namespace ivv
