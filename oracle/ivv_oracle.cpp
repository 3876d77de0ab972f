// FP64 CPU oracle for isogeometric volume ray integration
// (Fuchs & Hjelmervik, "Interactive Isogeometric Volume Visualization with
// Pixel-Accurate Geometry", TVCG 2015).
//
// TEST INFRASTRUCTURE ONLY.  Nothing here is part of the product path: only
// the tests, the smoke check and the benchmark's CPU-baseline leg may load it.
// It shares no code with the CUDA library; both only read the same seeded
// inputs.
//
// What it computes, in the paper's order:
//   * Eq. 1: trivariate tensor-product B-splines, evaluated by the Cox-de Boor
//     recurrence on the caller's (normalised) knots, with first partials.
//   * §4.1: all intersections of a pixel ray with the 6 boundary surfaces of
//     every block.  The paper rasterises a pixel-accurate tessellation; the
//     oracle instead finds the exact roots: each polynomial piece of a face is
//     converted to Bernstein form by collocation, subdivided by de Casteljau
//     with convex-hull rejection, and polished by Newton in FP64.
//   * §4.2, Alg. 2: blockwise depth pairing of the sorted hit list.
//   * §5.1 (Eqs. 6-7): the preimage of every sample point g_j on the ray is
//     found by Newton's method with a Householder-QR 3x3 solve, clamping to
//     [0,1]^3 and a halving line search ("RF").  A second, independent route
//     integrates the pulled-back ODE of §5.2 (Eqs. 10-15) with an embedded
//     Runge-Kutta-Fehlberg 4(5) pair.
//   * §3.2.1, Alg. 1 with supersampling: front-to-back compositing with K
//     midpoint sub-samples of a linearly interpolated scalar per interval.
//   * §5.3, Table 1: fixed-step explicit RK family on the analytic 2-D map of
//     the convergence study (lifted to 3-D), used to pin the tableaux.
//
// Readings of points the paper leaves open (all listed in the design notes):
//   alpha_src = 1 - exp(-sigma A xi)  => T = exp(-sigma A ds_i);
//   uniform sample distance ds in G arc length, last interval partial;
//   K midpoint sub-samples; background 0; early stop at alpha >= early_alpha;
//   V_par = pixel ray direction; front-facing := d . n_out < 0;
//   hits of one block with equal facing closer than 1e-9 diag are merged.
//
// Parity-pinned by tests/test_oracle_*.py (closed forms, printed Table 1,
// scipy's B-spline basis, brute force on tiny inputs).

#include <algorithm>
#include <atomic>
#include <cmath>
#include <limits>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

namespace {

typedef double V3[3];

inline double dot3(const double* a, const double* b) { return a[0]*b[0] + a[1]*b[1] + a[2]*b[2]; }
inline void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1]*b[2] - a[2]*b[1];
  c[1] = a[2]*b[0] - a[0]*b[2];
  c[2] = a[0]*b[1] - a[1]*b[0];
}
inline double norm3(const double* a) { return std::sqrt(dot3(a, a)); }

// ------------------------------------------------------------------ QR solve
// Householder QR of a 3x3 matrix and solution of A x = b (§5.1 names QR as
// the solver of the Newton system).  Returns false if R has a zero pivot.
bool qr_solve3(const double Ain[3][3], const double bin[3], double x[3]) {
  double A[3][3], b[3];
  for (int i = 0; i < 3; ++i) { b[i] = bin[i]; for (int j = 0; j < 3; ++j) A[i][j] = Ain[i][j]; }
  for (int k = 0; k < 3; ++k) {
    double nrm = 0;
    for (int i = k; i < 3; ++i) nrm += A[i][k] * A[i][k];
    nrm = std::sqrt(nrm);
    if (nrm == 0) continue;
    double alpha = A[k][k] > 0 ? -nrm : nrm;      // avoid cancellation
    double v[3] = {0, 0, 0};
    for (int i = k; i < 3; ++i) v[i] = A[i][k];
    v[k] -= alpha;
    double vv = 0;
    for (int i = k; i < 3; ++i) vv += v[i] * v[i];
    if (vv == 0) continue;
    for (int j = k; j < 3; ++j) {                  // A <- (I - 2 v v^T / v^T v) A
      double s = 0;
      for (int i = k; i < 3; ++i) s += v[i] * A[i][j];
      s = 2 * s / vv;
      for (int i = k; i < 3; ++i) A[i][j] -= s * v[i];
    }
    double s = 0;
    for (int i = k; i < 3; ++i) s += v[i] * b[i];
    s = 2 * s / vv;
    for (int i = k; i < 3; ++i) b[i] -= s * v[i];
  }
  for (int i = 2; i >= 0; --i) {                   // back substitution R x = Q^T b
    if (A[i][i] == 0) return false;
    double s = b[i];
    for (int j = i + 1; j < 3; ++j) s -= A[i][j] * x[j];
    x[i] = s / A[i][i];
  }
  return true;
}

double det3(const double J[3][3]) {
  return J[0][0]*(J[1][1]*J[2][2] - J[1][2]*J[2][1])
       - J[0][1]*(J[1][0]*J[2][2] - J[1][2]*J[2][0])
       + J[0][2]*(J[1][0]*J[2][1] - J[1][1]*J[2][0]);
}

// ------------------------------------------------------- B-spline (Eq. 1)
// All B-splines N_{i,p} of one knot vector at x, by the Cox-de Boor
// recurrence, plus their first derivatives.  x is clamped to [t_0, t_end];
// at x == t_end the last non-empty span is taken as closed on the right.
struct Basis1D {
  std::vector<double> t;   // knots, normalised to [0,1]
  int p = 0;
  int n = 0;               // number of basis functions / control points
  void eval(double x, std::vector<double>& N, std::vector<double>& dN) const {
    const int m = (int)t.size() - 1;               // last knot index
    if (x < t[0]) x = t[0];
    if (x > t[m]) x = t[m];
    std::vector<double> cur(m, 0.0);               // degree-0 functions
    int last_span = -1;
    for (int i = 0; i < m; ++i) if (t[i] < t[i + 1]) last_span = i;
    for (int i = 0; i < m; ++i) {
      if (t[i] <= x && x < t[i + 1]) cur[i] = 1.0;
    }
    if (x == t[m]) cur[last_span] = 1.0;
    std::vector<double> prev;                      // degree p-1 functions
    for (int q = 1; q <= p; ++q) {
      prev = cur;
      std::vector<double> nxt(m - q, 0.0);
      for (int i = 0; i < m - q; ++i) {
        double a = 0, b = 0;
        double d1 = t[i + q] - t[i], d2 = t[i + q + 1] - t[i + 1];
        if (d1 > 0) a = (x - t[i]) / d1 * prev[i];
        if (d2 > 0) b = (t[i + q + 1] - x) / d2 * prev[i + 1];
        nxt[i] = a + b;
      }
      cur.swap(nxt);
    }
    N.assign(cur.begin(), cur.begin() + n);
    dN.assign(n, 0.0);
    if (p == 0) return;
    // derivative: N'_{i,p} = p/(t_{i+p}-t_i) N_{i,p-1} - p/(t_{i+p+1}-t_{i+1}) N_{i+1,p-1}
    for (int i = 0; i < n; ++i) {
      double d1 = t[i + p] - t[i], d2 = t[i + p + 1] - t[i + 1];
      double v = 0;
      if (d1 > 0) v += p / d1 * prev[i];
      if (d2 > 0) v -= p / d2 * prev[i + 1];
      dN[i] = v;
    }
  }
};

// N, N' and N'' of one knot vector at x: the derivative formula of Eq. 1's
// B-splines applied twice,
//   N'_{i,q} = q/(t_{i+q}-t_i) N_{i,q-1} - q/(t_{i+q+1}-t_{i+1}) N_{i+1,q-1},
// once to the degree p-1 functions (giving N'_{.,p}) and once to the
// derivatives of the degree p-1 functions (giving N''_{.,p}).  Outside
// [t_0, t_end] the polynomials of the first or last non-empty span are
// continued (the recursion is polynomial in x), which is what the implicit
// Euler Newton iteration evaluates when an iterate leaves the parameter box.
void basis_eval2(const Basis1D& B, double x, std::vector<double>& N, std::vector<double>& dN,
                 std::vector<double>& ddN) {
  const std::vector<double>& t = B.t;
  const int p = B.p, n = B.n, m = (int)t.size() - 1;
  std::vector<std::vector<double>> Nq(p + 1);      // Nq[q][i] = N_{i,q}(x)
  Nq[0].assign(m, 0.0);
  int first_span = -1, last_span = -1;
  for (int i = 0; i < m; ++i)
    if (t[i] < t[i + 1]) {
      if (first_span < 0) first_span = i;
      last_span = i;
    }
  for (int i = 0; i < m; ++i) if (t[i] <= x && x < t[i + 1]) Nq[0][i] = 1.0;
  if (x >= t[m]) Nq[0][last_span] = 1.0;
  if (x < t[0]) Nq[0][first_span] = 1.0;
  for (int q = 1; q <= p; ++q) {
    Nq[q].assign(m - q, 0.0);
    for (int i = 0; i < m - q; ++i) {
      double a = 0, b = 0;
      const double d1 = t[i + q] - t[i], d2 = t[i + q + 1] - t[i + 1];
      if (d1 > 0) a = (x - t[i]) / d1 * Nq[q - 1][i];
      if (d2 > 0) b = (t[i + q + 1] - x) / d2 * Nq[q - 1][i + 1];
      Nq[q][i] = a + b;
    }
  }
  // derivative of the degree-q functions from the degree-(q-1) values v
  auto deriv = [&](int q, const std::vector<double>& v, int count) {
    std::vector<double> out(count, 0.0);
    for (int i = 0; i < count; ++i) {
      const double d1 = t[i + q] - t[i], d2 = t[i + q + 1] - t[i + 1];
      double w = 0;
      if (d1 > 0) w += q / d1 * v[i];
      if (d2 > 0 && i + 1 < (int)v.size()) w -= q / d2 * v[i + 1];
      out[i] = w;
    }
    return out;
  };
  N.assign(Nq[p].begin(), Nq[p].begin() + n);
  dN.assign(n, 0.0);
  ddN.assign(n, 0.0);
  if (p >= 1) dN = deriv(p, Nq[p - 1], n);
  if (p >= 2) {
    const std::vector<double> dprev = deriv(p - 1, Nq[p - 2], m - p + 1);   // N'_{i,p-1}
    ddN = deriv(p, dprev, n);
  }
}

struct Block {
  Basis1D B[3];
  std::vector<double> geom;    // [nw][nv][nu][3]
  std::vector<double> scal;    // [nw][nv][nu] or empty
  std::vector<double> disp;    // [nw][nv][nu][3] displacement u (§6.2) or empty
  double mean_abs_det = 1.0;   // mean of |det J| over [0,1]^3 (the block's volume in G)
};

// phi, J (J[r][c] = d phi_r / d p_c) and scalar (cp mode) at p in [0,1]^3.
void block_eval(const Block& b, const double p[3], double phi[3], double J[3][3], double* rho) {
  std::vector<double> N[3], dN[3];
  for (int d = 0; d < 3; ++d) b.B[d].eval(p[d], N[d], dN[d]);
  const int nu = b.B[0].n, nv = b.B[1].n, nw = b.B[2].n;
  for (int r = 0; r < 3; ++r) { phi[r] = 0; J[r][0] = J[r][1] = J[r][2] = 0; }
  double s = 0;
  for (int k = 0; k < nw; ++k) {
    if (N[2][k] == 0 && dN[2][k] == 0) continue;
    for (int j = 0; j < nv; ++j) {
      if (N[1][j] == 0 && dN[1][j] == 0) continue;
      for (int i = 0; i < nu; ++i) {
        if (N[0][i] == 0 && dN[0][i] == 0) continue;
        const size_t idx = ((size_t)k * nv + j) * nu + i;
        const double* c = &b.geom[3 * idx];
        const double w0 = N[0][i] * N[1][j] * N[2][k];
        const double wu = dN[0][i] * N[1][j] * N[2][k];
        const double wv = N[0][i] * dN[1][j] * N[2][k];
        const double ww = N[0][i] * N[1][j] * dN[2][k];
        for (int r = 0; r < 3; ++r) {
          phi[r] += w0 * c[r];
          J[r][0] += wu * c[r];
          J[r][1] += wv * c[r];
          J[r][2] += ww * c[r];
        }
        if (!b.scal.empty()) s += w0 * b.scal[idx];
      }
    }
  }
  if (rho) *rho = s;
}

// phi, J and the Hessian H[r][a][b] = d^2 phi_r / dp_a dp_b at p (p may lie
// outside [0,1]^3: the boundary elements' polynomials are continued).
void block_eval2(const Block& b, const double p[3], double phi[3], double J[3][3], double H[3][3][3]) {
  std::vector<double> N[3], dN[3], ddN[3];
  for (int d = 0; d < 3; ++d) basis_eval2(b.B[d], p[d], N[d], dN[d], ddN[d]);
  const int nu = b.B[0].n, nv = b.B[1].n, nw = b.B[2].n;
  for (int r = 0; r < 3; ++r) {
    phi[r] = 0;
    for (int a = 0; a < 3; ++a) {
      J[r][a] = 0;
      for (int c = 0; c < 3; ++c) H[r][a][c] = 0;
    }
  }
  for (int k = 0; k < nw; ++k)
    for (int j = 0; j < nv; ++j)
      for (int i = 0; i < nu; ++i) {
        // value, first and second derivative of each factor
        const double u[3] = {N[0][i], dN[0][i], ddN[0][i]};
        const double v[3] = {N[1][j], dN[1][j], ddN[1][j]};
        const double w[3] = {N[2][k], dN[2][k], ddN[2][k]};
        if (u[0] == 0 && u[1] == 0 && u[2] == 0) continue;
        if (v[0] == 0 && v[1] == 0 && v[2] == 0) continue;
        if (w[0] == 0 && w[1] == 0 && w[2] == 0) continue;
        const double* cp = &b.geom[3 * (((size_t)k * nv + j) * nu + i)];
        // derivative orders (ou, ov, ow) of d^2/dp_a dp_b: a, b in {0,1,2}
        for (int r = 0; r < 3; ++r) {
          phi[r] += u[0] * v[0] * w[0] * cp[r];
          J[r][0] += u[1] * v[0] * w[0] * cp[r];
          J[r][1] += u[0] * v[1] * w[0] * cp[r];
          J[r][2] += u[0] * v[0] * w[1] * cp[r];
          for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) {
              int o[3] = {0, 0, 0};
              ++o[a];
              ++o[c];
              H[r][a][c] += u[o[0]] * v[o[1]] * w[o[2]] * cp[r];
            }
        }
      }
}

enum { MODE_CP = 0, MODE_DETJ = 1, MODE_QUALITY = 2, MODE_VONMISES = 3 };

// J_u[r][c] = d u_r / d p_c of the displacement spline u: P -> R^3 (§6.2),
// same knots and basis as the geometry, Cox-de Boor at p.
void disp_jacobian(const Block& b, const double p[3], double Ju[3][3]) {
  std::vector<double> N[3], dN[3];
  for (int d = 0; d < 3; ++d) b.B[d].eval(p[d], N[d], dN[d]);
  const int nu = b.B[0].n, nv = b.B[1].n, nw = b.B[2].n;
  for (int r = 0; r < 3; ++r) Ju[r][0] = Ju[r][1] = Ju[r][2] = 0;
  for (int k = 0; k < nw; ++k)
    for (int j = 0; j < nv; ++j)
      for (int i = 0; i < nu; ++i) {
        const double* c = &b.disp[3 * (((size_t)k * nv + j) * nu + i)];
        const double wu = dN[0][i] * N[1][j] * N[2][k];
        const double wv = N[0][i] * dN[1][j] * N[2][k];
        const double ww = N[0][i] * N[1][j] * dN[2][k];
        for (int r = 0; r < 3; ++r) {
          Ju[r][0] += wu * c[r];
          Ju[r][1] += wv * c[r];
          Ju[r][2] += ww * c[r];
        }
      }
}

// §6.2 (Eq. 24): the Jacobian of u o phi^-1 at g = phi(p) solves
// J_phi(p)^T X = J_u(p)^T column by column (QR), the strain tensor is its
// symmetric part sigma = (X + X^T) / 2, and rho is the von Mises value
// sqrt(((s11 - s22)^2 + (s22 - s33)^2 + (s33 - s11)^2
//        + 6 (s12^2 + s23^2 + s31^2)) / 2)
// (the squares and the root, garbled in the printed equation, restored).
double von_mises(const Block& b, const double p[3], const double J[3][3]) {
  double Ju[3][3], JT[3][3], X[3][3];
  disp_jacobian(b, p, Ju);
  for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) JT[r][c] = J[c][r];
  for (int col = 0; col < 3; ++col) {
    const double rhs[3] = {Ju[col][0], Ju[col][1], Ju[col][2]};   // column col of J_u^T
    double x[3];
    qr_solve3(JT, rhs, x);
    for (int r = 0; r < 3; ++r) X[r][col] = x[r];
  }
  double sg[3][3];
  for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) sg[r][c] = 0.5 * (X[r][c] + X[c][r]);
  const double d01 = sg[0][0] - sg[1][1], d12 = sg[1][1] - sg[2][2], d20 = sg[2][2] - sg[0][0];
  const double q = d01 * d01 + d12 * d12 + d20 * d20 +
                   6.0 * (sg[0][1] * sg[0][1] + sg[1][2] * sg[1][2] + sg[2][0] * sg[2][0]);
  return std::sqrt(0.5 * q);
}

// The scalar field rho at p of block b for the volume's mode; J = J_phi(p).
double scalar_of(const Block& b, int mode, const double p[3], const double J[3][3], double rho_cp) {
  if (mode == MODE_CP) return rho_cp;
  if (mode == MODE_VONMISES) return von_mises(b, p, J);
  const double dj = det3(J);
  if (mode == MODE_DETJ) return dj;
  double f = 0;                                     // Eq. 23: det J / ||J||_F
  for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) f += J[r][c] * J[r][c];
  return dj / std::sqrt(f);
}

// ----------------------------------------------------------- face pieces
// Face f of a block: f = 0/1 -> u = 0/1, 2/3 -> v = 0/1, 4/5 -> w = 0/1.
// Face coordinates (a, b): u-faces (v, w), v-faces (w, u), w-faces (u, v);
// with det J > 0, d(phi)/da x d(phi)/db points to increasing normal coordinate,
// so the outward normal is -(phi_a x phi_b) on the 0-faces and + on the 1-faces.
inline void face_axes(int f, int& nd, int& ad, int& bd) {
  nd = f / 2;
  ad = (nd + 1) % 3;
  bd = (nd + 2) % 3;
}

struct Piece {                 // one polynomial piece of a boundary face
  int block, face;
  double a0, a1, b0, b1;       // parameter box of the piece (normalised)
  int pa, pb;                  // degrees along a, b
  std::vector<double> cp;      // Bernstein cp [(pa+1)*(pb+1)][3], a fastest
  double lo[3], hi[3];         // bbox of cp
};

double binom(int n, int k) {
  double r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}
double bern(int n, int i, double x) { return binom(n, i) * std::pow(x, i) * std::pow(1 - x, n - i); }

// Solve M x = y for an n x n system by Gaussian elimination with partial pivoting.
void gauss_solve(std::vector<double> M, std::vector<double>& y, int n, int nrhs) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r) if (std::fabs(M[r * n + c]) > std::fabs(M[piv * n + c])) piv = r;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(M[c * n + k], M[piv * n + k]);
      for (int k = 0; k < nrhs; ++k) std::swap(y[c * nrhs + k], y[piv * nrhs + k]);
    }
    for (int r = c + 1; r < n; ++r) {
      double f = M[r * n + c] / M[c * n + c];
      for (int k = c; k < n; ++k) M[r * n + k] -= f * M[c * n + k];
      for (int k = 0; k < nrhs; ++k) y[r * nrhs + k] -= f * y[c * nrhs + k];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    for (int k = 0; k < nrhs; ++k) {
      double s = y[c * nrhs + k];
      for (int j = c + 1; j < n; ++j) s -= M[c * n + j] * y[j * nrhs + k];
      y[c * nrhs + k] = s / M[c * n + c];
    }
  }
}

// Evaluate the face surface at (a, b) with partials, through the volume.
void face_point(const Block& blk, int f, double a, double b, double S[3], double Sa[3], double Sb[3], double p[3]) {
  int nd, ad, bd;
  face_axes(f, nd, ad, bd);
  p[nd] = (f % 2) ? 1.0 : 0.0;
  p[ad] = a;
  p[bd] = b;
  double J[3][3];
  block_eval(blk, p, S, J, nullptr);
  for (int r = 0; r < 3; ++r) { Sa[r] = J[r][ad]; Sb[r] = J[r][bd]; }
}

// Bernstein control points of one piece by collocation at interior points:
// S(s,t) = sum_m sum_n B_m(s) B_n(t) c_mn on the piece, solved for c.
void build_piece(const Block& blk, Piece& pc) {
  const int na = pc.pa + 1, nb = pc.pb + 1;
  std::vector<double> sa(na), sb(nb);
  for (int i = 0; i < na; ++i) sa[i] = (i + 0.5) / na;
  for (int i = 0; i < nb; ++i) sb[i] = (i + 0.5) / nb;
  // values Y[i][j][3] at (sa_i, sb_j)
  std::vector<double> Y(na * nb * 3);
  for (int j = 0; j < nb; ++j) for (int i = 0; i < na; ++i) {
    double S[3], Sa[3], Sb[3], p[3];
    face_point(blk, pc.face, pc.a0 + sa[i] * (pc.a1 - pc.a0), pc.b0 + sb[j] * (pc.b1 - pc.b0), S, Sa, Sb, p);
    for (int r = 0; r < 3; ++r) Y[(j * na + i) * 3 + r] = S[r];
  }
  // along a: for each j, solve Ma c = y  (Ma[i][m] = B_m(sa_i))
  std::vector<double> Ma(na * na), Mb(nb * nb);
  for (int i = 0; i < na; ++i) for (int m = 0; m < na; ++m) Ma[i * na + m] = bern(pc.pa, m, sa[i]);
  for (int i = 0; i < nb; ++i) for (int m = 0; m < nb; ++m) Mb[i * nb + m] = bern(pc.pb, m, sb[i]);
  std::vector<double> T(na * nb * 3);
  for (int j = 0; j < nb; ++j) {
    std::vector<double> y(na * 3);
    for (int i = 0; i < na; ++i) for (int r = 0; r < 3; ++r) y[i * 3 + r] = Y[(j * na + i) * 3 + r];
    gauss_solve(Ma, y, na, 3);
    for (int i = 0; i < na; ++i) for (int r = 0; r < 3; ++r) T[(j * na + i) * 3 + r] = y[i * 3 + r];
  }
  pc.cp.assign(na * nb * 3, 0.0);
  for (int i = 0; i < na; ++i) {
    std::vector<double> y(nb * 3);
    for (int j = 0; j < nb; ++j) for (int r = 0; r < 3; ++r) y[j * 3 + r] = T[(j * na + i) * 3 + r];
    gauss_solve(Mb, y, nb, 3);
    for (int j = 0; j < nb; ++j) for (int r = 0; r < 3; ++r) pc.cp[(j * na + i) * 3 + r] = y[j * 3 + r];
  }
  for (int r = 0; r < 3; ++r) { pc.lo[r] = 1e300; pc.hi[r] = -1e300; }
  for (int q = 0; q < na * nb; ++q) for (int r = 0; r < 3; ++r) {
    pc.lo[r] = std::min(pc.lo[r], pc.cp[q * 3 + r]);
    pc.hi[r] = std::max(pc.hi[r], pc.cp[q * 3 + r]);
  }
}

struct Volume {
  std::vector<Block> blocks;
  std::vector<Piece> pieces;
  int mode = MODE_CP;
  double diag = 1.0;           // diagonal of the control-point bbox
};

std::vector<double> breakpoints(const Basis1D& b) {
  std::vector<double> u;
  for (double x : b.t) if (u.empty() || x > u.back()) u.push_back(x);
  return u;
}

// ---------------------------------------------------------------- rays
struct Camera {
  int ortho;
  double eye[3], target[3], up[3];
  double fovy_deg, ortho_height;
};

// Pixel (x, y), row 0 at the top, through the pixel centre.
void make_ray(const Camera& c, int W, int H, double px, double py, double o[3], double d[3]) {
  double f[3] = {c.target[0] - c.eye[0], c.target[1] - c.eye[1], c.target[2] - c.eye[2]};
  double nf = norm3(f);
  for (int i = 0; i < 3; ++i) f[i] /= nf;
  double r[3];
  cross3(f, c.up, r);
  double nr = norm3(r);
  for (int i = 0; i < 3; ++i) r[i] /= nr;
  double u[3];
  cross3(r, f, u);
  const double nx = (px + 0.5) / W * 2.0 - 1.0;
  const double ny = 1.0 - (py + 0.5) / H * 2.0;
  const double aspect = (double)W / H;
  if (c.ortho) {
    const double h2 = 0.5 * c.ortho_height;
    for (int i = 0; i < 3; ++i) {
      o[i] = c.eye[i] + nx * h2 * aspect * r[i] + ny * h2 * u[i];
      d[i] = f[i];
    }
  } else {
    const double th = std::tan(0.5 * c.fovy_deg * M_PI / 180.0);
    double dd[3];
    for (int i = 0; i < 3; ++i) { o[i] = c.eye[i]; dd[i] = f[i] + nx * th * aspect * r[i] + ny * th * u[i]; }
    double n = norm3(dd);
    for (int i = 0; i < 3; ++i) d[i] = dd[i] / n;
  }
}

// ------------------------------------------------------ intersections (§4.1)
struct Hit {
  double t;
  double p[3];
  int block, face, front;
};

// Newton on S(a,b) - o - t d = 0 inside one piece, from (a,b) = start.
bool polish_hit(const Volume& V, const Piece& pc, const double o[3], const double d[3],
                double a, double b, Hit& out) {
  const Block& blk = V.blocks[pc.block];
  double S[3], Sa[3], Sb[3], p[3];
  face_point(blk, pc.face, a, b, S, Sa, Sb, p);
  double t = dot3(d, S) - dot3(d, o);
  const double tol = 1e-13 * V.diag;
  bool ok = false;
  for (int it = 0; it < 40; ++it) {
    double F[3];
    for (int r = 0; r < 3; ++r) F[r] = S[r] - o[r] - t * d[r];
    if (norm3(F) <= tol) { ok = true; break; }
    double A[3][3], rhs[3], x[3];
    for (int r = 0; r < 3; ++r) { A[r][0] = Sa[r]; A[r][1] = Sb[r]; A[r][2] = -d[r]; rhs[r] = -F[r]; }
    if (!qr_solve3(A, rhs, x)) return false;
    a += x[0]; b += x[1]; t += x[2];
    // stay within a margin of the piece so the evaluation remains meaningful
    const double ma = 0.5 * (pc.a1 - pc.a0), mb = 0.5 * (pc.b1 - pc.b0);
    if (a < pc.a0 - ma || a > pc.a1 + ma || b < pc.b0 - mb || b > pc.b1 + mb) return false;
    face_point(blk, pc.face, a, b, S, Sa, Sb, p);
  }
  if (!ok) {
    double F[3];
    for (int r = 0; r < 3; ++r) F[r] = S[r] - o[r] - t * d[r];
    if (norm3(F) > 1e-10 * V.diag) return false;
  }
  const double ea = 1e-9 * (pc.a1 - pc.a0), eb = 1e-9 * (pc.b1 - pc.b0);
  if (a < pc.a0 - ea || a > pc.a1 + ea || b < pc.b0 - eb || b > pc.b1 + eb) return false;
  if (t <= 0) return false;
  int nd, ad, bd;
  face_axes(pc.face, nd, ad, bd);
  a = std::min(std::max(a, pc.a0), pc.a1);
  b = std::min(std::max(b, pc.b0), pc.b1);
  face_point(blk, pc.face, a, b, S, Sa, Sb, p);
  double n[3];
  cross3(Sa, Sb, n);
  if (pc.face % 2 == 0) for (int r = 0; r < 3; ++r) n[r] = -n[r];
  out.t = t;
  for (int r = 0; r < 3; ++r) out.p[r] = p[r];
  out.block = pc.block;
  out.face = pc.face;
  out.front = dot3(d, n) < 0 ? 1 : 0;
  return true;
}

void decasteljau_split(const std::vector<double>& cp, int na, int nb, int dir,
                       std::vector<double>& L, std::vector<double>& R) {
  // split at 0.5 along a (dir 0) or b (dir 1); cp layout [j][i][3], i along a
  L = cp;
  R = cp;
  const int n = dir == 0 ? na : nb;
  const int m = dir == 0 ? nb : na;
  for (int line = 0; line < m; ++line) {
    std::vector<double> w(n * 3);
    auto at = [&](int k) { return dir == 0 ? (line * na + k) : (k * na + line); };
    for (int k = 0; k < n; ++k) for (int r = 0; r < 3; ++r) w[k * 3 + r] = cp[at(k) * 3 + r];
    // left gets the first point of each level, right the last
    for (int r = 0; r < 3; ++r) { L[at(0) * 3 + r] = w[r]; R[at(n - 1) * 3 + r] = w[(n - 1) * 3 + r]; }
    for (int lev = 1; lev < n; ++lev) {
      for (int k = 0; k < n - lev; ++k)
        for (int r = 0; r < 3; ++r) w[k * 3 + r] = 0.5 * (w[k * 3 + r] + w[(k + 1) * 3 + r]);
      for (int r = 0; r < 3; ++r) {
        L[at(lev) * 3 + r] = w[r];
        R[at(n - 1 - lev) * 3 + r] = w[(n - 1 - lev) * 3 + r];
      }
    }
  }
}

void intersect_piece(const Volume& V, const Piece& pc, const double o[3], const double d[3],
                     const double e1[3], const double e2[3], std::vector<Hit>& hits) {
  const int na = pc.pa + 1, nb = pc.pb + 1;
  struct Node { std::vector<double> cp; double s0, s1, t0, t1; int depth; };
  std::vector<Node> stack;
  stack.push_back({pc.cp, 0.0, 1.0, 0.0, 1.0, 0});
  const double pad = 1e-12 * V.diag;
  const double stop = 1e-7 * V.diag;
  std::vector<Hit> local;
  while (!stack.empty()) {
    Node nd = std::move(stack.back());
    stack.pop_back();
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300, zmax = -1e300;
    for (int q = 0; q < na * nb; ++q) {
      double w[3] = {nd.cp[q * 3] - o[0], nd.cp[q * 3 + 1] - o[1], nd.cp[q * 3 + 2] - o[2]};
      double x = dot3(w, e1), y = dot3(w, e2), z = dot3(w, d);
      xmin = std::min(xmin, x); xmax = std::max(xmax, x);
      ymin = std::min(ymin, y); ymax = std::max(ymax, y);
      zmax = std::max(zmax, z);
    }
    if (xmin > pad || xmax < -pad || ymin > pad || ymax < -pad || zmax < 0) continue;
    const double ext = std::max(xmax - xmin, ymax - ymin);
    if (ext < stop || nd.depth >= 48) {
      const double sa = 0.5 * (nd.s0 + nd.s1), sb = 0.5 * (nd.t0 + nd.t1);
      Hit h;
      if (polish_hit(V, pc, o, d, pc.a0 + sa * (pc.a1 - pc.a0), pc.b0 + sb * (pc.b1 - pc.b0), h)) {
        bool dup = false;
        for (const Hit& q : local)
          if (std::fabs(q.t - h.t) <= 1e-9 * V.diag) { dup = true; break; }
        if (!dup) local.push_back(h);
      }
      continue;
    }
    // split along the longer parameter direction in G
    double la = 0, lb = 0;
    for (int j = 0; j < nb; ++j) {
      double a0[3] = {nd.cp[(j * na) * 3], nd.cp[(j * na) * 3 + 1], nd.cp[(j * na) * 3 + 2]};
      const double* a1 = &nd.cp[(j * na + na - 1) * 3];
      double v[3] = {a1[0] - a0[0], a1[1] - a0[1], a1[2] - a0[2]};
      la = std::max(la, norm3(v));
    }
    for (int i = 0; i < na; ++i) {
      const double* b0 = &nd.cp[i * 3];
      const double* b1 = &nd.cp[((nb - 1) * na + i) * 3];
      double v[3] = {b1[0] - b0[0], b1[1] - b0[1], b1[2] - b0[2]};
      lb = std::max(lb, norm3(v));
    }
    const int dir = la >= lb ? 0 : 1;
    Node Lh, Rh;
    decasteljau_split(nd.cp, na, nb, dir, Lh.cp, Rh.cp);
    Lh.depth = Rh.depth = nd.depth + 1;
    if (dir == 0) {
      const double m = 0.5 * (nd.s0 + nd.s1);
      Lh.s0 = nd.s0; Lh.s1 = m; Rh.s0 = m; Rh.s1 = nd.s1;
      Lh.t0 = Rh.t0 = nd.t0; Lh.t1 = Rh.t1 = nd.t1;
    } else {
      const double m = 0.5 * (nd.t0 + nd.t1);
      Lh.t0 = nd.t0; Lh.t1 = m; Rh.t0 = m; Rh.t1 = nd.t1;
      Lh.s0 = Rh.s0 = nd.s0; Lh.s1 = Rh.s1 = nd.s1;
    }
    stack.push_back(std::move(Rh));
    stack.push_back(std::move(Lh));
  }
  hits.insert(hits.end(), local.begin(), local.end());
}

bool ray_hits_box(const double o[3], const double d[3], const double lo[3], const double hi[3], double pad) {
  double t0 = -1e300, t1 = 1e300;
  for (int r = 0; r < 3; ++r) {
    if (d[r] == 0) {
      if (o[r] < lo[r] - pad || o[r] > hi[r] + pad) return false;
      continue;
    }
    double a = (lo[r] - pad - o[r]) / d[r], b = (hi[r] + pad - o[r]) / d[r];
    if (a > b) std::swap(a, b);
    t0 = std::max(t0, a);
    t1 = std::min(t1, b);
  }
  return t1 >= t0 && t1 >= 0;
}

// All hits of a ray, sorted by (t, block, front), with merged duplicates.
std::vector<Hit> ray_hits(const Volume& V, const double o[3], const double d[3]) {
  double e1[3], e2[3];
  {
    double a[3] = {1, 0, 0};
    if (std::fabs(d[0]) > 0.6) { a[0] = 0; a[1] = 1; }
    cross3(d, a, e1);
    double n = norm3(e1);
    for (int r = 0; r < 3; ++r) e1[r] /= n;
    cross3(d, e1, e2);
  }
  std::vector<Hit> hits;
  for (const Piece& pc : V.pieces) {
    if (!ray_hits_box(o, d, pc.lo, pc.hi, 1e-9 * V.diag)) continue;
    intersect_piece(V, pc, o, d, e1, e2, hits);
  }
  std::sort(hits.begin(), hits.end(), [](const Hit& a, const Hit& b) {
    if (a.t != b.t) return a.t < b.t;
    if (a.block != b.block) return a.block < b.block;
    return a.front < b.front;
  });
  // merge hits of one block with equal facing closer than 1e-9 diag
  std::vector<Hit> out;
  for (const Hit& h : hits) {
    bool dup = false;
    for (const Hit& q : out)
      if (q.block == h.block && q.front == h.front && std::fabs(q.t - h.t) <= 1e-9 * V.diag) { dup = true; break; }
    if (!dup) out.push_back(h);
  }
  return out;
}

// ---------------------------------------------------- Alg. 2 (§4.2)
struct Pair {
  int block;
  double t_in, t_out;
  double p_in[3], p_out[3];
};

// Blockwise depth pairing: take the nearest unused back-facing hit, then the
// nearest unused front-facing hit of the same block; emit the pair; mark both
// used; repeat until no unused back-facing hit is left.  A back-facing hit
// without a partner is marked used and counted.
std::vector<Pair> pair_hits(const std::vector<Hit>& h, int* unmatched) {
  std::vector<char> used(h.size(), 0);
  std::vector<Pair> out;
  int um = 0;
  for (;;) {
    int back = -1;
    for (size_t i = 0; i < h.size(); ++i)
      if (!used[i] && !h[i].front && (back < 0 || h[i].t < h[back].t)) back = (int)i;
    if (back < 0) break;
    int front = -1;
    for (size_t i = 0; i < h.size(); ++i)
      if (!used[i] && h[i].front && h[i].block == h[back].block && (front < 0 || h[i].t < h[front].t))
        front = (int)i;
    used[back] = 1;
    if (front < 0) { ++um; continue; }
    used[front] = 1;
    Pair p;
    p.block = h[back].block;
    p.t_in = h[front].t;
    p.t_out = h[back].t;
    for (int r = 0; r < 3; ++r) { p.p_in[r] = h[front].p[r]; p.p_out[r] = h[back].p[r]; }
    out.push_back(p);
  }
  for (size_t i = 0; i < h.size(); ++i) if (!used[i]) ++um;
  if (unmatched) *unmatched = um;
  return out;
}

// ----------------------------------------------- RF inversion (§5.1, Eqs. 6-7)
// Newton on F(p) = phi(p) - g with a QR solve, clamped to [0,1]^3, with a
// halving line search on ||F||.  Returns iterations (negative on failure).
int invert_point(const Block& b, const double g[3], const double p0[3], double tol, int maxit, double p[3]) {
  for (int r = 0; r < 3; ++r) p[r] = std::min(std::max(p0[r], 0.0), 1.0);
  double phi[3], J[3][3];
  block_eval(b, p, phi, J, nullptr);
  double F[3] = {phi[0] - g[0], phi[1] - g[1], phi[2] - g[2]};
  double nF = norm3(F);
  for (int it = 0; it < maxit; ++it) {
    if (nF <= tol) return it;
    double rhs[3] = {-F[0], -F[1], -F[2]}, dx[3];
    if (!qr_solve3(J, rhs, dx)) return -1;
    double lam = 1.0;
    bool moved = false;
    for (int ls = 0; ls < 30; ++ls) {
      double q[3];
      for (int r = 0; r < 3; ++r) q[r] = std::min(std::max(p[r] + lam * dx[r], 0.0), 1.0);
      double phq[3], Jq[3][3];
      block_eval(b, q, phq, Jq, nullptr);
      double Fq[3] = {phq[0] - g[0], phq[1] - g[1], phq[2] - g[2]};
      double nq = norm3(Fq);
      if (nq < nF || ls == 29) {
        for (int r = 0; r < 3; ++r) { p[r] = q[r]; F[r] = Fq[r]; }
        for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) J[r][c] = Jq[r][c];
        moved = nq < nF;
        nF = nq;
        break;
      }
      lam *= 0.5;
    }
    if (!moved) return nF <= tol ? it + 1 : -2;
  }
  return nF <= tol ? maxit : -3;
}

// ------------------------------------------------- pulled-back ODE (§5.2)
// W(p) solves J_phi(p) W = V(phi(p)), V(g) = d + c [(g_in - g) - <g_in - g, d> d].
bool ode_rhs(const Block& b, const double p[3], const double g_in[3], const double d[3], double c, double W[3]) {
  double phi[3], J[3][3];
  block_eval(b, p, phi, J, nullptr);
  double e[3] = {g_in[0] - phi[0], g_in[1] - phi[1], g_in[2] - phi[2]};
  const double ed = dot3(e, d);
  double Vv[3];
  for (int r = 0; r < 3; ++r) Vv[r] = d[r] + c * (e[r] - ed * d[r]);
  return qr_solve3(J, Vv, W);
}

// One implicit Euler step of §5.2: p_next = p + h W(p_next), solved for the
// increment z = p_next - p by Newton on G(z) = z - h W(p + z) with the exact
// Jacobian of G from differentiating J_phi G = J_phi z - h V(phi):
//   J_phi(x) J_G(z) = H_phi(x)[z - G(z)] + (I - h J_V) J_phi(x),  x = p + z,
// J_V = c (d d^T - I) (V(g) = d + c [(g_in - g) - <g_in - g, d> d]), and
// H_phi(x)[v]_{ij} = sum_k d^2 phi_i / dx_j dx_k v_k.  A Newton step then
// solves (J_phi J_G) dz = -J_phi G.  z starts at 0, so the first iteration
// evaluates the map at p itself.  Iterates may leave the parameter box (the
// map's boundary polynomials are continued there, so G stays smooth); the
// iteration stops once |dz|_inf <= tol and the new point p + z is clamped to
// [0,1]^3 (§5.4: the ray is followed along the boundary).  §5.4 also names
// the case in which Newton does not converge because it keeps trying to
// leave the block, and answers it by stepping along the boundary of the
// parameter domain: if Newton does not converge within max_it iterations
// (or meets a singular system: the map is degenerate near the ray), the step
// is the explicit Euler step p + h W(p) from the first iteration's
// evaluation, clamped to [0,1]^3 (a step that moves along the boundary where
// W points out of the box).  ev(x, phi, J, H) evaluates the map.  Returns the
// iterations, or -1 if the step took the boundary step.
template <class Eval>
int irk1_step(Eval ev, const double p[3], double h, const double g_in[3], const double d[3], double c,
              double tol, int max_it, double pn[3]) {
  double z[3] = {0, 0, 0}, v0[3] = {0, 0, 0};
  bool conv = false;
  int it = 0;
  for (; it < max_it; ++it) {
    double x[3];
    for (int r = 0; r < 3; ++r) x[r] = p[r] + z[r];
    double phi[3], J[3][3], H[3][3][3];
    ev(x, phi, J, H);
    double e[3] = {g_in[0] - phi[0], g_in[1] - phi[1], g_in[2] - phi[2]};
    const double ed = dot3(e, d);
    double Vv[3], W[3];
    for (int r = 0; r < 3; ++r) Vv[r] = d[r] + c * (e[r] - ed * d[r]);
    if (!qr_solve3(J, Vv, W)) break;
    double G[3], v[3];
    for (int r = 0; r < 3; ++r) {
      v[r] = h * W[r];                  // z - G(z)
      G[r] = z[r] - v[r];
    }
    if (it == 0)
      for (int r = 0; r < 3; ++r) v0[r] = v[r];
    // M = H[v] + (I - h J_V) J,  (I - h J_V) = (1 + h c) I - h c d d^T
    double M[3][3], JG[3];
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) {
        double hv = 0;
        for (int k = 0; k < 3; ++k) hv += H[i][j][k] * v[k];
        double aj = 0;
        for (int k = 0; k < 3; ++k) {
          const double A = (i == k ? 1.0 + h * c : 0.0) - h * c * d[i] * d[k];
          aj += A * J[k][j];
        }
        M[i][j] = hv + aj;
      }
      JG[i] = -(J[i][0] * G[0] + J[i][1] * G[1] + J[i][2] * G[2]);
    }
    double dz[3];
    if (!qr_solve3(M, JG, dz)) break;
    for (int r = 0; r < 3; ++r) z[r] += dz[r];
    if (std::max(std::fabs(dz[0]), std::max(std::fabs(dz[1]), std::fabs(dz[2]))) <= tol) {
      ++it;
      conv = true;
      break;
    }
  }
  for (int r = 0; r < 3; ++r) pn[r] = std::min(std::max(p[r] + (conv ? z[r] : v0[r]), 0.0), 1.0);
  return conv ? it : -1;
}

// Runge-Kutta-Fehlberg 4(5) coefficients (Fehlberg 1969), 5th-order solution
// propagated, as the paper's "RKF".
const double F45_c[6] = {0, 1.0/4, 3.0/8, 12.0/13, 1.0, 1.0/2};
const double F45_a[6][5] = {
  {0, 0, 0, 0, 0},
  {1.0/4, 0, 0, 0, 0},
  {3.0/32, 9.0/32, 0, 0, 0},
  {1932.0/2197, -7200.0/2197, 7296.0/2197, 0, 0},
  {439.0/216, -8.0, 3680.0/513, -845.0/4104, 0},
  {-8.0/27, 2.0, -3544.0/2565, 1859.0/4104, -11.0/40}};
const double F45_b5[6] = {16.0/135, 0, 6656.0/12825, 28561.0/56430, -9.0/50, 2.0/55};
const double F45_b4[6] = {25.0/216, 0, 1408.0/2565, 2197.0/4104, -1.0/5, 0};

// One RKF45 step of size h from p; returns the error estimate (inf-norm).
double rkf45_step(const Block& b, const double p[3], double h, const double g_in[3], const double d[3],
                  double c, double pn[3], bool* ok) {
  double k[6][3];
  *ok = true;
  for (int s = 0; s < 6; ++s) {
    double q[3];
    for (int r = 0; r < 3; ++r) {
      double acc = p[r];
      for (int j = 0; j < s; ++j) acc += h * F45_a[s][j] * k[j][r];
      q[r] = std::min(std::max(acc, 0.0), 1.0);
    }
    if (!ode_rhs(b, q, g_in, d, c, k[s])) { *ok = false; return 1e300; }
  }
  double err = 0;
  for (int r = 0; r < 3; ++r) {
    double y5 = p[r], y4 = p[r];
    for (int s = 0; s < 6; ++s) { y5 += h * F45_b5[s] * k[s][r]; y4 += h * F45_b4[s] * k[s][r]; }
    pn[r] = std::min(std::max(y5, 0.0), 1.0);
    err = std::max(err, std::fabs(y5 - y4));
  }
  return err;
}

// ---------------------------------------------- compositing (Alg. 1, §3.2.1)
struct TF {
  std::vector<double> r, rgba;   // [n], [n][4]
  double sigma = 1, lo = 0, hi = 1;
};

void tf_lookup(const TF& tf, double x, double out[4]) {
  const int n = (int)tf.r.size();
  if (x <= tf.r[0]) { for (int c = 0; c < 4; ++c) out[c] = tf.rgba[c]; return; }
  if (x >= tf.r[n - 1]) { for (int c = 0; c < 4; ++c) out[c] = tf.rgba[(n - 1) * 4 + c]; return; }
  int i = 0;
  while (i + 1 < n - 1 && !(x < tf.r[i + 1])) ++i;
  const double w = tf.r[i + 1] - tf.r[i];
  const double f = w > 0 ? (x - tf.r[i]) / w : 1.0;
  for (int c = 0; c < 4; ++c) out[c] = (1 - f) * tf.rgba[i * 4 + c] + f * tf.rgba[(i + 1) * 4 + c];
}

double norm_scalar(const TF& tf, double rho) {
  double x = (rho - tf.lo) / (tf.hi - tf.lo);
  return std::min(std::max(x, 0.0), 1.0);
}

struct Accum { double C[3] = {0, 0, 0}; double a = 0; bool done = false; };

// One interval [s_{j-1}, s_j] of length ds_i with end scalars rho0, rho1:
// K midpoint sub-samples of the linear interpolant (supersampling), each
// composited front to back with T = exp(-sigma A ds_i / K).
void composite_interval(const TF& tf, int K, double early, double rho0, double rho1, double dsi, Accum& acc) {
  if (acc.done) return;
  for (int k = 1; k <= K; ++k) {
    const double rk = rho0 + (k - 0.5) / K * (rho1 - rho0);
    double c[4];
    tf_lookup(tf, norm_scalar(tf, rk), c);
    const double T = std::exp(-tf.sigma * c[3] * dsi / K);
    const double w = (1 - T) * (1 - acc.a);
    for (int r = 0; r < 3; ++r) acc.C[r] += w * c[r];
    acc.a += w;
  }
  if (acc.a >= early) acc.done = true;
}

struct Params {
  double ds; int K; double c; double early;
  int method;          // 0 = RF per sample, 1 = RKF45 ODE, 10 + k = fixed-step tableau k (one step per interval),
                       // 17 = implicit Euler (one step per interval)
  double newton_tol;   // relative to diag
  double rk_tol;
  double near_clip;    // > 0: near plane at this distance along the view direction
  int n_cut;           // cutting planes: points g with n.g + w > 0 are cut away
  double cut[4][4];
};

struct Tableau { int s; double a[6][6]; double b[6]; };
Tableau tableau(int method);

struct PixelStats { int npairs = 0, unmatched = 0, newton_fail = 0, nsamples = 0, rk_steps = 0, shrunk = 0; };

// Samples s_j = j ds (j = 0..floor(L/ds)) plus L when it lies more than
// 1e-12 diag beyond the last one.
std::vector<double> sample_points(double L, double ds, double diag) {
  std::vector<double> s;
  if (!(L > 0)) return s;
  const long n = (long)std::floor(L / ds);
  for (long j = 0; j <= n; ++j) s.push_back(j * ds);
  if (L - s.back() > 1e-12 * diag) s.push_back(L);
  return s;
}

void render_pair(const Volume& V, const TF& tf, const Params& P, const double o[3], const double d[3],
                 const Pair& pr, Accum& acc, PixelStats& st, std::vector<double>* trace) {
  const Block& b = V.blocks[pr.block];
  const double L = pr.t_out - pr.t_in;
  std::vector<double> s = sample_points(L, P.ds, V.diag);
  if (s.empty()) return;
  double g_in[3];
  for (int r = 0; r < 3; ++r) g_in[r] = o[r] + pr.t_in * d[r];
  double p[3] = {pr.p_in[0], pr.p_in[1], pr.p_in[2]};
  double rho_prev = 0;
  double h = P.ds;
  for (size_t j = 0; j < s.size(); ++j) {
    if (P.method == 0 || j == 0) {
      double g[3];
      for (int r = 0; r < 3; ++r) g[r] = o[r] + (pr.t_in + s[j]) * d[r];
      double q[3];
      int it = invert_point(b, g, p, P.newton_tol * V.diag, 50, q);
      if (it < 0) ++st.newton_fail;
      for (int r = 0; r < 3; ++r) p[r] = q[r];
    } else if (P.method >= 11 && P.method <= 16) {
      // one step of a fixed-step explicit method (the paper's RK family,
      // §5.3) from s_{j-1} to s_j; stage points and the result clamped to
      // [0,1]^3 (§5.4)
      const Tableau T = tableau(P.method - 10);
      const double hh = s[j] - s[j - 1];
      double k[6][3];
      bool ok = true;
      for (int st2 = 0; st2 < T.s && ok; ++st2) {
        double q[3];
        for (int r = 0; r < 3; ++r) {
          double acc2 = p[r];
          for (int m = 0; m < st2; ++m) acc2 += hh * T.a[st2][m] * k[m][r];
          q[r] = std::min(std::max(acc2, 0.0), 1.0);
        }
        ok = ode_rhs(b, q, g_in, d, P.c, k[st2]);
      }
      if (!ok) {
        ++st.newton_fail;
      } else {
        for (int r = 0; r < 3; ++r) {
          double acc2 = p[r];
          for (int st2 = 0; st2 < T.s; ++st2) acc2 += hh * T.b[st2] * k[st2][r];
          p[r] = std::min(std::max(acc2, 0.0), 1.0);
        }
        ++st.rk_steps;
      }
    } else if (P.method == 17) {
      // one implicit Euler step (§5.2) from s_{j-1} to s_j
      const double hh = s[j] - s[j - 1];
      double pn[3];
      auto ev = [&](const double x[3], double phi[3], double J[3][3], double H[3][3][3]) {
        block_eval2(b, x, phi, J, H);
      };
      // G(z) = 0 solved to |dz|_inf <= 1e-13 (parameter space), at most 50
      // Newton iterations; a step that does not converge takes the §5.4
      // boundary step and is counted
      if (irk1_step(ev, p, hh, g_in, d, P.c, 1e-13, 50, pn) < 0) ++st.newton_fail;
      for (int r = 0; r < 3; ++r) p[r] = pn[r];
      ++st.rk_steps;
    } else {
      // integrate the pulled-back ODE from s_{j-1} to s_j with RKF45
      double sc = s[j - 1];
      int guard = 0;
      while (sc < s[j] && guard++ < 100000) {
        const bool last = h >= s[j] - sc;          // this step lands on s_j
        const double hh = last ? s[j] - sc : h;
        bool ok;
        double pn[3];
        double err = rkf45_step(b, p, hh, g_in, d, P.c, pn, &ok);
        if (!ok) { ++st.newton_fail; break; }
        ++st.rk_steps;
        const double fac = err > 0 ? 0.9 * std::pow(P.rk_tol / err, 0.2) : 5.0;
        if (err <= P.rk_tol || hh <= 1e-12) {
          for (int r = 0; r < 3; ++r) p[r] = pn[r];
          sc = last ? s[j] : sc + hh;
          const double hn = hh * std::min(5.0, std::max(0.2, fac));
          h = last ? std::max(h, hn) : hn;          // a shortened step does not shrink h
        } else {
          h = hh * std::max(0.2, fac);
        }
      }
    }
    double phi[3], J[3][3], rc;
    block_eval(b, p, phi, J, &rc);
    const double rho = scalar_of(b, V.mode, p, J, rc);
    if (trace) {
      trace->push_back(s[j]);
      for (int r = 0; r < 3; ++r) trace->push_back(p[r]);
      trace->push_back(rho);
    }
    ++st.nsamples;
    if (j > 0) composite_interval(tf, P.K, P.early, rho_prev, rho, s[j] - s[j - 1], acc);
    rho_prev = rho;
    if (acc.done) break;
  }
}

// Cutting and near-clip planes (§5.5) on the depth-sorted intersections of
// one ray, before compositing.  Near plane: hits nearer than it are dropped,
// and a block whose nearest remaining hit is an exit gets an entry on the
// plane (the eye side of the plane lies inside that block).  Cutting plane:
// every entry/exit segment is shortened to the part with n.g + w <= 0.  An
// end that moves onto a plane gets its parameter point by Newton (§5.1) from
// the chord between the segment's original ends (from the exit for a new
// entry); a segment whose new end does not invert inside its block is
// dropped.
std::vector<Pair> clip_pairs(const Volume& V, const Params& P, const Camera& cam, const double o[3],
                             const double d[3], std::vector<Hit> hits, int* unmatched) {
  const double NaN = std::numeric_limits<double>::quiet_NaN();
  double t_near = 0;
  if (P.near_clip > 0) {
    double f[3] = {cam.target[0] - cam.eye[0], cam.target[1] - cam.eye[1], cam.target[2] - cam.eye[2]};
    const double nf = norm3(f);
    for (int r = 0; r < 3; ++r) f[r] /= nf;
    t_near = P.near_clip / dot3(d, f);
    std::vector<Hit> kept;
    for (const Hit& h : hits)
      if (h.t >= t_near) kept.push_back(h);
    hits.swap(kept);
    const size_t n0 = hits.size();
    for (size_t i = 0; i < n0; ++i) {
      bool nearest = true;
      for (size_t k = 0; k < n0; ++k)
        if (hits[k].block == hits[i].block && (hits[k].t < hits[i].t || (hits[k].t == hits[i].t && k < i)))
          nearest = false;
      if (nearest && !hits[i].front) {
        Hit e = hits[i];
        e.t = t_near;
        e.front = 1;
        e.face = -1;
        for (int r = 0; r < 3; ++r) e.p[r] = NaN;          // solved below
        hits.push_back(e);
      }
    }
  }
  std::vector<Pair> pairs = pair_hits(hits, unmatched);
  std::vector<Pair> out;
  const double tol = P.newton_tol * V.diag;
  for (Pair pr : pairs) {
    const double t_in0 = pr.t_in, t_out0 = pr.t_out;
    double t0 = pr.t_in, t1 = pr.t_out;
    for (int k = 0; k < P.n_cut; ++k) {
      const double* c = P.cut[k];
      const double fo = c[0] * o[0] + c[1] * o[1] + c[2] * o[2] + c[3];
      const double fd = c[0] * d[0] + c[1] * d[1] + c[2] * d[2];
      if (fd == 0) {
        if (fo > 0) t1 = t0 - 1;                           // all of the segment is cut away
        continue;
      }
      const double tc = -fo / fd;
      if (fd > 0) t1 = std::min(t1, tc);
      else t0 = std::max(t0, tc);
    }
    if (!(t1 > t0)) continue;
    const bool new_in = std::isnan(pr.p_in[0]) || t0 > t_in0, new_out = t1 < t_out0;
    const Block& b = V.blocks[pr.block];
    bool ok = true;
    double pin[3], pout[3];
    for (int r = 0; r < 3; ++r) { pin[r] = pr.p_in[r]; pout[r] = pr.p_out[r]; }
    if (new_in) {
      double g[3], guess[3];
      for (int r = 0; r < 3; ++r) g[r] = o[r] + t0 * d[r];
      const double w = (t_out0 > t_in0) ? (t0 - t_in0) / (t_out0 - t_in0) : 0.0;
      for (int r = 0; r < 3; ++r)
        guess[r] = std::isnan(pr.p_in[0]) ? pr.p_out[r] : pr.p_in[r] + w * (pr.p_out[r] - pr.p_in[r]);
      ok = invert_point(b, g, guess, tol, 100, pin) >= 0;
    }
    if (ok && new_out) {
      double g[3], guess[3];
      for (int r = 0; r < 3; ++r) g[r] = o[r] + t1 * d[r];
      const double w = (t_out0 > t_in0) ? (t1 - t_in0) / (t_out0 - t_in0) : 1.0;
      for (int r = 0; r < 3; ++r)
        guess[r] = std::isnan(pr.p_in[0]) ? pr.p_out[r] : pr.p_in[r] + w * (pr.p_out[r] - pr.p_in[r]);
      ok = invert_point(b, g, guess, tol, 100, pout) >= 0;
    }
    if (!ok) continue;
    pr.t_in = t0;
    pr.t_out = t1;
    for (int r = 0; r < 3; ++r) { pr.p_in[r] = pin[r]; pr.p_out[r] = pout[r]; }
    out.push_back(pr);
  }
  return out;
}

// Mean of |det J| over the parameter box, i.e. the integral of |det J| over
// [0,1]^3: 5-point Gauss-Legendre in every knot span of every direction
// (exact for the polynomial det J of a block up to degree 3 per direction).
double mean_abs_det(const Block& b) {
  const double gx[5] = {-0.9061798459386640, -0.5384693101056831, 0.0, 0.5384693101056831, 0.9061798459386640};
  const double gw[5] = {0.2369268850561891, 0.4786286704993665, 0.5688888888888889, 0.4786286704993665,
                        0.2369268850561891};
  std::vector<double> br[3];
  for (int k = 0; k < 3; ++k) br[k] = breakpoints(b.B[k]);
  double sum = 0;
  for (size_t i = 0; i + 1 < br[0].size(); ++i)
    for (size_t j = 0; j + 1 < br[1].size(); ++j)
      for (size_t k = 0; k + 1 < br[2].size(); ++k) {
        const double h[3] = {br[0][i + 1] - br[0][i], br[1][j + 1] - br[1][j], br[2][k + 1] - br[2][k]};
        for (int a = 0; a < 5; ++a)
          for (int c = 0; c < 5; ++c)
            for (int e = 0; e < 5; ++e) {
              const double p[3] = {br[0][i] + 0.5 * h[0] * (gx[a] + 1), br[1][j] + 0.5 * h[1] * (gx[c] + 1),
                                   br[2][k] + 0.5 * h[2] * (gx[e] + 1)};
              double phi[3], J[3][3];
              block_eval(b, p, phi, J, nullptr);
              sum += gw[a] * gw[c] * gw[e] * 0.125 * h[0] * h[1] * h[2] * std::fabs(det3(J));
            }
      }
  return sum;
}

// §5.4's first case: where the ray is outside the block just behind an entry
// (an entry that only touches the block's boundary, so that the moved entry
// point has no preimage in the block), the entry steps along the ray until
// the ray is inside the block again: 16 probes t0 + k (t1 - t0) / 16 with
// Newton from the chord guesses, then 50 bisections between the last probe
// outside and the first inside.  Returns false if no probe is inside.
bool walk_into_block(const Block& b, const double o[3], const double d[3], double t0, double t1,
                     const double p0[3], const double p1[3], double tol, double* t_new, double p_new[3]) {
  double t_lo = t0, t_hi = 0, p_hi[3], g[3], x[3];
  bool found = false;
  for (int k = 1; k <= 16 && !found; ++k) {
    const double tk = t0 + (t1 - t0) * k / 16.0;
    double x0[3];
    for (int r = 0; r < 3; ++r) {
      x0[r] = p0[r] + (p1[r] - p0[r]) * k / 16.0;
      g[r] = o[r] + tk * d[r];
    }
    if (invert_point(b, g, x0, tol, 100, x) >= 0) {
      found = true;
      t_hi = tk;
      for (int r = 0; r < 3; ++r) p_hi[r] = x[r];
    } else {
      t_lo = tk;
    }
  }
  if (!found) return false;
  for (int it = 0; it < 50; ++it) {
    const double tm = 0.5 * (t_lo + t_hi);
    for (int r = 0; r < 3; ++r) g[r] = o[r] + tm * d[r];
    if (invert_point(b, g, p_hi, tol, 100, x) >= 0) {
      t_hi = tm;
      for (int r = 0; r < 3; ++r) p_hi[r] = x[r];
    } else {
      t_lo = tm;
    }
  }
  *t_new = t_hi;
  for (int r = 0; r < 3; ++r) p_new[r] = p_hi[r];
  return true;
}

// §5.4, singular Jacobian at the entry point (Eq. 22): where |det J(p_in)|
// is below tau_det = 1e-6 times the block's mean |det J|, neither Newton nor
// the ODE's linear system can start at the entry, so the block is "shrunk":
// the entry moves a distance delta = 1e-4 diag along the ray,
// g~_in = g_in + delta d (reading: the paper adds the step to the entry in
// G, so its direction is the ray's), and p~_in solves phi(p) = g~_in by
// Newton (§5.1) started at x_0 = p_in + eps (p_out - p_in) / |p_out - p_in|
// with eps = 1e-4 (Eq. 22).  If the moved entry has no preimage in the block
// (the entry only touched its boundary), the entry walks along the ray into
// the block (walk_into_block).  A pair no longer than delta, or that never
// enters its block, is dropped.  Returns the pairs;
// *shrunk counts the moved entries, *dropped the dropped pairs.
std::vector<Pair> shrink_singular_entries(const Volume& V, const double o[3], const double d[3], double newton_tol,
                                          const std::vector<Pair>& in, int* shrunk, int* dropped) {
  std::vector<Pair> out;
  const double delta = 1e-4 * V.diag, eps = 1e-4;
  for (Pair pr : in) {
    const Block& b = V.blocks[pr.block];
    double phi[3], J[3][3];
    block_eval(b, pr.p_in, phi, J, nullptr);
    if (!(std::fabs(det3(J)) < 1e-6 * b.mean_abs_det)) {
      out.push_back(pr);
      continue;
    }
    if (shrunk) ++*shrunk;
    if (!(pr.t_out - pr.t_in > delta)) {
      if (dropped) ++*dropped;
      continue;
    }
    double dir[3] = {pr.p_out[0] - pr.p_in[0], pr.p_out[1] - pr.p_in[1], pr.p_out[2] - pr.p_in[2]};
    const double nd = norm3(dir);
    double x0[3], g[3], q[3];
    for (int r = 0; r < 3; ++r) x0[r] = pr.p_in[r] + (nd > 0 ? eps * dir[r] / nd : 0.0);
    pr.t_in += delta;
    for (int r = 0; r < 3; ++r) g[r] = o[r] + pr.t_in * d[r];
    if (invert_point(b, g, x0, newton_tol * V.diag, 100, q) < 0 &&
        !walk_into_block(b, o, d, pr.t_in, pr.t_out, pr.p_in, pr.p_out, newton_tol * V.diag, &pr.t_in, q)) {
      if (dropped) ++*dropped;
      continue;
    }
    for (int r = 0; r < 3; ++r) pr.p_in[r] = q[r];
    out.push_back(pr);
  }
  return out;
}

void render_pixel(const Volume& V, const TF& tf, const Params& P, const Camera& cam, int W, int H,
                  int x, int y, double out[4], PixelStats& st) {
  double o[3], d[3];
  make_ray(cam, W, H, x, y, o, d);
  std::vector<Hit> hits = ray_hits(V, o, d);
  int um = 0;
  std::vector<Pair> pairs = (P.near_clip > 0 || P.n_cut > 0) ? clip_pairs(V, P, cam, o, d, hits, &um)
                                                              : pair_hits(hits, &um);
  pairs = shrink_singular_entries(V, o, d, P.newton_tol, pairs, &st.shrunk, &um);
  st.npairs = (int)pairs.size();
  st.unmatched = um;
  Accum acc;
  for (const Pair& pr : pairs) {
    render_pair(V, tf, P, o, d, pr, acc, st, nullptr);
    if (acc.done) break;
  }
  out[0] = acc.C[0]; out[1] = acc.C[1]; out[2] = acc.C[2]; out[3] = acc.a;
}

// ------------------------------------- Table 1 harness (§5.3, convergence)
// phi(x,y,z) = (2x, y + 0.3 (1-x) sin(10 pi x), z), p_in = (0,0.3,.5), p_out = (1,0.7,.5).
void t1_map(const double p[3], double phi[3], double J[3][3]) {
  const double x = p[0], y = p[1], z = p[2];
  const double s = std::sin(10 * M_PI * x), c = std::cos(10 * M_PI * x);
  phi[0] = 2 * x;
  phi[1] = y + 0.3 * (1 - x) * s;
  phi[2] = z;
  J[0][0] = 2; J[0][1] = 0; J[0][2] = 0;
  J[1][0] = -0.3 * s + 0.3 * (1 - x) * 10 * M_PI * c; J[1][1] = 1; J[1][2] = 0;
  J[2][0] = 0; J[2][1] = 0; J[2][2] = 1;
}

// Second derivatives of the analytic map: only d^2 phi_1 / dx^2 is non-zero.
void t1_map2(const double p[3], double phi[3], double J[3][3], double H[3][3][3]) {
  t1_map(p, phi, J);
  for (int r = 0; r < 3; ++r)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) H[r][a][b] = 0;
  const double x = p[0], w = 10 * M_PI;
  H[1][0][0] = -0.6 * w * std::cos(w * x) - 0.3 * (1 - x) * w * w * std::sin(w * x);
}

void t1_rhs(const double p[3], const double g_in[3], const double d[3], double c, double W[3]) {
  double phi[3], J[3][3];
  t1_map(p, phi, J);
  double e[3] = {g_in[0] - phi[0], g_in[1] - phi[1], g_in[2] - phi[2]};
  const double ed = dot3(e, d);
  double Vv[3];
  for (int r = 0; r < 3; ++r) Vv[r] = d[r] + c * (e[r] - ed * d[r]);
  qr_solve3(J, Vv, W);
}

Tableau tableau(int method) {
  Tableau T;
  std::memset(&T, 0, sizeof(T));
  switch (method) {
    case 1:  // explicit Euler
      T.s = 1; T.b[0] = 1; break;
    case 2:  // explicit midpoint
      T.s = 2; T.a[1][0] = 0.5; T.b[1] = 1; break;
    case 3:  // Kutta's third-order method
      T.s = 3; T.a[1][0] = 0.5; T.a[2][0] = -1; T.a[2][1] = 2;
      T.b[0] = 1.0/6; T.b[1] = 2.0/3; T.b[2] = 1.0/6; break;
    case 4:  // classic RK4
      T.s = 4; T.a[1][0] = 0.5; T.a[2][1] = 0.5; T.a[3][2] = 1;
      T.b[0] = 1.0/6; T.b[1] = 1.0/3; T.b[2] = 1.0/3; T.b[3] = 1.0/6; break;
    case 5:  // Kutta's 3/8 rule
      T.s = 4; T.a[1][0] = 1.0/3; T.a[2][0] = -1.0/3; T.a[2][1] = 1; T.a[3][0] = 1; T.a[3][1] = -1; T.a[3][2] = 1;
      T.b[0] = 1.0/8; T.b[1] = 3.0/8; T.b[2] = 3.0/8; T.b[3] = 1.0/8; break;
    case 6:  // Fehlberg, fifth-order weights
      T.s = 6;
      for (int i = 0; i < 6; ++i) for (int j = 0; j < 5; ++j) T.a[i][j] = F45_a[i][j];
      for (int i = 0; i < 6; ++i) T.b[i] = F45_b5[i];
      break;
    default: T.s = 0;
  }
  return T;
}

}  // namespace

// =================================================================== C ABI
extern "C" {

typedef struct {
  int degree[3];
  int n_cp[3];
  const double* knots[3];
  const double* geom_cp;
  const double* scalar_cp;
  const double* disp_cp;       // [nw][nv][nu][3], the displacement for MODE_VONMISES
} orc_block_desc;

typedef struct {
  int ortho;
  double eye[3], target[3], up[3];
  double fovy_deg, ortho_height;
} orc_camera;

typedef struct {
  int n_knots;
  const double* r;
  const double* rgba;
  double sigma, lo, hi;
} orc_tf;

typedef struct {
  double ds; int supersample_k; double c; double early_alpha;
  int method; double newton_tol; double rk_tol;
  double near_clip; int n_cut; double cut[4][4];
} orc_params;

typedef struct { double t; double p[3]; int block, face, front; } orc_hit;
typedef struct { int block; double t_in, t_out; double p_in[3], p_out[3]; } orc_pair;
typedef struct { int npairs, unmatched, newton_fail, nsamples, rk_steps, shrunk; } orc_pixel_stats;

void* orc_volume_create(const orc_block_desc* blocks, int n_blocks, int mode, char* err, int errlen) {
  auto fail = [&](const char* m) -> void* {
    if (err && errlen > 0) std::snprintf(err, errlen, "%s", m);
    return nullptr;
  };
  if (!blocks || n_blocks <= 0) return fail("no blocks");
  if (mode < 0 || mode > 3) return fail("bad scalar mode");
  Volume* V = new Volume();
  V->mode = mode;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int bi = 0; bi < n_blocks; ++bi) {
    const orc_block_desc& d = blocks[bi];
    Block b;
    size_t ncp = 1;
    for (int k = 0; k < 3; ++k) {
      const int p = d.degree[k], n = d.n_cp[k];
      if (p < 1 || n < p + 1 || !d.knots[k]) { delete V; return fail("bad degree/n_cp/knots"); }
      const int nk = n + p + 1;
      std::vector<double> t(d.knots[k], d.knots[k] + nk);
      for (int i = 1; i < nk; ++i) if (t[i] < t[i - 1]) { delete V; return fail("knots not non-decreasing"); }
      const double a = t[0], z = t[nk - 1];
      if (!(z > a)) { delete V; return fail("empty knot range"); }
      for (double& x : t) x = (x - a) / (z - a);
      b.B[k].t = t; b.B[k].p = p; b.B[k].n = n;
      ncp *= n;
    }
    if (!d.geom_cp) { delete V; return fail("no geometry"); }
    b.geom.assign(d.geom_cp, d.geom_cp + 3 * ncp);
    if (mode == MODE_CP) {
      if (!d.scalar_cp) { delete V; return fail("scalar mode CP needs scalar control points"); }
      b.scal.assign(d.scalar_cp, d.scalar_cp + ncp);
    }
    if (mode == MODE_VONMISES) {
      if (!d.disp_cp) { delete V; return fail("scalar mode VONMISES needs displacement control points"); }
      b.disp.assign(d.disp_cp, d.disp_cp + 3 * ncp);
    }
    for (size_t q = 0; q < ncp; ++q) for (int r = 0; r < 3; ++r) {
      lo[r] = std::min(lo[r], b.geom[3 * q + r]);
      hi[r] = std::max(hi[r], b.geom[3 * q + r]);
    }
    V->blocks.push_back(std::move(b));
  }
  double dg[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
  V->diag = norm3(dg);
  for (Block& b : V->blocks) b.mean_abs_det = mean_abs_det(b);
  // pieces of the 6 faces of every block
  for (int bi = 0; bi < n_blocks; ++bi) {
    const Block& b = V->blocks[bi];
    for (int f = 0; f < 6; ++f) {
      int nd, ad, bd;
      face_axes(f, nd, ad, bd);
      std::vector<double> ua = breakpoints(b.B[ad]), ub = breakpoints(b.B[bd]);
      for (size_t i = 0; i + 1 < ua.size(); ++i) for (size_t j = 0; j + 1 < ub.size(); ++j) {
        Piece pc;
        pc.block = bi; pc.face = f;
        pc.a0 = ua[i]; pc.a1 = ua[i + 1]; pc.b0 = ub[j]; pc.b1 = ub[j + 1];
        pc.pa = b.B[ad].p; pc.pb = b.B[bd].p;
        build_piece(b, pc);
        V->pieces.push_back(std::move(pc));
      }
    }
  }
  return V;
}

void orc_volume_destroy(void* v) { delete (Volume*)v; }

double orc_volume_diag(void* v) { return ((Volume*)v)->diag; }
int orc_volume_npieces(void* v) { return (int)((Volume*)v)->pieces.size(); }

// phi [n][3], J [n][3][3], rho [n] (cp scalar or derived per the volume mode)
int orc_eval(void* v, int block, int n, const double* p, double* phi, double* J, double* rho) {
  Volume* V = (Volume*)v;
  if (block < 0 || block >= (int)V->blocks.size()) return -1;
  for (int i = 0; i < n; ++i) {
    double f[3], Jm[3][3], rc = 0;
    block_eval(V->blocks[block], p + 3 * i, f, Jm, &rc);
    if (phi) for (int r = 0; r < 3; ++r) phi[3 * i + r] = f[r];
    if (J) for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) J[9 * i + 3 * r + c] = Jm[r][c];
    if (rho) rho[i] = scalar_of(V->blocks[block], V->mode, p + 3 * i, Jm, rc);
  }
  return 0;
}

// 1-D basis values/derivatives of one direction of one block (for pins).
// phi [n][3], J [n][3][3] and the Hessian H [n][3][3][3] (H[r][a][b] =
// d^2 phi_r / dp_a dp_b) at n points of a block.
int orc_eval2(void* v, int block, int n, const double* p, double* phi, double* J, double* H) {
  Volume* V = (Volume*)v;
  if (block < 0 || block >= (int)V->blocks.size()) return -1;
  for (int i = 0; i < n; ++i) {
    double f[3], Jm[3][3], Hm[3][3][3];
    block_eval2(V->blocks[block], p + 3 * i, f, Jm, Hm);
    for (int r = 0; r < 3; ++r) {
      phi[3 * i + r] = f[r];
      for (int a = 0; a < 3; ++a) {
        J[9 * i + 3 * r + a] = Jm[r][a];
        for (int b = 0; b < 3; ++b) H[27 * i + 9 * r + 3 * a + b] = Hm[r][a][b];
      }
    }
  }
  return 0;
}

int orc_basis(void* v, int block, int dir, int n, const double* x, double* N, double* dN) {
  Volume* V = (Volume*)v;
  const Basis1D& B = V->blocks[block].B[dir];
  std::vector<double> a, b;
  for (int i = 0; i < n; ++i) {
    B.eval(x[i], a, b);
    for (int k = 0; k < B.n; ++k) { N[i * B.n + k] = a[k]; if (dN) dN[i * B.n + k] = b[k]; }
  }
  return B.n;
}

// Default scalar range: cp min/max (CP mode), else min/max over an n^3 grid
// of sample points of every block.
int orc_scalar_range(void* v, int n, double* lo, double* hi) {
  Volume* V = (Volume*)v;
  double a = 1e300, z = -1e300;
  for (const Block& b : V->blocks) {
    if (V->mode == MODE_CP) {
      for (double s : b.scal) { a = std::min(a, s); z = std::max(z, s); }
    } else {
      for (int k = 0; k < n; ++k) for (int j = 0; j < n; ++j) for (int i = 0; i < n; ++i) {
        double p[3] = {(i + 0.5) / n, (j + 0.5) / n, (k + 0.5) / n}, f[3], J[3][3], rc;
        block_eval(b, p, f, J, &rc);
        double s = scalar_of(b, V->mode, p, J, rc);
        a = std::min(a, s); z = std::max(z, s);
      }
    }
  }
  *lo = a; *hi = z;
  return 0;
}

void orc_ray(const orc_camera* c, int W, int H, double x, double y, double* o, double* d) {
  Camera cam;
  std::memcpy(&cam, c, sizeof(cam));
  make_ray(cam, W, H, x, y, o, d);
}

int orc_hits(void* v, const double* o, const double* d, int cap, orc_hit* out) {
  std::vector<Hit> h = ray_hits(*(Volume*)v, o, d);
  const int n = (int)h.size();
  for (int i = 0; i < n && i < cap; ++i) {
    out[i].t = h[i].t;
    for (int r = 0; r < 3; ++r) out[i].p[r] = h[i].p[r];
    out[i].block = h[i].block; out[i].face = h[i].face; out[i].front = h[i].front;
  }
  return n;
}

// Alg. 2 on a caller-built hit list (already sorted or not; pairing only
// depends on t).  Returns the number of pairs.
int orc_pair_hits(const orc_hit* in, int n, int cap, orc_pair* out, int* unmatched) {
  std::vector<Hit> h(n);
  for (int i = 0; i < n; ++i) {
    h[i].t = in[i].t;
    for (int r = 0; r < 3; ++r) h[i].p[r] = in[i].p[r];
    h[i].block = in[i].block; h[i].face = in[i].face; h[i].front = in[i].front;
  }
  std::vector<Pair> p = pair_hits(h, unmatched);
  for (int i = 0; i < (int)p.size() && i < cap; ++i) {
    out[i].block = p[i].block; out[i].t_in = p[i].t_in; out[i].t_out = p[i].t_out;
    for (int r = 0; r < 3; ++r) { out[i].p_in[r] = p[i].p_in[r]; out[i].p_out[r] = p[i].p_out[r]; }
  }
  return (int)p.size();
}

int orc_pixel_pairs(void* v, const orc_camera* c, int W, int H, int x, int y, int cap, orc_pair* out, int* unmatched) {
  double o[3], d[3];
  orc_ray(c, W, H, x, y, o, d);
  std::vector<Hit> h = ray_hits(*(Volume*)v, o, d);
  std::vector<Pair> p = shrink_singular_entries(*(Volume*)v, o, d, 1e-13, pair_hits(h, unmatched), nullptr, unmatched);
  for (int i = 0; i < (int)p.size() && i < cap; ++i) {
    out[i].block = p[i].block; out[i].t_in = p[i].t_in; out[i].t_out = p[i].t_out;
    for (int r = 0; r < 3; ++r) { out[i].p_in[r] = p[i].p_in[r]; out[i].p_out[r] = p[i].p_out[r]; }
  }
  return (int)p.size();
}

// The walk of §5.4's first case on one ray segment (test hook): returns 1
// and the first point of [t0, t1] inside the block, or 0.
int orc_walk_into_block(void* v, int block, const double* o, const double* d, double t0, double t1, const double* p0,
                        const double* p1, double* t_new, double* p_new) {
  const Volume* V = (const Volume*)v;
  return walk_into_block(V->blocks[block], o, d, t0, t1, p0, p1, 1e-13 * V->diag, t_new, p_new) ? 1 : 0;
}

int orc_invert(void* v, int block, const double* g, const double* p0, double tol, int maxit, double* p) {
  return invert_point(((Volume*)v)->blocks[block], g, p0, tol, maxit, p);
}

// Composite a run of scalar samples rho[0..n) at positions s[0..n) (Alg. 1
// with supersampling).  out = (R, G, B, A).
void orc_composite(const orc_tf* t, int K, double early, int n, const double* s, const double* rho, double* out) {
  TF tf;
  tf.r.assign(t->r, t->r + t->n_knots);
  tf.rgba.assign(t->rgba, t->rgba + 4 * t->n_knots);
  tf.sigma = t->sigma; tf.lo = t->lo; tf.hi = t->hi;
  Accum acc;
  for (int j = 1; j < n; ++j) composite_interval(tf, K, early, rho[j - 1], rho[j], s[j] - s[j - 1], acc);
  out[0] = acc.C[0]; out[1] = acc.C[1]; out[2] = acc.C[2]; out[3] = acc.a;
}

// Per-sample trace of one pair: rows (s, p0, p1, p2, rho).  Returns rows.
int orc_trace_pair(void* v, const orc_tf* t, const orc_params* prm, const double* o, const double* d,
                   const orc_pair* pr, int cap, double* rows) {
  Volume* V = (Volume*)v;
  TF tf;
  tf.r.assign(t->r, t->r + t->n_knots);
  tf.rgba.assign(t->rgba, t->rgba + 4 * t->n_knots);
  tf.sigma = t->sigma; tf.lo = t->lo; tf.hi = t->hi;
  Params P{prm->ds, prm->supersample_k, prm->c, 2.0, prm->method, prm->newton_tol, prm->rk_tol, 0.0, 0, {}};
  Pair p;
  p.block = pr->block; p.t_in = pr->t_in; p.t_out = pr->t_out;
  for (int r = 0; r < 3; ++r) { p.p_in[r] = pr->p_in[r]; p.p_out[r] = pr->p_out[r]; }
  Accum acc;
  PixelStats st;
  std::vector<double> tr;
  render_pair(*V, tf, P, o, d, p, acc, st, &tr);
  const int rows_n = (int)tr.size() / 5;
  for (int i = 0; i < rows_n && i < cap; ++i) for (int k = 0; k < 5; ++k) rows[i * 5 + k] = tr[i * 5 + k];
  return rows_n;
}

// Render pixels [x0,x1) x [y0,y1) of a W x H image into out[(y-y0)][(x-x0)][4].
// n_threads worker threads take chunks of 16 pixels.  Returns 0.
int orc_render(void* v, const orc_tf* t, const orc_camera* c, const orc_params* prm, int W, int H,
               int x0, int x1, int y0, int y1, int n_threads, double* out, orc_pixel_stats* stats) {
  Volume* V = (Volume*)v;
  TF tf;
  tf.r.assign(t->r, t->r + t->n_knots);
  tf.rgba.assign(t->rgba, t->rgba + 4 * t->n_knots);
  tf.sigma = t->sigma; tf.lo = t->lo; tf.hi = t->hi;
  Params P{prm->ds, prm->supersample_k, prm->c, prm->early_alpha, prm->method, prm->newton_tol, prm->rk_tol,
           prm->near_clip, prm->n_cut < 0 ? 0 : (prm->n_cut > 4 ? 4 : prm->n_cut), {}};
  for (int k = 0; k < P.n_cut; ++k)
    for (int c = 0; c < 4; ++c) P.cut[k][c] = prm->cut[k][c];
  Camera cam;
  std::memcpy(&cam, c, sizeof(cam));
  const int w = x1 - x0, h = y1 - y0;
  const long npx = (long)w * h;
  const long chunk = 16;                           // pixels per work item
  std::atomic<long> next(0);
  auto work = [&]() {
    for (;;) {
      const long c0 = next.fetch_add(chunk);
      if (c0 >= npx) break;
      for (long q = c0; q < c0 + chunk && q < npx; ++q) {
        const int row = (int)(q / w), i = (int)(q % w);
        PixelStats st;
        render_pixel(*V, tf, P, cam, W, H, x0 + i, y0 + row, out + (size_t)q * 4, st);
        if (stats) {
          orc_pixel_stats& s = stats[q];
          s.npairs = st.npairs; s.unmatched = st.unmatched; s.newton_fail = st.newton_fail;
          s.nsamples = st.nsamples; s.rk_steps = st.rk_steps; s.shrunk = st.shrunk;
        }
      }
    }
  };
  if (n_threads <= 1) {
    work();
  } else {
    std::vector<std::thread> th;
    for (int i = 0; i < n_threads; ++i) th.emplace_back(work);
    for (auto& x : th) x.join();
  }
  return 0;
}

// Entry/exit pairs (§4.1 intersections, Alg. 2, singular entries moved as
// §5.4 says) of the pixels [x0,x1) x [y0,y1) of a W x H image, without
// cutting planes: count[q], and for slot k
// < cap pairs[(k * npx + q) * 8 + (p_in[3], t_in, p_out[3], t_out)] and
// block[k * npx + q], q = (y - y0)(x1 - x0) + (x - x0).  Multithreaded as
// orc_render.  Returns 0.
int orc_window_pairs(void* v, const orc_camera* c, int W, int H, int x0, int x1, int y0, int y1, int n_threads,
                     int cap, int* count, double* pairs, int* block) {
  const Volume* V = (const Volume*)v;
  const int w = x1 - x0, h = y1 - y0;
  const long npx = (long)w * h;
  std::atomic<long> next(0);
  auto work = [&]() {
    for (;;) {
      const long c0 = next.fetch_add(16);
      if (c0 >= npx) break;
      for (long q = c0; q < c0 + 16 && q < npx; ++q) {
        double o[3], d[3];
        orc_ray(c, W, H, x0 + (int)(q % w), y0 + (int)(q / w), o, d);
        int um = 0;
        std::vector<Pair> pr = shrink_singular_entries(*V, o, d, 1e-13, pair_hits(ray_hits(*V, o, d), &um),
                                                       nullptr, &um);
        count[q] = (int)pr.size();
        for (int k = 0; k < (int)pr.size() && k < cap; ++k) {
          double* e = pairs + ((size_t)k * npx + q) * 8;
          for (int r = 0; r < 3; ++r) { e[r] = pr[k].p_in[r]; e[4 + r] = pr[k].p_out[r]; }
          e[3] = pr[k].t_in;
          e[7] = pr[k].t_out;
          block[(size_t)k * npx + q] = pr[k].block;
        }
      }
    }
  };
  if (n_threads <= 1) {
    work();
  } else {
    std::vector<std::thread> th;
    for (int i = 0; i < n_threads; ++i) th.emplace_back(work);
    for (auto& x : th) x.join();
  }
  return 0;
}

// Table 1 of §5.3: error of a fixed-step method on the analytic map.
// method: 1 Euler, 2 midpoint, 3 Kutta-3, 4 RK4, 5 RK4 3/8, 6 RKF (5th order
// weights), 7 RF with stopping tolerance rf_tol on ||F||, 8 implicit Euler.
// The ray is sampled every ds in G arc length from g_in to g_out (last step
// partial).  err = max_i distance of phi(p_i) to the ray.
int orc_table1_ex(int method, double ds, double c, double rf_tol, double* err, long* newton_iters);
int orc_table1(int method, double ds, double c, double rf_tol, double* err) {
  return orc_table1_ex(method, ds, c, rf_tol, err, nullptr);
}

// One implicit Euler step on the analytic map of the Table 1 harness from p
// with step h, Newton capped at max_it iterations to |dz| <= tol; g_in and d
// are the harness's.  pn receives the new point; returns irk1_step's value
// (-1: the §5.4 boundary step was taken).  For pinning that step directly.
int orc_t1_irk1_step(const double* p, double h, double c, double tol, int max_it, double* pn) {
  const double p_in[3] = {0.0, 0.3, 0.5}, p_out[3] = {1.0, 0.7, 0.5};
  double g_in[3], g_out[3], J[3][3];
  t1_map(p_in, g_in, J);
  t1_map(p_out, g_out, J);
  double d[3] = {g_out[0] - g_in[0], g_out[1] - g_in[1], g_out[2] - g_in[2]};
  const double L = norm3(d);
  for (int r = 0; r < 3; ++r) d[r] /= L;
  return irk1_step(t1_map2, p, h, g_in, d, c, tol, max_it, pn);
}

// As orc_table1; newton_iters (if not NULL) receives the Newton iterations
// of the implicit Euler steps (method 8).
int orc_table1_ex(int method, double ds, double c, double rf_tol, double* err, long* newton_iters) {
  const double p_in[3] = {0.0, 0.3, 0.5}, p_out[3] = {1.0, 0.7, 0.5};
  double g_in[3], g_out[3], J[3][3];
  t1_map(p_in, g_in, J);
  t1_map(p_out, g_out, J);
  double d[3] = {g_out[0] - g_in[0], g_out[1] - g_in[1], g_out[2] - g_in[2]};
  const double L = norm3(d);
  for (int r = 0; r < 3; ++r) d[r] /= L;
  auto dist = [&](const double p[3]) {
    double phi[3], Jm[3][3];
    t1_map(p, phi, Jm);
    double e[3] = {g_in[0] - phi[0], g_in[1] - phi[1], g_in[2] - phi[2]};
    const double ed = dot3(e, d);
    double q[3] = {e[0] - ed * d[0], e[1] - ed * d[1], e[2] - ed * d[2]};
    return norm3(q);
  };
  double p[3] = {p_in[0], p_in[1], p_in[2]};
  double e = dist(p);
  double s = 0;
  int steps = 0;
  if (newton_iters) *newton_iters = 0;
  if (method >= 1 && method <= 6) {
    Tableau T = tableau(method);
    while (s < L - 1e-14 && steps < 10000000) {
      const double h = std::min(ds, L - s);
      double k[6][3];
      for (int st = 0; st < T.s; ++st) {
        double q[3];
        for (int r = 0; r < 3; ++r) {
          double acc = p[r];
          for (int j = 0; j < st; ++j) acc += h * T.a[st][j] * k[j][r];
          q[r] = acc;
        }
        t1_rhs(q, g_in, d, c, k[st]);
      }
      for (int r = 0; r < 3; ++r) {
        double acc = p[r];
        for (int st = 0; st < T.s; ++st) acc += h * T.b[st] * k[st][r];
        p[r] = acc;
      }
      s += h;
      ++steps;
      e = std::max(e, dist(p));
    }
  } else if (method == 8) {
    while (s < L - 1e-14 && steps < 10000000) {
      const double h = std::min(ds, L - s);
      double pn[3];
      const int it = irk1_step(t1_map2, p, h, g_in, d, c, 1e-13, 50, pn);
      if (it < 0) return -1;
      if (newton_iters) *newton_iters += it;
      for (int r = 0; r < 3; ++r) p[r] = pn[r];
      s += h;
      ++steps;
      e = std::max(e, dist(p));
    }
  } else if (method == 7) {
    while (s < L - 1e-14 && steps < 10000000) {
      s = std::min(L, s + ds);
      double g[3] = {g_in[0] + s * d[0], g_in[1] + s * d[1], g_in[2] + s * d[2]};
      for (int it = 0; it < 100; ++it) {
        double phi[3], Jm[3][3];
        t1_map(p, phi, Jm);
        double F[3] = {phi[0] - g[0], phi[1] - g[1], phi[2] - g[2]};
        if (norm3(F) <= rf_tol) break;
        double rhs[3] = {-F[0], -F[1], -F[2]}, dx[3];
        qr_solve3(Jm, rhs, dx);
        for (int r = 0; r < 3; ++r) p[r] += dx[r];
      }
      ++steps;
      e = std::max(e, dist(p));
    }
  } else {
    return -1;
  }
  *err = e;
  return steps;
}

}  // extern "C"
