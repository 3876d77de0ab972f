// Host preparation of a multi-block B-spline volume (once per volume, not per
// frame).  Validates the input, normalises knots to [0,1], converts each block
// to Bezier elements by knot insertion (Boehm), raises every element to the
// common degree P, extracts the 6 boundary faces of every block (§4.1: "6
// surfaces per block") as Bezier face patches, checks det J > 0 (§5,
// assumption 4) and computes the default scalar range.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ivv_internal.h"
#include "strain.h"

namespace ivv {
namespace {

// Insert knot x once into (T, degree p, control points Q[n][D]) (Boehm).
void insert_knot(std::vector<double>& T, int p, std::vector<double>& Q, int D, double x) {
  const int n = (int)Q.size() / D;
  int k = -1;                                  // T[k] <= x < T[k+1]
  for (int i = 0; i + 1 < (int)T.size(); ++i)
    if (T[i] <= x && x < T[i + 1]) k = i;
  std::vector<double> R((n + 1) * D);
  for (int i = 0; i <= n; ++i) {
    for (int c = 0; c < D; ++c) {
      double v;
      if (i <= k - p) {
        v = Q[i * D + c];
      } else if (i >= k + 1) {
        v = Q[(i - 1) * D + c];
      } else {
        const double a = (x - T[i]) / (T[i + p] - T[i]);
        v = (1 - a) * Q[(i - 1) * D + c] + a * Q[i * D + c];
      }
      R[i * D + c] = v;
    }
  }
  T.insert(T.begin() + k + 1, x);
  Q.swap(R);
}

// Bezier segments of one clamped B-spline curve (n control points of
// dimension D), raised to degree P: out[nseg][P+1][D]; brk[nseg+1].
void extract_curve(const std::vector<double>& knots, int p, int D, const double* cp, int n, int P,
                   std::vector<double>& out, std::vector<double>& brk) {
  std::vector<double> T = knots;
  std::vector<double> Q(cp, cp + (size_t)n * D);
  brk.clear();
  for (double x : knots) if (brk.empty() || x > brk.back()) brk.push_back(x);
  for (size_t b = 1; b + 1 < brk.size(); ++b) {
    const double x = brk[b];
    int mult = 0;
    for (double y : T) if (y == x) ++mult;
    for (int r = mult; r < p; ++r) insert_knot(T, p, Q, D, x);
  }
  const int nseg = (int)brk.size() - 1;
  out.assign((size_t)nseg * (P + 1) * D, 0.0);
  for (int s = 0; s < nseg; ++s) {
    std::vector<double> seg(Q.begin() + (size_t)s * p * D, Q.begin() + (size_t)(s * p + p + 1) * D);
    for (int q = p; q < P; ++q) {                // degree elevation q -> q+1
      std::vector<double> up((q + 2) * D);
      for (int c = 0; c < D; ++c) {
        up[c] = seg[c];
        up[(q + 1) * D + c] = seg[q * D + c];
        for (int i = 1; i <= q; ++i) {
          const double a = (double)i / (q + 1);
          up[i * D + c] = a * seg[(i - 1) * D + c] + (1 - a) * seg[i * D + c];
        }
      }
      seg.swap(up);
    }
    std::copy(seg.begin(), seg.end(), out.begin() + (size_t)s * (P + 1) * D);
  }
}

void bernstein(int P, double x, double* b, double* db) {
  const double y = 1 - x;
  if (P == 2) {
    b[0] = y * y; b[1] = 2 * x * y; b[2] = x * x;
    db[0] = -2 * y; db[1] = 2 - 4 * x; db[2] = 2 * x;
  } else {
    b[0] = y * y * y; b[1] = 3 * x * y * y; b[2] = 3 * x * x * y; b[3] = x * x * x;
    db[0] = -3 * y * y; db[1] = 3 * y * (1 - 3 * x); db[2] = 3 * x * (2 - 3 * x); db[3] = 3 * x * x;
  }
}

int find_seg(const double* brk, int nseg, double x) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (brk[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

double det3(const double J[3][3]) {
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
         J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

// Oriented bounding box of a face patch's control points (relative to org):
// axes from the patch tangents at its centre, extents from the control
// points, padded by a relative 1e-6 so the FP32 copy stays conservative.
// Control points of the piece [t0, t1] of a Bezier curve of degree P with
// points c[0..P] (3-D, stride `stride` doubles between points), in place:
// de Casteljau at t1 keeps the left part, then at t0 / t1 keeps the right one.
void bezier_sub_curve(double* c, int P, int stride, double t0, double t1) {
  double w[4][3], l[4][3];
  for (int k = 0; k <= P; ++k)
    for (int r = 0; r < 3; ++r) w[k][r] = c[k * stride + r];
  for (int r = 0; r < 3; ++r) l[0][r] = w[0][r];
  for (int lev = 1; lev <= P; ++lev) {
    for (int k = 0; k + lev <= P; ++k)
      for (int r = 0; r < 3; ++r) w[k][r] += t1 * (w[k + 1][r] - w[k][r]);
    for (int r = 0; r < 3; ++r) l[lev][r] = w[0][r];
  }
  const double s = t1 > 0 ? t0 / t1 : 0.0;
  double out[4][3];
  for (int r = 0; r < 3; ++r) out[P][r] = l[P][r];
  for (int lev = 1; lev <= P; ++lev) {
    for (int k = 0; k + lev <= P; ++k)
      for (int r = 0; r < 3; ++r) l[k][r] += s * (l[k + 1][r] - l[k][r]);
    for (int r = 0; r < 3; ++r) out[P - lev][r] = l[P - lev][r];
  }
  for (int k = 0; k <= P; ++k)
    for (int r = 0; r < 3; ++r) c[k * stride + r] = out[k][r];
}

// The sub-patch [a0,a1] x [b0,b1] of a tensor-product Bezier patch with
// control net net[(bi * (P+1) + ai) * 3 + r], in place.
void bezier_sub_patch(double* net, int P, double a0, double a1, double b0, double b1) {
  const int n1 = P + 1;
  for (int bi = 0; bi < n1; ++bi) bezier_sub_curve(net + (size_t)bi * n1 * 3, P, 3, a0, a1);
  for (int ai = 0; ai < n1; ++ai) bezier_sub_curve(net + (size_t)ai * 3, P, n1 * 3, b0, b1);
}

void face_obb(const double* cp, int P, const double org[3], FaceMeta& m) {
  const int n1 = P + 1;
  double b[4], db[4];
  bernstein(P, 0.5, b, db);
  double Sa[3] = {0, 0, 0}, Sb[3] = {0, 0, 0};
  for (int j = 0; j < n1; ++j)
    for (int i = 0; i < n1; ++i)
      for (int r = 0; r < 3; ++r) {
        Sa[r] += db[i] * b[j] * cp[(j * n1 + i) * 4 + r];
        Sb[r] += b[i] * db[j] * cp[(j * n1 + i) * 4 + r];
      }
  auto norm = [](double* v) {
    const double n = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (n > 0) for (int r = 0; r < 3; ++r) v[r] /= n;
    return n;
  };
  double ax[3][3];
  for (int r = 0; r < 3; ++r) ax[0][r] = Sa[r];
  double nrm[3] = {Sa[1] * Sb[2] - Sa[2] * Sb[1], Sa[2] * Sb[0] - Sa[0] * Sb[2], Sa[0] * Sb[1] - Sa[1] * Sb[0]};
  if (norm(ax[0]) == 0 || norm(nrm) == 0) {           // degenerate: axis-aligned box
    for (int a = 0; a < 3; ++a)
      for (int r = 0; r < 3; ++r) ax[a][r] = a == r ? 1.0 : 0.0;
  } else {
    for (int r = 0; r < 3; ++r) ax[2][r] = nrm[r];
    ax[1][0] = ax[2][1] * ax[0][2] - ax[2][2] * ax[0][1];
    ax[1][1] = ax[2][2] * ax[0][0] - ax[2][0] * ax[0][2];
    ax[1][2] = ax[2][0] * ax[0][1] - ax[2][1] * ax[0][0];
    norm(ax[1]);
  }
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300}, ext = 0;
  for (int k = 0; k < n1 * n1; ++k)
    for (int a = 0; a < 3; ++a) {
      const double x = ax[a][0] * cp[k * 4] + ax[a][1] * cp[k * 4 + 1] + ax[a][2] * cp[k * 4 + 2];
      lo[a] = std::min(lo[a], x);
      hi[a] = std::max(hi[a], x);
    }
  for (int a = 0; a < 3; ++a) ext = std::max(ext, hi[a] - lo[a]);
  for (int r = 0; r < 3; ++r) {
    double c = org[r];
    for (int a = 0; a < 3; ++a) c += ax[a][r] * 0.5 * (lo[a] + hi[a]);
    m.obb_c[r] = (float)c;
  }
  for (int a = 0; a < 3; ++a) {
    for (int r = 0; r < 3; ++r) m.obb_ax[a][r] = (float)ax[a][r];
    m.obb_h[a] = (float)(0.5 * (hi[a] - lo[a]) + 1e-6 * ext + 1e-6 * std::fabs(org[0] + org[1] + org[2]));
  }
}

}  // namespace

namespace {

// Value and first partials of one field stored as Bezier elements (el, org:
// the geometry with its scalar channel, or the displacement) at p.
void eval_elements(const HostVolume& hv, const std::vector<double>& el, const std::vector<double>& eorg, int block,
                   const double p[3], double f[3], double J[3][3], double* rho_cp) {
  const BlockInfo& B = hv.blocks[block];
  const int P = hv.P, n1 = P + 1;
  int e[3];
  double loc[3], sc[3];
  for (int d = 0; d < 3; ++d) {
    const double* brk = &hv.brk[B.brk_off[d]];
    const double x = std::min(std::max(p[d], 0.0), 1.0);
    e[d] = find_seg(brk, B.nseg[d], x);
    sc[d] = 1.0 / (brk[e[d] + 1] - brk[e[d]]);
    loc[d] = (x - brk[e[d]]) * sc[d];
  }
  const int eid = B.elem_off + (e[2] * B.nseg[1] + e[1]) * B.nseg[0] + e[0];
  const double* C = &el[(size_t)eid * n1 * n1 * n1 * 4];
  const double* org = &eorg[(size_t)eid * 4];
  double bu[4], dbu[4], bv[4], dbv[4], bw[4], dbw[4];
  bernstein(P, loc[0], bu, dbu);
  bernstein(P, loc[1], bv, dbv);
  bernstein(P, loc[2], bw, dbw);
  for (int r = 0; r < 3; ++r) { f[r] = 0; J[r][0] = J[r][1] = J[r][2] = 0; }
  double rho = 0;
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n1; ++j)
      for (int k = 0; k < n1; ++k) {
        const double* c = C + ((i * n1 + j) * n1 + k) * 4;
        const double w0 = bu[i] * bv[j] * bw[k];
        for (int r = 0; r < 3; ++r) {
          f[r] += w0 * c[r];
          J[r][0] += dbu[i] * bv[j] * bw[k] * c[r] * sc[0];
          J[r][1] += bu[i] * dbv[j] * bw[k] * c[r] * sc[1];
          J[r][2] += bu[i] * bv[j] * dbw[k] * c[r] * sc[2];
        }
        rho += w0 * c[3];
      }
  for (int r = 0; r < 3; ++r) f[r] += org[r];
  if (rho_cp) *rho_cp = rho;
}

}  // namespace

void host_eval(const HostVolume& hv, int block, const double p[3], double phi[3], double J[3][3],
               double* rho_cp) {
  eval_elements(hv, hv.elem, hv.elem_org, block, p, phi, J, rho_cp);
}

double host_scalar(const HostVolume& hv, int block, const double p[3], const double J[3][3], double rho_cp) {
  if (hv.mode == IVV_SCALAR_CP) return rho_cp;
  if (hv.mode == IVV_SCALAR_VONMISES) {
    double u[3], Ju[3][3];
    eval_elements(hv, hv.disp, hv.disp_org, block, p, u, Ju, nullptr);
    return von_mises<double>(J, Ju);
  }
  const double dj = det3(J);
  if (hv.mode == IVV_SCALAR_DETJ) return dj;
  double f = 0;
  for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) f += J[r][c] * J[r][c];
  return dj / std::sqrt(f);
}

ivv_status prepare_volume(const ivv_block_desc* blocks, int n_blocks, int mode, HostVolume& hv,
                          std::string& err) {
  if (!blocks || n_blocks <= 0) { err = "no blocks"; return IVV_ERR_INVALID_ARG; }
  if (mode < IVV_SCALAR_CP || mode > IVV_SCALAR_VONMISES) { err = "bad scalar mode"; return IVV_ERR_INVALID_ARG; }
  hv = HostVolume();
  hv.mode = mode;
  hv.n_blocks = n_blocks;
  int P = 2;
  for (int b = 0; b < n_blocks; ++b) {
    for (int d = 0; d < 3; ++d) {
      const int p = blocks[b].degree[d], n = blocks[b].n_cp[d];
      if (p < 1) { err = "degree must be >= 1"; return IVV_ERR_INVALID_ARG; }
      if (p > 3) { err = "degrees above 3 are not supported"; return IVV_ERR_UNSUPPORTED; }
      if (n < p + 1) { err = "n_cp must be >= degree + 1"; return IVV_ERR_INVALID_ARG; }
      if (!blocks[b].knots[d]) { err = "missing knot vector"; return IVV_ERR_INVALID_ARG; }
      P = std::max(P, p);
    }
    if (!blocks[b].geom_cp) { err = "missing geometry control points"; return IVV_ERR_INVALID_ARG; }
    if (mode == IVV_SCALAR_CP && !blocks[b].scalar_cp) {
      err = "IVV_SCALAR_CP needs scalar control points"; return IVV_ERR_INVALID_ARG;
    }
    if (mode == IVV_SCALAR_VONMISES && !blocks[b].disp_cp) {
      err = "IVV_SCALAR_VONMISES needs displacement control points"; return IVV_ERR_INVALID_ARG;
    }
  }
  // channels carried through the extraction: (x, y, z, rho), plus the
  // displacement (u_x, u_y, u_z) for the von Mises scalar
  const int nc = mode == IVV_SCALAR_VONMISES ? 7 : 4;
  hv.P = P;
  const int n1 = P + 1;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  double slo = 1e300, shi = -1e300;
  for (int b = 0; b < n_blocks; ++b) {
    const ivv_block_desc& d = blocks[b];
    std::vector<double> kn[3];
    for (int k = 0; k < 3; ++k) {
      const int p = d.degree[k], n = d.n_cp[k], nk = n + p + 1;
      kn[k].assign(d.knots[k], d.knots[k] + nk);
      for (int i = 1; i < nk; ++i)
        if (!(kn[k][i] >= kn[k][i - 1])) { err = "knots must be non-decreasing"; return IVV_ERR_INVALID_ARG; }
      const double a = kn[k][0], z = kn[k][nk - 1];
      if (!(z > a)) { err = "empty knot range"; return IVV_ERR_INVALID_ARG; }
      for (int i = 0; i <= p; ++i)
        if (kn[k][i] != a || kn[k][nk - 1 - i] != z) { err = "knot vectors must be clamped"; return IVV_ERR_INVALID_ARG; }
      for (int i = p + 1; i < n; ++i) {
        int m = 0;
        for (int j = 0; j < nk; ++j) if (kn[k][j] == kn[k][i]) ++m;
        if (m > p) { err = "interior knot multiplicity exceeds the degree"; return IVV_ERR_INVALID_ARG; }
      }
      for (double& x : kn[k]) x = (x - a) / (z - a);
    }
    const int nu = d.n_cp[0], nv = d.n_cp[1], nw = d.n_cp[2];
    // grid[w][v][u][nc] = (x, y, z, rho[, u_x, u_y, u_z])
    std::vector<double> grid((size_t)nu * nv * nw * nc);
    for (size_t q = 0; q < (size_t)nu * nv * nw; ++q) {
      for (int r = 0; r < 3; ++r) {
        const double v = d.geom_cp[3 * q + r];
        if (!std::isfinite(v)) { err = "non-finite control point"; return IVV_ERR_INVALID_ARG; }
        grid[nc * q + r] = v;
        lo[r] = std::min(lo[r], v);
        hi[r] = std::max(hi[r], v);
      }
      const double s = (mode == IVV_SCALAR_CP) ? d.scalar_cp[q] : 0.0;
      if (!std::isfinite(s)) { err = "non-finite scalar control point"; return IVV_ERR_INVALID_ARG; }
      grid[nc * q + 3] = s;
      slo = std::min(slo, s);
      shi = std::max(shi, s);
      for (int r = 0; r < nc - 4; ++r) {
        const double u = d.disp_cp[3 * q + r];
        if (!std::isfinite(u)) { err = "non-finite displacement control point"; return IVV_ERR_INVALID_ARG; }
        grid[nc * q + 4 + r] = u;
      }
    }
    // extraction along u, then v, then w (tensor product)
    int dims[3] = {nu, nv, nw};
    std::vector<double> brk[3];
    for (int axis = 0; axis < 3; ++axis) {
      const int n = dims[axis];
      int other[2];
      int oi = 0;
      for (int a = 0; a < 3; ++a) if (a != axis) other[oi++] = a;
      std::vector<double> seg_out;
      std::vector<double> line((size_t)n * nc);
      int nout = -1;
      std::vector<double> next;
      int ndims[3] = {dims[0], dims[1], dims[2]};
      for (int i1 = 0; i1 < dims[other[1]]; ++i1)
        for (int i0 = 0; i0 < dims[other[0]]; ++i0) {
          auto index = [&](const int* dd, int along, int a0, int a1) {
            int c[3];
            c[axis] = along; c[other[0]] = a0; c[other[1]] = a1;
            return ((size_t)c[2] * dd[1] + c[1]) * dd[0] + c[0];
          };
          for (int t = 0; t < n; ++t)
            for (int c = 0; c < nc; ++c) line[t * nc + c] = grid[index(dims, t, i0, i1) * nc + c];
          extract_curve(kn[axis], d.degree[axis], nc, line.data(), n, P, seg_out, brk[axis]);
          if (nout < 0) {
            nout = (int)(seg_out.size() / nc);
            ndims[axis] = nout;
            next.assign((size_t)ndims[0] * ndims[1] * ndims[2] * nc, 0.0);
          }
          for (int t = 0; t < nout; ++t)
            for (int c = 0; c < nc; ++c) next[index(ndims, t, i0, i1) * nc + c] = seg_out[t * nc + c];
        }
      grid.swap(next);
      dims[axis] = ndims[axis];
    }
    BlockInfo B;
    for (int k = 0; k < 3; ++k) {
      B.nseg[k] = (int)brk[k].size() - 1;
      B.brk_off[k] = (int)hv.brk.size();
      hv.brk.insert(hv.brk.end(), brk[k].begin(), brk[k].end());
    }
    B.elem_off = hv.n_elems();
    B.tau_det = 0.f;
    B.sing_faces = 0;
    B.uniform = 0;
    B.mode = mode;
    for (int k = 0; k < 3; ++k) {
      bool uni = true;
      for (int i = 0; i <= B.nseg[k]; ++i)
        if (std::fabs(brk[k][i] - (double)i / B.nseg[k]) > 1e-12) uni = false;
      if (uni) B.uniform |= 1 << k;
    }
    // elements, i-major ((i*(P+1)+j)*(P+1)+k); geometry relative to the
    // element's first control point, which keeps FP32 partials accurate
    for (int ew = 0; ew < B.nseg[2]; ++ew)
      for (int ev = 0; ev < B.nseg[1]; ++ev)
        for (int eu = 0; eu < B.nseg[0]; ++eu) {
          const size_t g0 = (((size_t)(ew * n1) * dims[1]) + (ev * n1)) * dims[0] + (eu * n1);
          const double org[3] = {grid[g0 * nc], grid[g0 * nc + 1], grid[g0 * nc + 2]};
          for (int c = 0; c < 3; ++c) hv.elem_org.push_back(org[c]);
          hv.elem_org.push_back(0.0);
          if (nc == 7) {                  // the displacement, relative to its first control point
            for (int c = 0; c < 3; ++c) hv.disp_org.push_back(grid[g0 * nc + 4 + c]);
            hv.disp_org.push_back(0.0);
          }
          for (int i = 0; i < n1; ++i)
            for (int j = 0; j < n1; ++j)
              for (int k = 0; k < n1; ++k) {
                const size_t g = (((size_t)(ew * n1 + k) * dims[1]) + (ev * n1 + j)) * dims[0] + (eu * n1 + i);
                for (int c = 0; c < 3; ++c) hv.elem.push_back(grid[g * nc + c] - org[c]);
                hv.elem.push_back(grid[g * nc + 3]);
                if (nc == 7) {
                  for (int c = 0; c < 3; ++c) hv.disp.push_back(grid[g * nc + 4 + c] - grid[g0 * nc + 4 + c]);
                  hv.disp.push_back(0.0);
                }
              }
        }
    hv.blocks.push_back(B);
  }
  double dg[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
  hv.diag = std::sqrt(dg[0] * dg[0] + dg[1] * dg[1] + dg[2] * dg[2]);
  if (!(hv.diag > 0)) { err = "degenerate control-point bounding box"; return IVV_ERR_DEGENERATE; }

  // faces: 6 per block, one Bezier patch per element on the face; a patch
  // whose control net spans more than diag/6 is cut into k x k sub-patches
  // (k <= 4, exact de Casteljau extraction) so that every patch is small
  // against the volume (tight culling boxes, near-planar Newton problems)
  for (int b = 0; b < n_blocks; ++b) {
    const BlockInfo& B = hv.blocks[b];
    for (int f = 0; f < 6; ++f) {
      const int nd = f / 2, ad = (nd + 1) % 3, bd = (nd + 2) % 3;
      const int side = f % 2;
      for (int eb = 0; eb < B.nseg[bd]; ++eb)
        for (int ea = 0; ea < B.nseg[ad]; ++ea) {
          int e[3];
          e[nd] = side ? B.nseg[nd] - 1 : 0;
          e[ad] = ea;
          e[bd] = eb;
          const int eid = B.elem_off + (e[2] * B.nseg[1] + e[1]) * B.nseg[0] + e[0];
          const double* C = &hv.elem[(size_t)eid * n1 * n1 * n1 * 4];
          const double* eorg = &hv.elem_org[(size_t)eid * 4];
          // the element's face net, absolute, index bi * n1 + ai
          std::vector<double> net((size_t)n1 * n1 * 3);
          double nlo[3] = {1e300, 1e300, 1e300}, nhi[3] = {-1e300, -1e300, -1e300};
          for (int bi = 0; bi < n1; ++bi)
            for (int ai = 0; ai < n1; ++ai) {
              int l[3];
              l[nd] = side ? P : 0;
              l[ad] = ai;
              l[bd] = bi;
              const double* c = C + ((l[0] * n1 + l[1]) * n1 + l[2]) * 4;
              for (int r = 0; r < 3; ++r) {
                const double g = eorg[r] + c[r];
                net[((size_t)bi * n1 + ai) * 3 + r] = g;
                nlo[r] = std::min(nlo[r], g);
                nhi[r] = std::max(nhi[r], g);
              }
            }
          const double ndiag = std::sqrt((nhi[0] - nlo[0]) * (nhi[0] - nlo[0]) + (nhi[1] - nlo[1]) * (nhi[1] - nlo[1]) +
                                         (nhi[2] - nlo[2]) * (nhi[2] - nlo[2]));
          const int k = std::max(1, std::min(4, (int)std::ceil(ndiag / (hv.diag / 6.0) - 1e-9)));
          const double* ba = &hv.brk[B.brk_off[ad]];
          const double* bb = &hv.brk[B.brk_off[bd]];
          for (int sb = 0; sb < k; ++sb)
            for (int sa = 0; sa < k; ++sa) {
              std::vector<double> sub = net;
              if (k > 1) bezier_sub_patch(sub.data(), P, (double)sa / k, (double)(sa + 1) / k, (double)sb / k,
                                          (double)(sb + 1) / k);
              FaceMeta m;
              m.block = b;
              m.face = f;
              const double a0 = ba[ea] + (ba[ea + 1] - ba[ea]) * sa / k, a1 = ba[ea] + (ba[ea + 1] - ba[ea]) * (sa + 1) / k;
              const double b0 = bb[eb] + (bb[eb + 1] - bb[eb]) * sb / k, b1 = bb[eb] + (bb[eb + 1] - bb[eb]) * (sb + 1) / k;
              FaceMeta64 m64{sa == 0 ? ba[ea] : a0, sa == k - 1 ? ba[ea + 1] : a1, sb == 0 ? bb[eb] : b0,
                             sb == k - 1 ? bb[eb + 1] : b1, {0, 0, 0}};
              m.a0 = (float)m64.a0; m.a1 = (float)m64.a1; m.b0 = (float)m64.b0; m.b1 = (float)m64.b1;
              double flo[3] = {1e300, 1e300, 1e300}, fhi[3] = {-1e300, -1e300, -1e300};
              double forg[3] = {sub[0], sub[1], sub[2]};
              for (int q = 0; q < n1 * n1; ++q) {
                for (int r = 0; r < 3; ++r) {
                  const double g = sub[(size_t)q * 3 + r];
                  hv.face_cp.push_back(g - forg[r]);
                  flo[r] = std::min(flo[r], g);
                  fhi[r] = std::max(fhi[r], g);
                }
                hv.face_cp.push_back(0.0);
              }
              for (int r = 0; r < 3; ++r) {
                // round outward so the float box contains the double box
                m.lo[r] = std::nextafter((float)flo[r], -1e30f);
                m.hi[r] = std::nextafter((float)fhi[r], 1e30f);
                m.org[r] = (float)forg[r];
                m64.org[r] = forg[r];
              }
              face_obb(&hv.face_cp[hv.face_cp.size() - (size_t)n1 * n1 * 4], P, forg, m);
              hv.faces.push_back(m);
              hv.faces64.push_back(m64);
            }
        }
    }
  }

  // det J > 0 at sample points of every element, and the mean |det J| per block
  hv.mean_abs_det.assign(n_blocks, 0.0);
  const double sp[3] = {0.05, 0.5, 0.95};
  for (int b = 0; b < n_blocks; ++b) {
    BlockInfo& B = hv.blocks[b];
    const double* bu = &hv.brk[B.brk_off[0]];
    const double* bv = &hv.brk[B.brk_off[1]];
    const double* bw = &hv.brk[B.brk_off[2]];
    double sum = 0;
    long cnt = 0;
    for (int ew = 0; ew < B.nseg[2]; ++ew)
      for (int ev = 0; ev < B.nseg[1]; ++ev)
        for (int eu = 0; eu < B.nseg[0]; ++eu)
          for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c)
              for (int e = 0; e < 3; ++e) {
                double p[3] = {bu[eu] + sp[a] * (bu[eu + 1] - bu[eu]), bv[ev] + sp[c] * (bv[ev + 1] - bv[ev]),
                               bw[ew] + sp[e] * (bw[ew + 1] - bw[ew])};
                double phi[3], J[3][3];
                host_eval(hv, b, p, phi, J, nullptr);
                const double dj = det3(J);
                if (!(dj > 0)) {
                  err = "det J <= 0 inside block " + std::to_string(b) +
                        " (the parametrisation must be orientation preserving)";
                  return IVV_ERR_DEGENERATE;
                }
                sum += dj;
                ++cnt;
              }
    (void)sum;
    (void)cnt;
    // mean |det J| over [0,1]^3 (the block's volume in G): 5-point
    // Gauss-Legendre per knot span and direction, exact for det J
    static const double gx[5] = {-0.9061798459386640, -0.5384693101056831, 0.0, 0.5384693101056831,
                                 0.9061798459386640};
    static const double gw[5] = {0.2369268850561891, 0.4786286704993665, 0.5688888888888889, 0.4786286704993665,
                                 0.2369268850561891};
    double vol = 0;
    for (int ew = 0; ew < B.nseg[2]; ++ew)
      for (int ev = 0; ev < B.nseg[1]; ++ev)
        for (int eu = 0; eu < B.nseg[0]; ++eu) {
          const double h[3] = {bu[eu + 1] - bu[eu], bv[ev + 1] - bv[ev], bw[ew + 1] - bw[ew]};
          for (int a = 0; a < 5; ++a)
            for (int c = 0; c < 5; ++c)
              for (int e = 0; e < 5; ++e) {
                double p[3] = {bu[eu] + 0.5 * h[0] * (gx[a] + 1), bv[ev] + 0.5 * h[1] * (gx[c] + 1),
                               bw[ew] + 0.5 * h[2] * (gx[e] + 1)};
                double phi[3], J[3][3];
                host_eval(hv, b, p, phi, J, nullptr);
                vol += gw[a] * gw[c] * gw[e] * 0.125 * h[0] * h[1] * h[2] * std::fabs(det3(J));
              }
        }
    hv.mean_abs_det[b] = vol;
    B.tau_det = (float)(1e-6 * hv.mean_abs_det[b]);
    // faces on which det J comes within 1e-2 of the mean (9 x 9 points per
    // face element, edges included): entries there may need §5.4's shrink,
    // whose threshold is 1e-6 of the mean
    B.sing_faces = 0;
    const double* br[3] = {bu, bv, bw};
    for (int f = 0; f < 6; ++f) {
      const int nd = f >> 1, ad = (nd + 1) % 3, bd = (nd + 2) % 3;
      double mn = 1e300;
      for (int sa = 0; sa < B.nseg[ad]; ++sa)
        for (int sb = 0; sb < B.nseg[bd]; ++sb)
          for (int i = 0; i <= 8; ++i)
            for (int j = 0; j <= 8; ++j) {
              double p[3];
              p[nd] = (f & 1) ? 1.0 : 0.0;
              p[ad] = br[ad][sa] + (br[ad][sa + 1] - br[ad][sa]) * i / 8.0;
              p[bd] = br[bd][sb] + (br[bd][sb + 1] - br[bd][sb]) * j / 8.0;
              double phi[3], J[3][3];
              host_eval(hv, b, p, phi, J, nullptr);
              mn = std::min(mn, std::fabs(det3(J)));
            }
      if (mn < 1e-2 * hv.mean_abs_det[b]) B.sing_faces |= 1 << f;
    }
    if (B.sing_faces) hv.any_singular = true;
  }

  // default scalar range
  if (mode == IVV_SCALAR_CP) {
    hv.def_lo = slo;
    hv.def_hi = shi;
  } else {
    const int n = 64;
    double a = 1e300, z = -1e300;
    for (int b = 0; b < n_blocks; ++b)
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            double p[3] = {(i + 0.5) / n, (j + 0.5) / n, (k + 0.5) / n}, phi[3], J[3][3];
            host_eval(hv, b, p, phi, J, nullptr);
            const double s = host_scalar(hv, b, p, J, 0.0);
            a = std::min(a, s);
            z = std::max(z, s);
          }
    hv.def_lo = a;
    hv.def_hi = z;
  }
  if (!(hv.def_hi > hv.def_lo)) hv.def_hi = hv.def_lo + 1.0;
  return IVV_OK;
}

}  // namespace ivv
