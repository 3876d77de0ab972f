// Internal declarations shared by the host preparation (host_prep.cpp), the
// C-ABI (ivv_api.cu) and the kernel launchers (k_*.cu).  Not installed.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ivv.h"

namespace ivv {

constexpr int kTileW = 16;          // K2 screen tile (one CTA)
constexpr int kTileH = 8;
constexpr int kMaxFrags = 32;       // fragment slots per pixel (A-buffer)
constexpr int kMaxPairs = 16;       // entry/exit pair slots per pixel

// Face patch record: block, face index (0/1: u=0/1, 2/3: v=0/1, 4/5: w=0/1),
// parameter box of the patch on its face, the patch origin (its control
// points are stored relative to it) and the bbox of its control points.
struct FaceMeta {
  int block;
  int face;
  float a0, a1, b0, b1;
  float org[3];
  float lo[3], hi[3];
  // oriented box of the control points: centre, axes (rows: tangent a,
  // its orthogonal complement in the tangent plane, normal), half extents
  float obb_c[3];
  float obb_ax[3][3];
  float obb_h[3];
};

struct FaceMeta64 {
  double a0, a1, b0, b1;
  double org[3];
};

// Floats per element in the scalar-only array: (P+1)^3 scalar control points
// padded to a multiple of 8, so every element is 32-byte aligned and is read
// with 256-bit loads (64 for cubic, 32 for quadratic elements).
constexpr int rho_stride32(int P) { return ((P + 1) * (P + 1) * (P + 1) + 7) & ~7; }

struct BlockInfo {
  int nseg[3];
  int brk_off[3];     // offsets into the breakpoint arrays
  int elem_off;       // first Bezier element of the block
  float tau_det;      // |det J| below which MIXED precision solves in FP64
  int uniform;        // bit d set: breakpoints of direction d are i / nseg[d]
  int mode;           // IVV_SCALAR_* of the block's volume
  int sing_faces;     // bit f set: det J comes close to 0 on face f (singular entries possible, §5.4)
};

// Host image of a prepared volume (see host_prep.cpp).
struct HostVolume {
  int P = 3;                       // common Bezier degree (2 or 3)
  int mode = 0;                    // IVV_SCALAR_*
  int n_blocks = 0;
  std::vector<BlockInfo> blocks;
  std::vector<double> brk;         // concatenated breakpoints (normalised)
  std::vector<double> elem;        // [E][(P+1)^3][4] (x, y, z, rho), i-major, xyz relative to elem_org
  std::vector<double> elem_org;    // [E][4] element origin (first control point), w = 0
  std::vector<double> disp;        // IVV_SCALAR_VONMISES: [E][(P+1)^3][4] (u_x, u_y, u_z, 0) relative to disp_org
  std::vector<double> disp_org;    // [E][4] the element's first displacement control point, w = 0
  std::vector<double> face_cp;     // [F][(P+1)^2][4] (x, y, z, 0) relative to the face origin, a fastest
  std::vector<FaceMeta> faces;
  std::vector<FaceMeta64> faces64;
  std::vector<double> mean_abs_det;
  bool any_singular = false;       // some block has a face where det J comes close to 0
  double diag = 1.0;               // diagonal of the control-point bbox
  double def_lo = 0.0, def_hi = 1.0;   // default scalar range
  int n_elems() const { return (int)(elem.size() / (4 * (size_t)(P + 1) * (P + 1) * (P + 1))); }
  int n_faces() const { return (int)faces.size(); }
};

// Builds the host image.  Returns IVV_OK or an error with a message.
ivv_status prepare_volume(const ivv_block_desc* blocks, int n_blocks, int scalar_mode,
                          HostVolume& out, std::string& err);

// Host-side FP64 evaluation of phi, J and the scalar on the Bezier elements
// (used for the det J check and the default scalar range).
void host_eval(const HostVolume& hv, int block, const double p[3], double phi[3], double J[3][3],
               double* rho_cp);

// The volume's scalar at p of `block` from J = J_phi(p) and the control-point
// scalar there (IVV_SCALAR_* of the volume), FP64.
double host_scalar(const HostVolume& hv, int block, const double p[3], const double J[3][3], double rho_cp);

}  // namespace ivv
