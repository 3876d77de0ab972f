// Stage 2 (§4.2): per-pixel depth sorting of the fragment list and blockwise
// entry/exit pairing (Alg. 2).
//   K4 pair -- one thread per pixel: load the pixel's fragment slots (the
//              A-buffer written by K2), insertion-sort them by
//              (depth, block, facing), merge duplicates of one block with equal
//              facing (hits on edges shared by two patches or two faces), then
//              repeatedly take the nearest unused back-facing record and the
//              nearest unused front-facing record of the same block (Alg. 2).
//              Pairs are written in that order, which is front to back for
//              non-overlapping blocks.  Pixels with pairs are appended to the
//              work queue of the integrator; the others get a zero pixel.
#include <cuda_runtime.h>

#include "ivv_device.cuh"

namespace ivv {

namespace {

// Sorting and pairing of the fragments of pixel `pix` (slot index
// slot * stride + pix); returns the number of pairs written.  A pixel
// without pairs gets a zero RGBA in *zero_out (if not NULL).
template <typename R>
__device__ __forceinline__ int pair_pixel(size_t pix, size_t stride, R tau_dup,
                                          const typename Vec4T<R>::type* __restrict__ frag_tp,
                                          const unsigned* __restrict__ frag_meta, const int* __restrict__ frag_count,
                                          typename Vec4T<R>::type* __restrict__ pair_in,
                                          typename Vec4T<R>::type* __restrict__ pair_out, int* __restrict__ pair_block,
                                          int* __restrict__ pair_count, int max_pairs, float4* zero_out,
                                          unsigned& um, unsigned& pov, int max_frags = kMaxFrags) {
  typedef typename Vec4T<R>::type V4;
  int n = frag_count[pix];
  n = n < max_frags ? n : max_frags;
  R t[kMaxFrags], pp[kMaxFrags][3];
  unsigned m[kMaxFrags];
  for (int i = 0; i < n; ++i) {
    const V4 f = frag_tp[(size_t)i * stride + pix];
    t[i] = f.x;
    pp[i][0] = f.y;
    pp[i][1] = f.z;
    pp[i][2] = f.w;
    m[i] = frag_meta[(size_t)i * stride + pix];
  }
  int in_idx[kMaxPairs], out_idx[kMaxPairs];
  const int np = pair_fragments<R>(n, t, m, pp, tau_dup, max_pairs, in_idx, out_idx, um, pov);
  for (int q = 0; q < np; ++q) {
    const size_t o = (size_t)q * stride + pix;
    pair_in[o] = frag_tp[(size_t)in_idx[q] * stride + pix];
    pair_out[o] = frag_tp[(size_t)out_idx[q] * stride + pix];
    pair_block[o] = (int)(m[in_idx[q]] >> 4);
  }
  pair_count[pix] = np;
  if (np == 0 && zero_out) *zero_out = make_float4(0.f, 0.f, 0.f, 0.f);
  return np;
}

// pair_pixel with the cutting and near-clip planes (§5.5) of `cl`, for the
// pixel (xw, yw) of cl.cam's window: records in front of the near plane are
// dropped; a block whose nearest remaining record is an exit gets an entry on
// the near plane; every pair is clipped to the kept side of each cutting
// plane (empty pairs dropped); moved ends carry a chord guess and a solve
// flag in pair_block.
template <typename R>
__device__ __forceinline__ int pair_pixel_clip(size_t pix, size_t stride, R tau_dup,
                                               const typename Vec4T<R>::type* __restrict__ frag_tp,
                                               const unsigned* __restrict__ frag_meta,
                                               const int* __restrict__ frag_count,
                                               typename Vec4T<R>::type* __restrict__ pair_in,
                                               typename Vec4T<R>::type* __restrict__ pair_out,
                                               int* __restrict__ pair_block, int* __restrict__ pair_count,
                                               int max_pairs, float4* zero_out, unsigned& um, unsigned& pov,
                                               const ClipArgs<R>& cl, int xw, int yw, int max_frags) {
  typedef typename Vec4T<R>::type V4;
  R o[3], d[3];
  make_ray<R>(cl.cam, cl.cam.x0 + xw, cl.cam.y0 + yw, o, d);
  R t_near = R(0);
  if (cl.near > R(0)) t_near = cl.near / (d[0] * cl.f[0] + d[1] * cl.f[1] + d[2] * cl.f[2]);
  int n0 = frag_count[pix];
  n0 = n0 < max_frags ? n0 : max_frags;
  R t[kMaxFrags], pp[kMaxFrags][3];
  unsigned m[kMaxFrags];
  int n = 0;
  for (int i = 0; i < n0; ++i) {
    const V4 f = frag_tp[(size_t)i * stride + pix];
    if (cl.near > R(0) && f.x < t_near) continue;
    t[n] = f.x;
    pp[n][0] = f.y;
    pp[n][1] = f.z;
    pp[n][2] = f.w;
    m[n] = frag_meta[(size_t)i * stride + pix];
    ++n;
  }
  unsigned synth = 0;                  // bit i: record i is an entry on the near plane
  if (cl.near > R(0)) {
    const int nr = n;
    for (int i = 0; i < nr && n < kMaxFrags; ++i) {
      if (m[i] & 1u) continue;         // entries need no partner
      bool nearest = true;
      for (int k = 0; k < nr; ++k)
        if ((m[k] >> 4) == (m[i] >> 4) && (t[k] < t[i] || (t[k] == t[i] && k < i))) nearest = false;
      if (!nearest) continue;
      t[n] = t_near;
      pp[n][0] = pp[n][1] = pp[n][2] = R(0);
      m[n] = (m[i] & ~15u) | 1u;
      synth |= 1u << n;
      ++n;
    }
  }
  int in_idx[kMaxPairs], out_idx[kMaxPairs];
  const int np = pair_fragments<R>(n, t, m, pp, tau_dup, max_pairs, in_idx, out_idx, um, pov);
  int kept = 0;
  for (int q = 0; q < np; ++q) {
    const int a = in_idx[q], b = out_idx[q];
    R t0 = t[a], t1 = t[b];
    for (int k = 0; k < cl.n_cut; ++k) {
      const R fo = cl.cut[k][0] * o[0] + cl.cut[k][1] * o[1] + cl.cut[k][2] * o[2] + cl.cut[k][3];
      const R fd = cl.cut[k][0] * d[0] + cl.cut[k][1] * d[1] + cl.cut[k][2] * d[2];
      if (fd == R(0)) {
        if (fo > R(0)) t1 = t0 - R(1);
        continue;
      }
      const R tc = -fo / fd;
      if (fd > R(0)) t1 = tc < t1 ? tc : t1;
      else t0 = tc > t0 ? tc : t0;
    }
    if (!(t1 > t0)) continue;
    const bool s_in = (synth >> a) & 1u;
    const bool new_in = s_in || t0 > t[a], new_out = t1 < t[b];
    const R len = t[b] - t[a];
    R gi[3], go[3];
    const R w0 = len > R(0) ? (t0 - t[a]) / len : R(0), w1 = len > R(0) ? (t1 - t[a]) / len : R(1);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      gi[r] = s_in ? pp[b][r] : (new_in ? pp[a][r] + w0 * (pp[b][r] - pp[a][r]) : pp[a][r]);
      go[r] = new_out ? (s_in ? pp[b][r] : pp[a][r] + w1 * (pp[b][r] - pp[a][r])) : pp[b][r];
    }
    const size_t o2 = (size_t)kept * stride + pix;
    V4 ri, ro;
    ri.x = t0; ri.y = gi[0]; ri.z = gi[1]; ri.w = gi[2];
    ro.x = t1; ro.y = go[0]; ro.z = go[1]; ro.w = go[2];
    pair_in[o2] = ri;
    pair_out[o2] = ro;
    pair_block[o2] = (int)(m[a] >> 4) | (new_in ? kSolveIn : 0) | (new_out ? kSolveOut : 0) | (s_in ? kGuessIn : 0);
    ++kept;
  }
  pair_count[pix] = kept;
  if (kept == 0 && zero_out) *zero_out = make_float4(0.f, 0.f, 0.f, 0.f);
  return kept;
}

// Newton for the world point g in block B from p (line search on |F|, p
// clamped to [0,1]^3, §5.1); true when |phi(p) - g| <= tol.  MIXED: the 3x3
// solve switches to FP64 where |det J| < tau_det (counted in n64); iters
// accumulates the iterations.
template <int P, typename R, bool MIXED>
__device__ __forceinline__ bool clip_newton(const DevVolume& V, const BlockInfo& B, const R g[3], R p[3], R tol,
                                            unsigned long long& iters, unsigned long long& n64) {
  R phi[3], J[3][3], rc, F[3];
  eval_block<P, R, false>(V, B, p, phi, J, rc);
  for (int r = 0; r < 3; ++r) F[r] = phi[r] - g[r];
  R nF = sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
  for (int it = 0; it < 50; ++it) {
    if (nF <= tol) return true;
    ++iters;
    R rhs[3] = {-F[0], -F[1], -F[2]}, dx[3];
    const R det = solve3<R>(J, rhs, dx);
    if constexpr (MIXED) {
      if (fabs(det) < R(B.tau_det)) {
        double Jd[3][3], bd[3], xd[3];
        for (int r = 0; r < 3; ++r) {
          bd[r] = rhs[r];
          for (int k = 0; k < 3; ++k) Jd[r][k] = J[r][k];
        }
        solve3<double>(Jd, bd, xd);
        for (int r = 0; r < 3; ++r) dx[r] = R(xd[r]);
        ++n64;
      }
    }
    R lam = R(1);
    bool moved = false;
    for (int ls = 0; ls < 12 && !moved; ++ls, lam *= R(0.5)) {
      R q[3], Jq[3][3], Fq[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const R v = p[r] + lam * dx[r];
        q[r] = v < R(0) ? R(0) : (v > R(1) ? R(1) : v);
      }
      eval_block<P, R, false>(V, B, q, phi, Jq, rc);
      for (int r = 0; r < 3; ++r) Fq[r] = phi[r] - g[r];
      const R nq = sqrt(Fq[0] * Fq[0] + Fq[1] * Fq[1] + Fq[2] * Fq[2]);
      if (nq < nF) {
        moved = true;
        nF = nq;
        for (int r = 0; r < 3; ++r) {
          p[r] = q[r];
          F[r] = Fq[r];
          for (int k = 0; k < 3; ++k) J[r][k] = Jq[r][k];
        }
      }
    }
    if (!moved) break;
  }
  return nF <= tol;
}

// Newton tolerance of the fix-up solves at world point g: 1e-6 diag (FP32)
// or 1e-12 diag (FP64), plus the rounding of g itself.
template <typename R>
__device__ __forceinline__ R fixup_tol(const R g[3], float diag) {
  const R tol = sizeof(R) == 4 ? R(1e-6) * R(diag) : R(1e-12) * R(diag);
  const R m = fmax(fabs(g[0]), fmax(fabs(g[1]), fabs(g[2])));
  return tol + R(sizeof(R) == 4 ? 2e-7 : 1e-15) * m;
}

// §5.4's first case: where the ray is outside the block just behind an entry
// (an entry that only touched the block's boundary, so that the moved entry
// point has no preimage in the block), the entry steps along the ray until
// the ray is inside the block again: 16 probes t0 + k (t1 - t0) / 16 with
// Newton from the chord guesses, then 24 bisections between the last probe
// outside and the first inside.  Returns false if no probe is inside.
template <int P, typename R, bool MIXED>
__device__ bool walk_into_block(const DevVolume& V, const BlockInfo& B, const R o[3], const R d[3], R t0,
                                             R t1, const R p0[3], const R p1[3], R& t_new, R p_new[3],
                                             unsigned long long& iters, unsigned long long& n64) {
  R t_lo = t0, t_hi = t1, p_hi[3], g[3], x[3];
  bool found = false;
  for (int k = 1; k <= 16 && !found; ++k) {
    const R tk = t0 + (t1 - t0) * R(k) / R(16);
    for (int r = 0; r < 3; ++r) {
      const R v = p0[r] + (p1[r] - p0[r]) * R(k) / R(16);
      x[r] = v < R(0) ? R(0) : (v > R(1) ? R(1) : v);
      g[r] = o[r] + tk * d[r];
    }
    if (clip_newton<P, R, MIXED>(V, B, g, x, fixup_tol<R>(g, V.diag), iters, n64)) {
      found = true;
      t_hi = tk;
      for (int r = 0; r < 3; ++r) p_hi[r] = x[r];
    } else {
      t_lo = tk;
    }
  }
  if (!found) return false;
  for (int it = 0; it < 24; ++it) {
    const R tm = R(0.5) * (t_lo + t_hi);
    for (int r = 0; r < 3; ++r) {
      x[r] = p_hi[r];
      g[r] = o[r] + tm * d[r];
    }
    if (clip_newton<P, R, MIXED>(V, B, g, x, fixup_tol<R>(g, V.diag), iters, n64)) {
      t_hi = tm;
      for (int r = 0; r < 3; ++r) p_hi[r] = x[r];
    } else {
      t_lo = tm;
    }
  }
  t_new = t_hi;
  for (int r = 0; r < 3; ++r) p_new[r] = p_hi[r];
  return true;
}

// The clip fix-up: one thread per active pixel solves the flagged ends of
// its pairs; a pair whose end does not invert inside its block gets zero
// length (skipped by stage 3).  Newton starts: an entry listed for the
// learned guess (kGuessIn, guess != NULL) first from the network's guess; then
// from the guess in the pair record (the chord of the segment's ends, the
// exit point for an entry on the near plane, Eq. 22's x_0 for a moved
// singular entry); a moved singular entry (kShrunk) also from the centre of
// the parameter box and from its exit point.
template <int P, typename R, bool MIXED>
__global__ void __launch_bounds__(128) k4_clip_solve(DevVolume V, DevCamera<R> cam, int npix,
                                                     typename Vec4T<R>::type* __restrict__ pair_in,
                                                     typename Vec4T<R>::type* __restrict__ pair_out,
                                                     int* __restrict__ pair_block, const int* __restrict__ pair_count,
                                                     const int* __restrict__ active,
                                                     const int* __restrict__ n_active, const float4* __restrict__ gp,
                                                     const int* __restrict__ gidx, DevStats* __restrict__ st) {
  typedef typename Vec4T<R>::type V4;
  pdl_wait();
  const int nact = *n_active;
  unsigned long long c_it = 0, c_64 = 0;
  for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < nact; item += gridDim.x * blockDim.x) {
    const int pix = active[item];
    const int np = pair_count[pix];
    R o[3], d[3];
    make_ray<R>(cam, cam.x0 + pix % cam.w, cam.y0 + pix / cam.w, o, d);
    for (int q = 0; q < np; ++q) {
      const size_t slot = (size_t)q * npix + pix;
      const int bf = pair_block[slot];
      const int blk = bf & kBlockMask;
      if (!(bf & (kSolveIn | kSolveOut))) {
        if (bf != blk) pair_block[slot] = blk;
        continue;
      }
      const BlockInfo B = V.blocks[blk];
      bool ok = true;
      for (int e = 0; e < 2 && ok; ++e) {
        if (!(bf & (e == 0 ? kSolveIn : kSolveOut))) continue;
        V4 rec = e == 0 ? pair_in[slot] : pair_out[slot];
        const V4 other = e == 0 ? pair_out[slot] : pair_in[slot];
        R g[3], pq[3];
        for (int r = 0; r < 3; ++r) g[r] = o[r] + R(rec.x) * d[r];
        const R tol_g = fixup_tol<R>(g, V.diag);
        const bool learned = e == 0 && (bf & kGuessIn) && gp != nullptr;
        const int n_starts = (e == 0 && (bf & kShrunk)) ? 4 : 2;
        ok = false;
        for (int k = learned ? 0 : 1; k < n_starts && !ok; ++k) {
          if (k == 0) {
            const float4 h = gp[gidx[slot]];
            pq[0] = R(h.x); pq[1] = R(h.y); pq[2] = R(h.z);
          } else if (k == 1) {
            pq[0] = R(rec.y); pq[1] = R(rec.z); pq[2] = R(rec.w);
          } else if (k == 2) {
            pq[0] = pq[1] = pq[2] = R(0.5);
          } else {
            pq[0] = R(other.y); pq[1] = R(other.z); pq[2] = R(other.w);
          }
          for (int r = 0; r < 3; ++r) pq[r] = pq[r] < R(0) ? R(0) : (pq[r] > R(1) ? R(1) : pq[r]);
          ok = clip_newton<P, R, MIXED>(V, B, g, pq, tol_g, c_it, c_64);
        }
        if (!ok && e == 0 && (bf & kShrunk)) {
          // a moved singular entry without a preimage: walk into the block
          R t_new, p0[3] = {R(rec.y), R(rec.z), R(rec.w)};
          const R p1[3] = {R(other.y), R(other.z), R(other.w)};
          ok = walk_into_block<P, R, MIXED>(V, B, o, d, R(rec.x), R(other.x), p0, p1, t_new, pq, c_it, c_64);
          if (ok) rec.x = t_new;
        }
        rec.y = pq[0]; rec.z = pq[1]; rec.w = pq[2];
        if (e == 0) pair_in[slot] = rec; else pair_out[slot] = rec;
      }
      if (!ok) {
        V4 ro = pair_out[slot];
        ro.x = pair_in[slot].x;          // zero length: dropped by stage 3
        pair_out[slot] = ro;
        atomicAdd(&st->unmatched, 1ull);
      }
      pair_block[slot] = blk;
    }
  }
  if (c_it) atomicAdd(&st->entry_newton, c_it);
  if (c_64) atomicAdd(&st->fp64_solves, c_64);
}

// det J at the entry of one pair (FP64 arithmetic on the FP32 Jacobian in
// mixed precision, as the FP64 solves).
template <int P, typename R, bool MIXED>
__device__ __forceinline__ double entry_det(const DevVolume& V, const BlockInfo& B, const R p[3]) {
  R phi[3], J[3][3], rc;
  eval_block<P, R, false>(V, B, p, phi, J, rc);
  if (MIXED || sizeof(R) == 8)
    return (double)J[0][0] * ((double)J[1][1] * J[2][2] - (double)J[1][2] * J[2][1]) -
           (double)J[0][1] * ((double)J[1][0] * J[2][2] - (double)J[1][2] * J[2][0]) +
           (double)J[0][2] * ((double)J[1][0] * J[2][1] - (double)J[1][1] * J[2][0]);
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

// Learned-guess listing (before the clip fix-up): with `singular`, the
// entries of flagged blocks whose det J is below tau_det move delta along
// the ray as §5.4 says (x_0 of Eq. 22 in the pair record, kSolveIn |
// kGuessIn | kShrunk); every kGuessIn entry is then appended to the list
// (world point and block) for the guess network.
template <int P, typename R, bool MIXED>
__global__ void __launch_bounds__(128) k4_guess_mark(DevVolume V, DevCamera<R> cam, int npix,
                                                     typename Vec4T<R>::type* __restrict__ pair_in,
                                                     typename Vec4T<R>::type* __restrict__ pair_out,
                                                     int* __restrict__ pair_block, const int* __restrict__ pair_count,
                                                     const int* __restrict__ active,
                                                     const int* __restrict__ n_active, int singular, GuessList gl,
                                                     DevStats* __restrict__ st) {
  typedef typename Vec4T<R>::type V4;
  pdl_wait();
  const int nact = *n_active;
  const R delta = R(1e-4) * R(V.diag), eps = R(1e-4);
  unsigned long long c_shrink = 0, c_drop = 0;
  for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < nact; item += gridDim.x * blockDim.x) {
    const int pix = active[item];
    const int np = pair_count[pix];
    R o[3], d[3];
    make_ray<R>(cam, cam.x0 + pix % cam.w, cam.y0 + pix / cam.w, o, d);
    for (int q = 0; q < np; ++q) {
      const size_t slot = (size_t)q * npix + pix;
      int bf = pair_block[slot];
      const BlockInfo B = V.blocks[bf & kBlockMask];
      V4 in = pair_in[slot];
      const V4 out = pair_out[slot];
      if (singular && B.sing_faces && !(bf & kSolveIn) && out.x > in.x) {
        const R p[3] = {R(in.y), R(in.z), R(in.w)};
        if (fabs(entry_det<P, R, MIXED>(V, B, p)) < (double)B.tau_det) {
          ++c_shrink;
          if (!(R(out.x) - R(in.x) > delta)) {
            V4 ro = out;
            ro.x = in.x;                                 // zero length: dropped by stage 3
            pair_out[slot] = ro;
            ++c_drop;
          } else {
            R dir[3] = {R(out.y) - p[0], R(out.z) - p[1], R(out.w) - p[2]};
            const R nd = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
            in.x = R(in.x) + delta;
            const R x0[3] = {p[0] + (nd > R(0) ? eps * dir[0] / nd : R(0)),
                             p[1] + (nd > R(0) ? eps * dir[1] / nd : R(0)),
                             p[2] + (nd > R(0) ? eps * dir[2] / nd : R(0))};
            in.y = x0[0]; in.z = x0[1]; in.w = x0[2];
            pair_in[slot] = in;
            bf |= kSolveIn | kGuessIn | kShrunk;
          }
        }
      }
      if (bf & kGuessIn) {
        const int k = atomicAdd(gl.n, 1);
        const R t = R(in.x);
        gl.g[k] = make_float4(float(o[0] + t * d[0]), float(o[1] + t * d[1]), float(o[2] + t * d[2]), 0.f);
        gl.blk[k] = bf & kBlockMask;
        gl.gidx[slot] = k;
      }
      pair_block[slot] = bf;
    }
  }
  if (c_shrink) atomicAdd(&st->entry_shrinks, c_shrink);
  if (c_drop) atomicAdd(&st->unmatched, c_drop);
}

// §5.4, singular Jacobian at the entry point (Eq. 22): for the pairs of
// blocks with a face flagged at creation (det J comes close to 0 there),
// det J is evaluated at the entry; below tau_det (1e-6 of the block's mean
// |det J|) neither Newton nor the ODE's linear system can start there, so the
// block is "shrunk": the entry moves delta = 1e-4 diag along the ray and its
// parameter point is found by Newton from x_0 = p_in + eps (p_out - p_in) /
// |p_out - p_in|, eps = 1e-4 (Eq. 22).  A pair not longer than delta, or
// whose new entry does not invert inside the block, gets zero length
// (stage 3 skips it).  One thread per active pixel.
template <int P, typename R, bool MIXED>
__global__ void __launch_bounds__(128) k4_entry_fix(DevVolume V, DevCamera<R> cam, int npix,
                                                    typename Vec4T<R>::type* __restrict__ pair_in,
                                                    typename Vec4T<R>::type* __restrict__ pair_out,
                                                    const int* __restrict__ pair_block,
                                                    const int* __restrict__ pair_count,
                                                    const int* __restrict__ active, const int* __restrict__ n_active,
                                                    DevStats* __restrict__ st) {
  typedef typename Vec4T<R>::type V4;
  pdl_wait();
  const int nact = *n_active;
  const R delta = R(1e-4) * R(V.diag), eps = R(1e-4);
  unsigned long long c_shrink = 0, c_it = 0, c_64 = 0, c_drop = 0;
  for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < nact; item += gridDim.x * blockDim.x) {
    const int pix = active[item];
    const int np = pair_count[pix];
    R o[3], d[3];
    make_ray<R>(cam, cam.x0 + pix % cam.w, cam.y0 + pix / cam.w, o, d);
    for (int q = 0; q < np; ++q) {
      const size_t slot = (size_t)q * npix + pix;
      const BlockInfo B = V.blocks[pair_block[slot] & kBlockMask];
      if (!B.sing_faces) continue;
      V4 in = pair_in[slot];
      const V4 out = pair_out[slot];
      if (!(out.x > in.x)) continue;                     // already empty
      const R p[3] = {R(in.y), R(in.z), R(in.w)};
      if (!(fabs(entry_det<P, R, MIXED>(V, B, p)) < (double)B.tau_det)) continue;
      ++c_shrink;
      bool ok = R(out.x) - R(in.x) > delta;
      if (ok) {
        R dir[3] = {R(out.y) - p[0], R(out.z) - p[1], R(out.w) - p[2]};
        const R nd = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
        R x[3], g[3];
        const R t_in = R(in.x) + delta;
        for (int r = 0; r < 3; ++r) g[r] = o[r] + t_in * d[r];
        // Newton from Eq. 22's x_0; where the map degenerates faster than
        // linearly toward the face, Newton from x_0 overshoots out of the
        // block and its line search cannot recover: then from the centre of
        // the parameter box, then from the exit point (the root is unique)
        const R tol_g = fixup_tol<R>(g, V.diag);
        const R p_out[3] = {R(out.y), R(out.z), R(out.w)};
        ok = false;
        for (int k = 0; k < 3 && !ok; ++k) {
          for (int r = 0; r < 3; ++r) {
            const R v = k == 0 ? p[r] + (nd > R(0) ? eps * dir[r] / nd : R(0)) : (k == 1 ? R(0.5) : p_out[r]);
            x[r] = v < R(0) ? R(0) : (v > R(1) ? R(1) : v);
          }
          ok = clip_newton<P, R, MIXED>(V, B, g, x, tol_g, c_it, c_64);
        }
        R t_new = t_in;
        if (!ok) ok = walk_into_block<P, R, MIXED>(V, B, o, d, t_in, R(out.x), p, p_out, t_new, x, c_it, c_64);
        if (ok) {
          in.x = t_new;
          in.y = x[0];
          in.z = x[1];
          in.w = x[2];
          pair_in[slot] = in;
        }
      }
      if (!ok) {
        V4 ro = out;
        ro.x = in.x;                                     // zero length: dropped by stage 3
        pair_out[slot] = ro;
        ++c_drop;
      }
    }
  }
  if (c_shrink) atomicAdd(&st->entry_shrinks, c_shrink);
  if (c_it) atomicAdd(&st->entry_newton, c_it);
  if (c_64) atomicAdd(&st->fp64_solves, c_64);
  if (c_drop) atomicAdd(&st->unmatched, c_drop);
}

// Block-aggregated append of the active pixels to the integrator's queue
// (every thread of the 256-thread block of one 16 x 16 tile calls it): the
// tile's active pixels land contiguously, so the 32 consecutive queue items
// an integrator warp takes are neighbours even where the tile is only partly
// covered.  Within the tile they are grouped by path length len (8 bands
// relative to the tile's longest, longest first; warp tile order within a
// band), so that the pixels of one warp take similar times: the integrators
// refill a warp only when all its lanes are idle.  Also the counters that
// every render keeps.
__device__ __forceinline__ void pair_epilogue(int pix, int np, float len, unsigned um, unsigned pov,
                                              int* __restrict__ active, int* __restrict__ n_active,
                                              DevStats* __restrict__ st, int ns = 0,
                                              const SampleCount* sc = nullptr) {
  constexpr int kBands = 8;
  __shared__ int s_cnt[kBands][8];    // [band][warp]: active pixels, then their offsets
  __shared__ unsigned s_max;
  __shared__ int s_base, s_tot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool act = np > 0;
  const float key = act && isfinite(len) && len > 0.f ? len : 0.f;   // a non-finite length goes to band 0
  unsigned wmax = __float_as_uint(key);           // non-negative floats order as their bits
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
  if (threadIdx.x == 0) s_max = 0u;
  __syncthreads();
  if (lane == 0) atomicMax(&s_max, wmax);
  __syncthreads();
  const float kmax = __uint_as_float(s_max);
  const int band = kmax > 0.f ? max(0, min(kBands - 1, (int)((float)kBands * (key / kmax)))) : 0;
  unsigned my_band_mask = 0u;
#pragma unroll
  for (int b = 0; b < kBands; ++b) {
    const unsigned m = __ballot_sync(0xffffffffu, act && band == b);
    if (band == b) my_band_mask = m;
    if (lane == 0) s_cnt[b][warp] = __popc(m);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int b = kBands - 1; b >= 0; --b)         // longest band first
      for (int w = 0; w < 8; ++w) {
        const int c = s_cnt[b][w];
        s_cnt[b][w] = tot;
        tot += c;
      }
    s_base = tot > 0 ? atomicAdd(n_active, tot) : 0;
    s_tot = tot;
  }
  __syncthreads();
  const int loc = act ? s_cnt[band][warp] + __popc(my_band_mask & ((1u << lane) - 1u)) : 0;
  if (act) active[s_base + loc] = pix;
  if (sc != nullptr) {
    // the tile's run of the sample list: an exclusive scan of its active
    // pixels' sample counts in queue order, one atomic for the tile
    __shared__ int s_ns[256];
    __shared__ int s_wsum[8];
    __shared__ int s_sbase;
    const int tot = s_tot;
    if (act) s_ns[loc] = ns;
    __syncthreads();
    const int v = (int)threadIdx.x < tot ? s_ns[threadIdx.x] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int w = 0; w < 8; ++w) {
        const int c = s_wsum[w];
        s_wsum[w] = acc;
        acc += c;
      }
      int b = 0;
      if (acc > 0) {
        b = atomicAdd(sc->total, acc);
        if (b < 0 || b > 0x7fffffff - acc) sc->total[1] = 1;     // the list passed INT_MAX
      }
      s_sbase = b;
    }
    __syncthreads();
    if ((int)threadIdx.x < tot) {
      const int item = s_base + (int)threadIdx.x;
      sc->off[item] = s_sbase + s_wsum[warp] + incl - v;
      sc->cnt[item] = v;
    }
  }
  unsigned long long cu = um, cp = pov, cr = act ? 1 : 0, cpairs = np;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cu += __shfl_down_sync(0xffffffffu, cu, o);
    cp += __shfl_down_sync(0xffffffffu, cp, o);
    cr += __shfl_down_sync(0xffffffffu, cr, o);
    cpairs += __shfl_down_sync(0xffffffffu, cpairs, o);
  }
  if (lane == 0) {
    if (cu) atomicAdd(&st->unmatched, cu);
    if (cp) atomicAdd(&st->pair_overflow, cp);
    if (cr) atomicAdd(&st->rays, cr);
    if (cpairs) atomicAdd(&st->pairs, cpairs);
  }
}

// Pixel of thread threadIdx.x of 16x16 tile (tx, ty): warp w covers the 8x4
// block at (8 (w & 1), 4 (w >> 1)) of the tile.  Pixels are queued in this
// order, so the 32 lanes of an integrator warp start on a compact pixel block
// whose rays cross the same elements (shared control-point loads).
__device__ __forceinline__ void tile_pixel(int tx, int ty, int& x, int& y) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  x = tx * 16 + (warp & 1) * 8 + (lane & 7);
  y = ty * 16 + (warp >> 1) * 4 + (lane >> 3);
}

template <typename R>
__global__ void __launch_bounds__(256) k4_pair(int w, int npix, R tau_dup, const typename Vec4T<R>::type* __restrict__ frag_tp,
                                               const unsigned* __restrict__ frag_meta,
                                               const int* __restrict__ frag_count,
                                               typename Vec4T<R>::type* __restrict__ pair_in,
                                               typename Vec4T<R>::type* __restrict__ pair_out,
                                               int* __restrict__ pair_block, int* __restrict__ pair_count,
                                               int max_pairs, int* __restrict__ active, int* __restrict__ n_active,
                                               float4* __restrict__ out_rgba, ClipArgs<R> clip,
                                               int* __restrict__ tile_flag, int max_frags, SampleCount sc,
                                               DevStats* __restrict__ st) {
  pdl_wait();
  // a tile none of whose warp tiles had a candidate patch was finished by
  // the cull (pair counts and zero pixels): nothing to do
  if (tile_flag != nullptr && tile_flag[blockIdx.x] == 0) return;
  const int tiles_x = (w + 15) / 16;
  int x, y;
  tile_pixel(blockIdx.x % tiles_x, blockIdx.x / tiles_x, x, y);
  const int pix = y * w + x;
  int np = 0;
  unsigned um = 0, pov = 0;
  if (x < w && pix < npix) {
    if (clip.on)
      np = pair_pixel_clip<R>(pix, npix, tau_dup, frag_tp, frag_meta, frag_count, pair_in, pair_out, pair_block,
                              pair_count, max_pairs, out_rgba ? out_rgba + pix : nullptr, um, pov, clip, x, y,
                              max_frags);
    else
      np = pair_pixel<R>(pix, npix, tau_dup, frag_tp, frag_meta, frag_count, pair_in, pair_out, pair_block,
                         pair_count, max_pairs, out_rgba ? out_rgba + pix : nullptr, um, pov, max_frags);
  }
  float len = 0.f;                                  // the pixel's path length through the volume
  int ns = 0;                                       // its samples (counted here when sc.off is set)
  for (int q = 0; q < np; ++q) {
    const size_t o = (size_t)q * npix + pix;
    const float L = (float)(pair_out[o].x - pair_in[o].x);
    len += L;
    if (sc.off != nullptr && L > 0.f) ns += pair_sample_count(L, sc.ds, sc.tail_eps);
  }
  pair_epilogue(pix, np, len, um, pov, active, n_active, st, ns, sc.off != nullptr ? &sc : nullptr);
  // every thread read the flag before the epilogue's barriers: clear it for
  // the next frame
  if (tile_flag != nullptr && threadIdx.x == 0) tile_flag[blockIdx.x] = 0;
}

// Batched form: pixel `pix` of the batch's pixel space belongs to request
// rq with pix0[rq] <= pix < pix0[rq + 1]; its duplicate tolerance follows
// the request's volume and its empty-pixel zero goes to the request's image.
__global__ void __launch_bounds__(256) kb4_pair(BatchArgs ba, int npix, const float4* __restrict__ frag_tp,
                                                const unsigned* __restrict__ frag_meta,
                                                const int* __restrict__ frag_count, float4* __restrict__ pair_in,
                                                float4* __restrict__ pair_out, int* __restrict__ pair_block,
                                                int* __restrict__ pair_count, int* __restrict__ active,
                                                int* __restrict__ n_active, DevStats* __restrict__ st) {
  const int rq = batch_find(ba.tile16, ba.nreq, blockIdx.x);
  const DevRequest& q = ba.req[rq];
  const int t = blockIdx.x - __ldg(ba.tile16 + rq);
  const int tiles_x = (q.cam.w + 15) / 16;
  int x, y;
  tile_pixel(t % tiles_x, t / tiles_x, x, y);
  const int pix = __ldg(ba.pix0 + rq) + y * q.cam.w + x;
  int np = 0;
  unsigned um = 0, pov = 0;
  if (x < q.cam.w && y < q.cam.h) {
    const float tau = 1e-5f * q.diag;
    np = pair_pixel<float>(pix, npix, tau, frag_tp, frag_meta, frag_count, pair_in, pair_out, pair_block,
                           pair_count, kMaxPairs, q.out + (pix - __ldg(ba.pix0 + rq)), um, pov);
  }
  pair_epilogue(pix, np, 0.f, um, pov, active, n_active, st);
}

}  // namespace

template <typename R>
void launch_pair(const DevVolume& V, int w, int npix, float diag, const typename Vec4T<R>::type* frag_tp,
                 const unsigned* frag_meta, const int* frag_count, typename Vec4T<R>::type* pair_in,
                 typename Vec4T<R>::type* pair_out, int* pair_block, int* pair_count, int max_pairs, int* active,
                 int* n_active, float4* out_rgba_zero, const ClipArgs<R>& clip, int* tile_flag, DevStats* st,
                 cudaStream_t s, const SampleCount* count) {
  if (npix <= 0) return;
  const R tau = sizeof(R) == 4 ? R(1e-5) * R(diag) : R(1e-9) * R(diag);
  if (w <= 0) return;
  const int h = npix / w;
  SampleCount sc{0.f, 0.f, nullptr, nullptr, nullptr};
  if (count != nullptr) sc = *count;
  launch_pdl(k4_pair<R>, dim3(((w + 15) / 16) * ((h + 15) / 16)), dim3(256), s, w, npix, tau, frag_tp, frag_meta,
             frag_count, pair_in, pair_out, pair_block, pair_count, max_pairs, active, n_active, out_rgba_zero, clip,
             tile_flag, V.max_frags, sc, st);
}

void launch_batch_pair(const BatchArgs& ba, int tiles16, int npix, const float4* frag_tp, const unsigned* frag_meta,
                       const int* frag_count, float4* pair_in, float4* pair_out, int* pair_block, int* pair_count,
                       int* active, int* n_active, DevStats* st, cudaStream_t s) {
  if (npix <= 0 || tiles16 <= 0) return;
  kb4_pair<<<tiles16, 256, 0, s>>>(ba, npix, frag_tp, frag_meta, frag_count, pair_in, pair_out,
                                             pair_block, pair_count, active, n_active, st);
}

template void launch_pair<float>(const DevVolume&, int, int, float, const float4*, const unsigned*, const int*,
                                 float4*, float4*, int*, int*, int, int*, int*, float4*, const ClipArgs<float>&,
                                 int*, DevStats*, cudaStream_t, const SampleCount*);
template void launch_pair<double>(const DevVolume&, int, int, float, const Dbl4*, const unsigned*, const int*, Dbl4*,
                                  Dbl4*, int*, int*, int, int*, int*, float4*, const ClipArgs<double>&, int*,
                                  DevStats*, cudaStream_t, const SampleCount*);

template <typename R>
void launch_clip_solve(const DevVolume& V, const DevCamera<R>& cam, int npix, typename Vec4T<R>::type* pair_in,
                       typename Vec4T<R>::type* pair_out, int* pair_block, const int* pair_count, const int* active,
                       const int* n_active, bool mixed, const GuessList* guess, DevStats* st, int num_sms,
                       cudaStream_t s) {
  if (npix <= 0) return;
  int grid = num_sms * 8;
  const int useful = (npix + 127) / 128;
  grid = grid < useful ? grid : useful;
  const float4* gp = guess ? guess->p : nullptr;
  const int* gidx = guess ? guess->gidx : nullptr;
#define IVV_CLIP(PP, MM)                                                                                        \
  launch_pdl(k4_clip_solve<PP, R, MM>, dim3(grid), dim3(128), s, V, cam, npix, pair_in, pair_out, pair_block, \
             pair_count, active, n_active, gp, gidx, st)
  const bool m = mixed && sizeof(R) == 4;
  if (V.P == 2) {
    if (m) IVV_CLIP(2, true); else IVV_CLIP(2, false);
  } else {
    if (m) IVV_CLIP(3, true); else IVV_CLIP(3, false);
  }
#undef IVV_CLIP
}

template void launch_clip_solve<float>(const DevVolume&, const DevCamera<float>&, int, float4*, float4*, int*,
                                       const int*, const int*, const int*, bool, const GuessList*, DevStats*, int,
                                       cudaStream_t);
template void launch_clip_solve<double>(const DevVolume&, const DevCamera<double>&, int, Dbl4*, Dbl4*, int*,
                                        const int*, const int*, const int*, bool, const GuessList*, DevStats*, int,
                                        cudaStream_t);

template <typename R>
void launch_guess_mark(const DevVolume& V, const DevCamera<R>& cam, int npix, typename Vec4T<R>::type* pair_in,
                       typename Vec4T<R>::type* pair_out, int* pair_block, const int* pair_count, const int* active,
                       const int* n_active, bool singular, bool mixed, const GuessList& guess, DevStats* st,
                       int num_sms, cudaStream_t s) {
  if (npix <= 0) return;
  int grid = num_sms * 8;
  const int useful = (npix + 127) / 128;
  grid = grid < useful ? grid : useful;
  const int sg = singular ? 1 : 0;
#define IVV_MARK(PP, MM)                                                                                        \
  launch_pdl(k4_guess_mark<PP, R, MM>, dim3(grid), dim3(128), s, V, cam, npix, pair_in, pair_out, pair_block, \
             pair_count, active, n_active, sg, guess, st)
  const bool m = mixed && sizeof(R) == 4;
  if (V.P == 2) {
    if (m) IVV_MARK(2, true); else IVV_MARK(2, false);
  } else {
    if (m) IVV_MARK(3, true); else IVV_MARK(3, false);
  }
#undef IVV_MARK
}

template void launch_guess_mark<float>(const DevVolume&, const DevCamera<float>&, int, float4*, float4*, int*,
                                       const int*, const int*, const int*, bool, bool, const GuessList&, DevStats*,
                                       int, cudaStream_t);
template void launch_guess_mark<double>(const DevVolume&, const DevCamera<double>&, int, Dbl4*, Dbl4*, int*,
                                        const int*, const int*, const int*, bool, bool, const GuessList&, DevStats*,
                                        int, cudaStream_t);

template <typename R>
void launch_entry_fix(const DevVolume& V, const DevCamera<R>& cam, int npix, typename Vec4T<R>::type* pair_in,
                      typename Vec4T<R>::type* pair_out, const int* pair_block, const int* pair_count,
                      const int* active, const int* n_active, bool mixed, DevStats* st, int num_sms, cudaStream_t s) {
  if (npix <= 0) return;
  int grid = num_sms * 8;
  const int useful = (npix + 127) / 128;
  grid = grid < useful ? grid : useful;
#define IVV_FIX(PP, MM)                                                                                          \
  launch_pdl(k4_entry_fix<PP, R, MM>, dim3(grid), dim3(128), s, V, cam, npix, pair_in, pair_out, pair_block,   \
             pair_count, active, n_active, st)
  const bool m = mixed && sizeof(R) == 4;
  if (V.P == 2) {
    if (m) IVV_FIX(2, true); else IVV_FIX(2, false);
  } else {
    if (m) IVV_FIX(3, true); else IVV_FIX(3, false);
  }
#undef IVV_FIX
}

template void launch_entry_fix<float>(const DevVolume&, const DevCamera<float>&, int, float4*, float4*, const int*,
                                      const int*, const int*, const int*, bool, DevStats*, int, cudaStream_t);
template void launch_entry_fix<double>(const DevVolume&, const DevCamera<double>&, int, Dbl4*, Dbl4*, const int*,
                                       const int*, const int*, const int*, bool, DevStats*, int, cudaStream_t);

}  // namespace ivv

namespace ivv {
namespace {

__global__ void k_export_pairs(int npix, int max_pairs, const float4* __restrict__ pin, const float4* __restrict__ pout,
                               const int* __restrict__ pblk, const int* __restrict__ pcnt, int* __restrict__ out_count,
                               float* __restrict__ out_pairs, int* __restrict__ out_block) {
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  int n = pcnt[pix];
  n = n < max_pairs ? n : max_pairs;
  out_count[pix] = n;
  for (int q = 0; q < n; ++q) {
    const size_t s = (size_t)q * npix + pix;
    const float4 a = pin[s], b = pout[s];
    float* o = out_pairs + s * 8;
    o[0] = a.y; o[1] = a.z; o[2] = a.w; o[3] = a.x;
    o[4] = b.y; o[5] = b.z; o[6] = b.w; o[7] = b.x;
    out_block[s] = pblk[s];
  }
}

}  // namespace

void launch_export_pairs(int npix, int max_pairs, bool fp64, const void* pin, const void* pout, const int* pblk,
                         const int* pcnt, int* out_count, float* out_pairs, int* out_block, cudaStream_t s) {
  (void)fp64;
  if (npix <= 0) return;
  k_export_pairs<<<(npix + 255) / 256, 256, 0, s>>>(npix, max_pairs, (const float4*)pin, (const float4*)pout, pblk,
                                                    pcnt, out_count, out_pairs, out_block);
}

}  // namespace ivv
