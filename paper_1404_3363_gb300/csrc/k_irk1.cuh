// Stage 3 with the paper's implicit Euler method (§5.2): one step per sample
// interval [s_j, s_{j+1}] of the pulled-back ODE p' = W(p) (§5.2),
//     p_{j+1} = p_j + h W(p_{j+1}),   h = s_{j+1} - s_j,
// solved for the increment z = p_{j+1} - p_j by Newton on
//     G(z) = z - h W(p_j + z) = 0
// with the exact Jacobian of G: differentiating J_phi G = J_phi z - h V(phi)
// gives
//     J_phi(x) J_G(z) = H_phi(x)[z - G(z)] + (I - h J_V) J_phi(x),  x = p_j + z,
// J_V = c (d d^T - I) for V(g) = d + c [(g_in - g) - <g_in - g, d> d], and
// H_phi(x)[v]_{ab} = sum_k d^2 phi_a / dx_b dx_k v_k.  A Newton step solves
// (J_phi J_G) dz = -J_phi G; both 3x3 systems go through the adjugate.
// z starts at 0, so the first Newton iteration of a step evaluates the map at
// the sample point p_j itself, which also gives the scalar there for the
// compositing of [s_{j-1}, s_j] (Alg. 1, as K5).  Newton iterates may leave
// the parameter box: the boundary element's polynomials are continued there,
// so G stays smooth; a converged step (|dz|_inf <= kIrkTol) ends at p_j + z
// clamped to [0,1]^3 (§5.4: the ray is followed along the boundary).  A step
// whose Newton does not converge within kIrkMaxIter iterations, or meets a
// singular system (the map degenerates near the ray), falls back to the
// clamped explicit Euler step p_j + h W(p_j).
//
// K5i integrate_irk1 -- persistent kernel over the same work queue as K5;
// one map evaluation (phi, J_phi, H_phi and, in control-point mode, rho) per
// lane and loop iteration.
#pragma once

#include "k_integrate.cuh"

namespace ivv {

constexpr float kIrkTol = 2e-6f;   // |dz|_inf at which a Newton solve stops (FP32)
constexpr int kIrkMaxIter = 12;

// Bernstein polynomials of degree P at x with first and second derivatives.
template <int P>
__device__ __forceinline__ void bernstein2(float x, float b[P + 1], float db[P + 1], float ddb[P + 1]) {
  const float y = 1.f - x;
  if (P == 2) {
    b[0] = y * y; b[1] = 2.f * x * y; b[2] = x * x;
    db[0] = -2.f * y; db[1] = 2.f - 4.f * x; db[2] = 2.f * x;
    ddb[0] = 2.f; ddb[1] = -4.f; ddb[2] = 2.f;
  } else {
    const float x2 = x * x, y2 = y * y;
    b[0] = y2 * y; b[1] = 3.f * x * y2; b[2] = 3.f * x2 * y; b[3] = x2 * x;
    db[0] = -3.f * y2; db[1] = 3.f * y * (1.f - 3.f * x);
    db[2] = 3.f * x * (2.f - 3.f * x); db[3] = 3.f * x2;
    ddb[0] = 6.f * y; ddb[1] = 6.f * x - 12.f * y; ddb[2] = 6.f * y - 12.f * x; ddb[3] = 6.f * x;
  }
}

// phi, J (J[r][a] = d phi_r / dp_a), the Hessian H[r][a][b] and (control
// points mode) the scalar at p of block B (outside [0,1]^3 the nearest
// element's polynomials are continued), sum-factorised: for each i the
// (j, k) slab is contracted along w (value, first and second w-derivative),
// then along v, then the u contraction accumulates the ten distinct partials
// per channel.
template <int P>
__device__ __forceinline__ void eval_block_h(const DevVolume& V, const BlockInfo& B, const float p[3], float phi[3],
                                             float J[3][3], float H[3][3][3], float& rho) {
  constexpr int N = P + 1;
  float loc[3], sc[3];
  int e[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float x = p[d];
    const float xc = x < 0.f ? 0.f : (x > 1.f ? 1.f : x);
    if ((B.uniform >> d) & 1) {
      int k = (int)(xc * (float)B.nseg[d]);
      k = k < B.nseg[d] - 1 ? k : B.nseg[d] - 1;
      e[d] = k;
      loc[d] = x * (float)B.nseg[d] - (float)k;
      sc[d] = (float)B.nseg[d];
    } else {
      float lc;
      e[d] = locate<float>(V.brk32 + B.brk_off[d], B.nseg[d], xc, lc, sc[d]);
      loc[d] = (x - __ldg(V.brk32 + B.brk_off[d] + e[d])) * sc[d];
    }
  }
  const size_t eid = (size_t)(B.elem_off + (e[2] * B.nseg[1] + e[1]) * B.nseg[0] + e[0]);
  const float4* cp = V.elem32 + eid * (N * N * N);
  float bu[N], dbu[N], ddbu[N], bv[N], dbv[N], ddbv[N], bw[N], dbw[N], ddbw[N];
  bernstein2<P>(loc[0], bu, dbu, ddbu);
  bernstein2<P>(loc[1], bv, dbv, ddbv);
  bernstein2<P>(loc[2], bw, dbw, ddbw);
  // u-level accumulators per channel: value, u, v, w, uu, uv, uw, vv, vw, ww
  float acc[10][3];
#pragma unroll
  for (int q = 0; q < 10; ++q) acc[q][0] = acc[q][1] = acc[q][2] = 0.f;
  float s = 0.f;
#pragma unroll 1
  for (int i = 0; i < N; ++i) {
    // v-level: value, v, vv of the w-value; value, v of the w-derivative; value of w''
    float s00[3] = {0, 0, 0}, s01[3] = {0, 0, 0}, s02[3] = {0, 0, 0}, s10[3] = {0, 0, 0}, s11[3] = {0, 0, 0},
          s20[3] = {0, 0, 0};
    float ss = 0.f;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float4 row[N];
      ldg_row<N>(cp + (i * N + j) * N, row);
      float t0[3] = {0, 0, 0}, t1[3] = {0, 0, 0}, t2[3] = {0, 0, 0};
      float ts = 0.f;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const float c[3] = {row[k].x, row[k].y, row[k].z};
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          t0[r] = fmaf(bw[k], c[r], t0[r]);
          t1[r] = fmaf(dbw[k], c[r], t1[r]);
          t2[r] = fmaf(ddbw[k], c[r], t2[r]);
        }
        ts = fmaf(bw[k], row[k].w, ts);
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        s00[r] = fmaf(bv[j], t0[r], s00[r]);
        s01[r] = fmaf(dbv[j], t0[r], s01[r]);
        s02[r] = fmaf(ddbv[j], t0[r], s02[r]);
        s10[r] = fmaf(bv[j], t1[r], s10[r]);
        s11[r] = fmaf(dbv[j], t1[r], s11[r]);
        s20[r] = fmaf(bv[j], t2[r], s20[r]);
      }
      ss = fmaf(bv[j], ts, ss);
    }
    const float u0 = pick<N>(bu, i), u1 = pick<N>(dbu, i), u2 = pick<N>(ddbu, i);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      acc[0][r] = fmaf(u0, s00[r], acc[0][r]);   // value
      acc[1][r] = fmaf(u1, s00[r], acc[1][r]);   // u
      acc[2][r] = fmaf(u0, s01[r], acc[2][r]);   // v
      acc[3][r] = fmaf(u0, s10[r], acc[3][r]);   // w
      acc[4][r] = fmaf(u2, s00[r], acc[4][r]);   // uu
      acc[5][r] = fmaf(u1, s01[r], acc[5][r]);   // uv
      acc[6][r] = fmaf(u1, s10[r], acc[6][r]);   // uw
      acc[7][r] = fmaf(u0, s02[r], acc[7][r]);   // vv
      acc[8][r] = fmaf(u0, s11[r], acc[8][r]);   // vw
      acc[9][r] = fmaf(u0, s20[r], acc[9][r]);   // ww
    }
    s = fmaf(u0, ss, s);
  }
  const float4 og = __ldg(V.org32 + eid);
  phi[0] = acc[0][0] + og.x;
  phi[1] = acc[0][1] + og.y;
  phi[2] = acc[0][2] + og.z;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    J[r][0] = acc[1][r] * sc[0];
    J[r][1] = acc[2][r] * sc[1];
    J[r][2] = acc[3][r] * sc[2];
    H[r][0][0] = acc[4][r] * sc[0] * sc[0];
    H[r][0][1] = H[r][1][0] = acc[5][r] * sc[0] * sc[1];
    H[r][0][2] = H[r][2][0] = acc[6][r] * sc[0] * sc[2];
    H[r][1][1] = acc[7][r] * sc[1] * sc[1];
    H[r][1][2] = H[r][2][1] = acc[8][r] * sc[1] * sc[2];
    H[r][2][2] = acc[9][r] * sc[2] * sc[2];
  }
  rho = s;
}

// Solve A x = b in R (the adjugate); returns det A.
template <typename R>
__device__ __forceinline__ R solve3_any(const float A[3][3], const float b[3], float x[3]) {
  R Ad[3][3], bd[3], xd[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    bd[r] = R(b[r]);
#pragma unroll
    for (int k = 0; k < 3; ++k) Ad[r][k] = R(A[r][k]);
  }
  const R det = solve3<R>(Ad, bd, xd);
#pragma unroll
  for (int r = 0; r < 3; ++r) x[r] = float(xd[r]);
  return det;
}

template <int P, bool MIXED, bool STATS>
__global__ void __launch_bounds__(128, 3) k5_irk1(DevVolume V, DevCamera<float> cam, DevTF tf, IntegrateArgs args,
                                                  const float4* __restrict__ pair_in,
                                                  const float4* __restrict__ pair_out,
                                                  const int* __restrict__ pair_block,
                                                  const int* __restrict__ pair_count,
                                                  const int* __restrict__ active, const int* __restrict__ n_active,
                                                  int* __restrict__ queue_head, float4* __restrict__ out,
                                                  DevStats* __restrict__ st) {
  __shared__ float s_r[256];
  __shared__ float4 s_rgba[256];
  __shared__ unsigned char s_seg[kTfTable];
  for (int i = threadIdx.x; i < tf.n; i += blockDim.x) {
    s_r[i] = tf.r[i];
    s_rgba[i] = tf.rgba[i];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kTfTable; i += blockDim.x) {
    const float x = (float)i / (float)kTfTable;
    int k = 0;
    while (k < tf.n - 2 && s_r[k + 1] <= x) ++k;
    s_seg[i] = (unsigned char)k;
  }
  __syncthreads();
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int nact = *n_active;
  if (nact == 0) return;
  const int npix = args.npix;
  const float ds = args.ds, cc = args.c, early = args.early_alpha;
  const float tail_eps = 1e-12f * V.diag;
  unsigned long long c_eval = 0, c_steps = 0, c_samp = 0, c_fp64 = 0, c_cap = 0;
  float max_dp = 0.f;

  int pix = -1;           // -1: needs a pixel; -2: queue drained
  int q = 0, np = 0, j = 0, nsamp = 0, nlast = 0, it = 0;
  bool fresh = true;      // the lane needs its next pair
  BlockInfo B = V.blocks[0];
  float d[3], g_in[3], p[3], z[3], v0[3];
  float h = 0.f, L = 0.f, rho_prev = 0.f;
  Acc<float> acc;

  WarpQueue wq(nact, queue_head, nullptr);
  for (;;) {
    if (__ballot_sync(0xffffffffu, pix >= 0) == 0) {     // the whole warp is idle: refill
      if (wq.done()) break;
      const int item = wq.take(lane, queue_head);
      if (pix == -1) {
        if (item < nact) {
          pix = __ldg(active + item);
          acc.C[0] = acc.C[1] = acc.C[2] = acc.a = 0.f;
          np = __ldg(pair_count + pix);
          q = -1;
          fresh = true;
        } else {
          pix = -2;
        }
      }
      wq.drained |= __ballot_sync(0xffffffffu, pix == -2);
    }

    bool live = pix >= 0;
    if (live && fresh) {
      bool found = false;
      while (!found && ++q < np) {
        const size_t slot = (size_t)q * npix + pix;
        const float4 pi = pair_in[slot];
        const float4 po = pair_out[slot];
        L = po.x - pi.x;
        if (!(L > 0.f)) continue;
        B = V.blocks[__ldg(pair_block + slot)];
        float o[3];
        make_ray<float>(cam, cam.x0 + pix % cam.w, cam.y0 + pix / cam.w, o, d);
#pragma unroll
        for (int r = 0; r < 3; ++r) g_in[r] = o[r] + pi.x * d[r];
        p[0] = pi.y; p[1] = pi.z; p[2] = pi.w;
        const float fl = floorf(L / ds);
        nsamp = (int)fl;
        nlast = nsamp + ((L - fl * ds > tail_eps) ? 1 : 0);
        j = 0;
        it = 0;
        z[0] = z[1] = z[2] = 0.f;
        found = true;
      }
      fresh = false;
      if (!found) {
        out[pix] = make_float4(acc.C[0], acc.C[1], acc.C[2], acc.a);
        pix = -1;
        live = false;
      }
    }
    if (!live) continue;                             // idle lanes issue no loads
    // ---- this iteration's evaluation point x = p + z (may leave the box)
    float x[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) x[r] = p[r] + z[r];
    float phi[3], J[3][3], H[3][3][3], rc;
    eval_block_h<P>(V, B, x, phi, J, H, rc);
    if (STATS) ++c_eval;
    if (it == 0) {
      // x is the sample point p_j: its scalar, and the interval ending there
      float rho;
      rho = scalar_at<P, float>(V, B, V.mode, x, J, rc);
      if (j > 0) {
        const float s1 = (j <= nsamp) ? (float)j * ds : L;
        composite_interval<float>(s_r, s_rgba, s_seg, tf, args.K, rho_prev, rho, s1 - (float)(j - 1) * ds, acc);
      }
      if (STATS) {
        ++c_samp;
        max_dp = fmaxf(max_dp, pixel_error<float>(cam, phi, pix % cam.w, pix / cam.w));
      }
      rho_prev = rho;
      if (acc.a >= early || j >= nlast) {
        fresh = true;                  // pair (or pixel) done
        if (acc.a >= early) q = np;
        continue;
      }
      h = ((j + 1 <= nsamp) ? (float)(j + 1) * ds : L) - (float)j * ds;
    }
    // ---- one Newton iteration on G(z) = z - h W(p + z)
    float e[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) e[r] = g_in[r] - phi[r];
    const float ed = e[0] * d[0] + e[1] * d[1] + e[2] * d[2];
    float Vv[3], W[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) Vv[r] = d[r] + cc * (e[r] - ed * d[r]);
    float detJ = 0.f;
    {
      float Jc[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) Jc[a][b] = J[a][b];
      detJ = solve3<float>(Jc, Vv, W);
    }
    const bool wide = MIXED && fabsf(detJ) < B.tau_det;
    if (wide) {
      solve3_any<double>(J, Vv, W);
      if (STATS) ++c_fp64;
    }
    float G[3], v[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      v[r] = h * W[r];                   // z - G(z)
      G[r] = z[r] - v[r];
    }
    if (it == 0) {
      v0[0] = v[0]; v0[1] = v[1]; v0[2] = v[2];   // the explicit Euler step, kept for a fallback
    }
    // M = H[v] + (I - h J_V) J,  (I - h J_V) = (1 + h c) I - h c d d^T
    const float hc = h * cc;
    float M[3][3], rhs[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float hv = H[a][b][0] * v[0] + H[a][b][1] * v[1] + H[a][b][2] * v[2];
        const float dj = d[0] * J[0][b] + d[1] * J[1][b] + d[2] * J[2][b];
        M[a][b] = hv + (1.f + hc) * J[a][b] - hc * d[a] * dj;
      }
      rhs[a] = -(J[a][0] * G[0] + J[a][1] * G[1] + J[a][2] * G[2]);
    }
    float dz[3];
    const float detM = wide ? solve3_any<double>(M, rhs, dz) : solve3<float>(M, rhs, dz);
#pragma unroll
    for (int r = 0; r < 3; ++r) z[r] += dz[r];
    ++it;
    const float mdz = fmaxf(fabsf(dz[0]), fmaxf(fabsf(dz[1]), fabsf(dz[2])));
    const bool singular = detJ == 0.f || detM == 0.f || !(mdz == mdz) || !(fabsf(v0[0]) + fabsf(v0[1]) + fabsf(v0[2]) < 1e30f);
    const bool conv = !singular && mdz <= kIrkTol;
    if (conv || singular || it >= kIrkMaxIter) {
      if (STATS && !conv) ++c_cap;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        float pn = p[r] + (conv ? z[r] : v0[r]);
        pn = pn == pn ? pn : p[r];
        p[r] = pn < 0.f ? 0.f : (pn > 1.f ? 1.f : pn);
        z[r] = 0.f;
      }
      it = 0;
      ++j;
      if (STATS) ++c_steps;
    }
  }
  if (MIXED) {
    unsigned long long vv = c_fp64;
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) vv += __shfl_down_sync(0xffffffffu, vv, o2);
    if (lane == 0 && vv) atomicAdd(&st->fp64_solves, vv);
  }
  if (STATS) {
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
      c_eval += __shfl_down_sync(0xffffffffu, c_eval, o2);
      c_steps += __shfl_down_sync(0xffffffffu, c_steps, o2);
      c_samp += __shfl_down_sync(0xffffffffu, c_samp, o2);
      c_cap += __shfl_down_sync(0xffffffffu, c_cap, o2);
      max_dp = fmaxf(max_dp, __shfl_down_sync(0xffffffffu, max_dp, o2));
    }
    if (lane == 0) {
      atomicAdd(&st->rhs_evals, c_eval);
      atomicAdd(&st->rk_steps, c_steps);
      atomicAdd(&st->samples, c_samp);
      atomicAdd(&st->step_cap, c_cap);
      atomic_max_nonneg_float(&st->max_delta_p_bits, max_dp);
    }
  }
}

template <int P>
void launch_irk1_p(const DevVolume& V, const DevCamera<float>& cam, const DevTF& tf, const IntegrateArgs& a,
                   bool mixed, bool stats, const float4* pin, const float4* pout, const int* pblk, const int* pcnt,
                   const int* active, const int* n_active, int* queue_head, float4* out, DevStats* st, int num_sms,
                   cudaStream_t s) {
  static int per_sm[4] = {-1, -1, -1, -1};
  const int v = (mixed ? 2 : 0) + (stats ? 1 : 0);
  if (per_sm[v] < 0) {
    int n = 1;
    if (v == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k5_irk1<P, false, false>, 128, 0);
    if (v == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k5_irk1<P, false, true>, 128, 0);
    if (v == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k5_irk1<P, true, false>, 128, 0);
    if (v == 3) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k5_irk1<P, true, true>, 128, 0);
    per_sm[v] = n < 1 ? 1 : n;
  }
  int grid = num_sms * per_sm[v];
  const int max_useful = (a.npix + 127) / 128;
  if (grid > max_useful) grid = max_useful > 0 ? max_useful : 1;
#define IVV_K5I(MM, SS) \
  launch_pdl(k5_irk1<P, MM, SS>, dim3(grid), dim3(128), s, V, cam, tf, a, pin, pout, pblk, pcnt, active, n_active, \
             queue_head, out, st)
  if (mixed) { if (stats) IVV_K5I(true, true); else IVV_K5I(true, false); }
  else { if (stats) IVV_K5I(false, true); else IVV_K5I(false, false); }
#undef IVV_K5I
}

}  // namespace ivv
