// Stage 3 with the paper's fixed-step explicit Runge-Kutta family (§5.2-5.3:
// Euler, midpoint, Kutta's third-order method, classic RK4, the 3/8 rule and
// Fehlberg's fifth-order weights): one step of the tableau per sample
// interval [s_{j-1}, s_j] of the pulled-back ODE p' = W(p) (§5.2), stage
// points and results clamped to [0,1]^3 (§5.4), compositing as in K5.
//
// K5f integrate_fixed -- persistent kernel over the same work queue as K5;
// each lane runs a small state machine with one right-hand side per loop
// iteration (so the lanes of a warp stay converged on the spline work):
//   stage 0   W and rho at the current sample point p(s_j); composite the
//             interval ending there; start the next step with K_0 = W;
//   stage k   K_k = W(p + h sum_{m<k} a_km K_m); after the last stage
//             p <- p + h sum_m b_m K_m and back to stage 0.
// The step is the sample distance (the last one partial), so samples need
// no dense output and every sample costs exactly s right-hand sides.
#pragma once

#include "k_integrate.cuh"

namespace ivv {

template <int P, typename R, bool MIXED, bool STATS>
__global__ void __launch_bounds__(128, 4) k5_fixed(DevVolume V, DevCamera<R> cam, DevTF tf, IntegrateArgs args,
                                                   RkTableau T, const typename Vec4T<R>::type* __restrict__ pair_in,
                                                   const typename Vec4T<R>::type* __restrict__ pair_out,
                                                   const int* __restrict__ pair_block,
                                                   const int* __restrict__ pair_count,
                                                   const int* __restrict__ active, const int* __restrict__ n_active,
                                                   int* __restrict__ queue_head, float4* __restrict__ out,
                                                   DevStats* __restrict__ st) {
  typedef typename Vec4T<R>::type V4;
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
  const R ds = R(args.ds), cc = R(args.c), early = R(args.early_alpha);
  const R tail_eps = R(1e-12) * R(V.diag);
  const int ns = T.s;
  unsigned long long c_rhs = 0, c_steps = 0, c_samp = 0, c_fp64 = 0;
  float max_dp = 0.f;

  int pix = -1;           // -1: needs a pixel; -2: queue drained
  int q = 0, np = 0, stage = 0, j = 0, nsamp = 0, nlast = 0;
  BlockInfo B = V.blocks[0];
  R o[3], d[3], g_in[3], p[3], K[kRkStagesMax][3];
  R h = 0, L = 0, rho_prev = 0;
  bool fresh = true;      // next stage-0 evaluation starts a pair
  Acc<R> acc;

  WarpQueue wq(nact, queue_head, nullptr);
  for (;;) {
    if (__ballot_sync(0xffffffffu, pix >= 0) == 0) {     // the whole warp is idle: refill
      if (wq.done()) break;
      const int item = wq.take(lane, queue_head);
      if (pix == -1) {
        if (item < nact) {
          pix = __ldg(active + item);
          const int xw = pix % cam.w, yw = pix / cam.w;
          make_ray<R>(cam, cam.x0 + xw, cam.y0 + yw, o, d);
          acc.C[0] = acc.C[1] = acc.C[2] = acc.a = R(0);
          np = __ldg(pair_count + pix);
          q = -1;
          fresh = true;
          stage = 0;
        } else {
          pix = -2;
        }
      }
      wq.drained |= __ballot_sync(0xffffffffu, pix == -2);
    }

    bool live = pix >= 0;
    if (live && fresh) {
      // the next pair with a positive length, or the end of the pixel
      bool found = false;
      while (!found && ++q < np) {
        const size_t slot = (size_t)q * npix + pix;
        const V4 pi = pair_in[slot];
        const V4 po = pair_out[slot];
        L = R(po.x) - R(pi.x);
        if (!(L > R(0))) continue;
        B = V.blocks[__ldg(pair_block + slot)];
#pragma unroll
        for (int r = 0; r < 3; ++r) g_in[r] = o[r] + R(pi.x) * d[r];
        p[0] = R(pi.y); p[1] = R(pi.z); p[2] = R(pi.w);
        const R fl = floor(L / ds);
        nsamp = (int)fl;
        nlast = nsamp + ((L - fl * ds > tail_eps) ? 1 : 0);
        j = 0;
        stage = 0;
        found = true;
      }
      if (!found) {
        out[pix] = make_float4((float)acc.C[0], (float)acc.C[1], (float)acc.C[2], (float)acc.a);
        pix = -1;
        live = false;
      }
    }
    if (!live) continue;                             // idle lanes issue no loads
    // ---- the evaluation point of this lane
    R x[3];
    if (stage > 0) {
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        R sum = R(0);
#pragma unroll
        for (int m = 0; m < kRkStagesMax - 1; ++m)
          if (m < stage) sum += R(T.a[stage][m]) * K[m][r];
        const R v = p[r] + h * sum;
        x[r] = v < R(0) ? R(0) : (v > R(1) ? R(1) : v);
      }
    } else {
      x[0] = p[0]; x[1] = p[1]; x[2] = p[2];
    }
    R W[3], rho, phi[3];
    rhs_eval<P, R, MIXED, true>(V, B, x, g_in, d, cc, V.mode, W, rho, phi, c_fp64);
    if (STATS) ++c_rhs;
#pragma unroll
    for (int m = 0; m < kRkStagesMax; ++m)
      if (m == stage) {
        K[m][0] = W[0]; K[m][1] = W[1]; K[m][2] = W[2];
      }
    if (stage == 0) {
      // rho at sample s_j: composite [s_{j-1}, s_j]
      if (fresh) {
        fresh = false;
      } else {
        const R s1 = (j <= nsamp) ? R(j) * ds : L;
        const R s0 = R(j - 1) * ds;
        composite_interval<R>(s_r, s_rgba, s_seg, tf, args.K, rho_prev, rho, s1 - s0, acc);
      }
      if (STATS) {
        ++c_samp;
        max_dp = fmaxf(max_dp, pixel_error<R>(cam, phi, pix % cam.w, pix / cam.w));
      }
      rho_prev = rho;
      if (acc.a >= early || j >= nlast) {
        fresh = true;                  // pair (or pixel) done
        if (acc.a >= early) q = np;
        continue;
      }
      const R s_next = (j + 1 <= nsamp) ? R(j + 1) * ds : L;
      h = s_next - R(j) * ds;
    }
    if (stage == ns - 1) {
      // the step is complete: p(s_{j+1})
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        R sum = R(0);
#pragma unroll
        for (int m = 0; m < kRkStagesMax; ++m)
          if (m < ns) sum += R(T.b[m]) * K[m][r];
        const R v = p[r] + h * sum;
        p[r] = v < R(0) ? R(0) : (v > R(1) ? R(1) : v);
      }
      ++j;
      stage = 0;
      if (STATS) ++c_steps;
    } else {
      ++stage;
    }
  }
  if (MIXED) {
    unsigned long long v = c_fp64;
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) v += __shfl_down_sync(0xffffffffu, v, o2);
    if (lane == 0 && v) atomicAdd(&st->fp64_solves, v);
  }
  if (STATS) {
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
      c_rhs += __shfl_down_sync(0xffffffffu, c_rhs, o2);
      c_steps += __shfl_down_sync(0xffffffffu, c_steps, o2);
      c_samp += __shfl_down_sync(0xffffffffu, c_samp, o2);
      max_dp = fmaxf(max_dp, __shfl_down_sync(0xffffffffu, max_dp, o2));
    }
    if (lane == 0) {
      atomicAdd(&st->rhs_evals, c_rhs);
      atomicAdd(&st->rk_steps, c_steps);
      atomicAdd(&st->samples, c_samp);
      atomic_max_nonneg_float(&st->max_delta_p_bits, max_dp);
    }
  }
}

template <int P>
void launch_fixed_p(const DevVolume& V, const DevCamera<float>& cam, const DevTF& tf, const IntegrateArgs& a,
                    const RkTableau& T, bool mixed, bool stats, const float4* pin, const float4* pout,
                    const int* pblk, const int* pcnt, const int* active, const int* n_active, int* queue_head,
                    float4* out, DevStats* st, int num_sms, cudaStream_t s) {
  static int per_sm[4] = {-1, -1, -1, -1};
  const int v = (mixed ? 2 : 0) + (stats ? 1 : 0);
  if (per_sm[v] < 0) {
    int n = 1;
    if (v == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k5_fixed<P, float, false, false>, 128, 0);
    if (v == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k5_fixed<P, float, false, true>, 128, 0);
    if (v == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k5_fixed<P, float, true, false>, 128, 0);
    if (v == 3) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k5_fixed<P, float, true, true>, 128, 0);
    per_sm[v] = n < 1 ? 1 : n;
  }
  int grid = num_sms * per_sm[v];
  const int max_useful = (a.npix + 127) / 128;
  if (grid > max_useful) grid = max_useful > 0 ? max_useful : 1;
#define IVV_K5F(MM, SS) \
  launch_pdl(k5_fixed<P, float, MM, SS>, dim3(grid), dim3(128), s, V, cam, tf, a, T, pin, pout, pblk, pcnt, \
             active, n_active, queue_head, out, st)
  if (mixed) { if (stats) IVV_K5F(true, true); else IVV_K5F(true, false); }
  else { if (stats) IVV_K5F(false, true); else IVV_K5F(false, false); }
#undef IVV_K5F
}

}  // namespace ivv
