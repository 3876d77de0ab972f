// Stage 3 (§5.2, §3.2.1): ray integration in parameter space.
//
// K5 integrate -- persistent kernel; each warp takes 32 pixels at a time from
// the work queue filled by K4.  For every entry/exit pair of a pixel, in front
// to back order, the pulled-back view ray
//     p'(s) = W(p),  J_phi(p) W(p) = V(phi(p)),                     (Eqs. 13-15)
//     V(g)  = d + c [(g_in - g) - <g_in - g, d> d]                  (Eqs. 10-11)
// is integrated from p(0) = p_in with the embedded Bogacki-Shampine 3(2) pair
// (FSAL: 3 new right-hand sides per step) under absolute error control in
// parameter space.  Steps are shortened to land exactly on the sample points
// s_j = j ds and on the exit s = L; p is clamped to [0,1]^3 (§5.4).  At each
// sample the scalar rho (control points, det J or Eq. 23) is taken from the
// right-hand side evaluated at the step end, and the interval [s_{j-1}, s_j]
// is composited with K midpoint sub-samples of the linearly interpolated
// scalar (supersampling) by Alg. 1 with T = exp(-sigma A ds_i / K).
// A pixel stops when its opacity reaches early_alpha.
#pragma once

#include <cuda_runtime.h>

#include "ivv_device.cuh"

namespace ivv {

template <typename R> struct Acc { R C[3]; R a; };

// W(p) = J_phi(p)^-1 V(phi(p)) and, when asked, rho(p) and phi(p).  UI and
// XYZ pick the contraction's form (outer-loop unroll; without the scalar
// channel) where that is the faster one.
template <int P, typename R, bool MIXED, bool WANT_RHO, int UI = 1, bool XYZ = false>
__device__ __forceinline__ void rhs_eval(const DevVolume& V, const BlockInfo& B, const R p[3], const R g_in[3],
                                         const R d[3], R c, int mode, R W[3], R& rho, R phi[3],
                                         unsigned long long& n_fp64) {
  R J[3][3], rc;
  if (WANT_RHO && mode == IVV_SCALAR_CP)
    eval_block<P, R, true, false, UI>(V, B, p, phi, J, rc);
  else
    eval_block<P, R, false, XYZ, UI>(V, B, p, phi, J, rc);
  R e[3] = {g_in[0] - phi[0], g_in[1] - phi[1], g_in[2] - phi[2]};
  const R ed = e[0] * d[0] + e[1] * d[1] + e[2] * d[2];
  R v[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) v[r] = d[r] + c * (e[r] - ed * d[r]);
  const R det = solve3<R>(J, v, W);
  if constexpr (MIXED) {
    if (fabs(det) < R(B.tau_det)) {
      double Jd[3][3], vd[3], Wd[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        vd[r] = v[r];
#pragma unroll
        for (int k = 0; k < 3; ++k) Jd[r][k] = J[r][k];
      }
      solve3<double>(Jd, vd, Wd);
#pragma unroll
      for (int r = 0; r < 3; ++r) W[r] = R(Wd[r]);
      ++n_fp64;
    }
  }
  if (WANT_RHO) {
    if (mode == IVV_SCALAR_CP) {
      rho = rc;
    } else if (mode == IVV_SCALAR_DETJ) {
      rho = det;
    } else {
      rho = scalar_at<P, R>(V, B, mode, p, J, rc);
    }
  }
}

// s + hh, snapped to L when the step reaches the end of the pair.
template <typename R> __device__ __forceinline__ R last_end(R s, R hh, R L) {
  const R e = s + hh;
  return e >= L ? L : e;
}

// Bogacki-Shampine 3(2) arithmetic shared by the fused integrator and the
// trace kernel (k_trace.cuh), written as explicit fused multiply-adds so both
// kernels round alike and take the same steps.
template <typename R> __device__ __forceinline__ R fmar(R a, R b, R c);   // a b + c
template <> __device__ __forceinline__ float fmar<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ double fmar<double>(double a, double b, double c) { return __fma_rn(a, b, c); }
// stage points q2 = p + hh/2 k1, q3 = p + 3hh/4 k2
template <typename R> __device__ __forceinline__ R bs3_q2(R p, R hh, R k1) { return fmar(R(0.5) * hh, k1, p); }
template <typename R> __device__ __forceinline__ R bs3_q3(R p, R hh, R k2) { return fmar(R(0.75) * hh, k2, p); }
// third-order solution p + hh (2/9 k1 + 1/3 k2 + 4/9 k3)
template <typename R> __device__ __forceinline__ R bs3_pn(R p, R hh, R k1, R k2, R k3) {
  return fmar(hh, fmar(R(4.0 / 9.0), k3, fmar(R(1.0 / 3.0), k2, R(2.0 / 9.0) * k1)), p);
}
// error combination without the k4 term, and the local error with it
template <typename R> __device__ __forceinline__ R bs3_e3(R k1, R k2, R k3) {
  return fmar(R(1.0 / 9.0), k3, fmar(R(1.0 / 12.0), k2, R(-5.0 / 72.0) * k1));
}
template <typename R> __device__ __forceinline__ R bs3_err(R hh, R e3, R k4) { return hh * fmar(R(-1.0 / 8.0), k4, e3); }
// cubic Hermite dense output at th in [0, 1] of a step of length hh from
// (p0, k0) to (p1, k1)
template <typename R> __device__ __forceinline__ R hermite(R th, R hh, R p0, R k0, R p1, R k1) {
  const R t2 = th * th, t3 = t2 * th;
  const R h00 = fmar(R(2), t3, fmar(R(-3), t2, R(1))), h10 = fmar(R(-2), t2, t3 + th);
  const R h01 = fmar(R(-2), t3, R(3) * t2), h11 = t3 - t2;
  return fmar(h11 * hh, k1, fmar(h01, p1, fmar(h10 * hh, k0, h00 * p0)));
}

template <typename R> __device__ __forceinline__ R pow_third(R x);
template <> __device__ __forceinline__ float pow_third<float>(float x) { return exp2f(__log2f(x) * (1.f / 3.f)); }
template <> __device__ __forceinline__ double pow_third<double>(double x) { return cbrt(x); }

template <typename R> __device__ __forceinline__ R fast_exp(R x);
template <> __device__ __forceinline__ float fast_exp<float>(float x) { return __expf(x); }
template <> __device__ __forceinline__ double fast_exp<double>(double x) { return exp(x); }

// Alg. 1 over the interval [s_{j-1}, s_j] of length dsi with K midpoint
// sub-samples of the linearly interpolated scalar (§3.2.1 supersampling).
// The TF is piecewise linear in the normalised scalar and constant outside
// [r_0, r_{n-1}]; when both interval ends fall into the same piece, the K
// sub-sample colours are the same linear interpolation of the two end
// colours, so two TF lookups serve all K sub-samples.
// KC > 0: K is the compile-time constant KC (loop unrolled, the piece test
// hoisted); KC = 0: K at run time.  Both round identically.
template <typename R, int KC>
__device__ __forceinline__ void composite_interval_k(const float* s_r, const float4* s_rgba,
                                                     const unsigned char* s_seg, const DevTF& tf, int K, R rho0,
                                                     R rho1, R dsi, Acc<R>& acc) {
  const int nk = KC > 0 ? KC : K;
  const R invK = KC > 0 ? R(1.0 / KC) : R(1) / R(K);
  const R dr = rho1 - rho0;
  const R tau_scale = R(tf.sigma) * dsi * invK;
  const R x0 = (rho0 - R(tf.lo)) * R(tf.inv_range), x1 = (rho1 - R(tf.lo)) * R(tf.inv_range);
  int g0, g1;
  const float4 c0 = tf_eval_seg(s_r, s_rgba, s_seg, tf.n, (float)x0, g0);
  const float4 c1 = tf_eval_seg(s_r, s_rgba, s_seg, tf.n, (float)x1, g1);
  if (g0 == g1) {
    const float4 dc = make_float4(c1.x - c0.x, c1.y - c0.y, c1.z - c0.z, c1.w - c0.w);
#pragma unroll
    for (int k = 0; k < nk; ++k) {
      const float f = (float)((R(k) + R(0.5)) * invK);
      const float4 c = make_float4(c0.x + f * dc.x, c0.y + f * dc.y, c0.z + f * dc.z, c0.w + f * dc.w);
      const R T = fast_exp<R>(-tau_scale * R(c.w));
      const R w = (R(1) - T) * (R(1) - acc.a);
      acc.C[0] += w * R(c.x);
      acc.C[1] += w * R(c.y);
      acc.C[2] += w * R(c.z);
      acc.a += w;
    }
  } else {
#pragma unroll 1
    for (int k = 0; k < nk; ++k) {
      const R fk = (R(k) + R(0.5)) * invK;
      const R rk = rho0 + fk * dr;
      R x = (rk - R(tf.lo)) * R(tf.inv_range);
      x = x < R(0) ? R(0) : (x > R(1) ? R(1) : x);
      const float4 c = tf_eval(s_r, s_rgba, s_seg, tf.n, (float)x);
      const R T = fast_exp<R>(-tau_scale * R(c.w));
      const R w = (R(1) - T) * (R(1) - acc.a);
      acc.C[0] += w * R(c.x);
      acc.C[1] += w * R(c.y);
      acc.C[2] += w * R(c.z);
      acc.a += w;
    }
  }
}

template <typename R>
__device__ __forceinline__ void composite_interval(const float* s_r, const float4* s_rgba, const unsigned char* s_seg,
                                                   const DevTF& tf, int K, R rho0, R rho1, R dsi, Acc<R>& acc) {
  if (K == 4)
    composite_interval_k<R, 4>(s_r, s_rgba, s_seg, tf, K, rho0, rho1, dsi, acc);
  else
    composite_interval_k<R, 0>(s_r, s_rgba, s_seg, tf, K, rho0, rho1, dsi, acc);
}

// Pixel-accuracy error Delta P (Eq. 5) of the world point phi for pixel
// (xw, yw) of the window of cam: twice the larger screen offset, in pixels.
template <typename R, typename RC>
__device__ __forceinline__ float pixel_error(const DevCamera<RC>& cam, const R phi[3], int xw, int yw) {
  RC sx, sy, ph[3] = {RC(phi[0]), RC(phi[1]), RC(phi[2])};
  project<RC>(cam, ph, sx, sy);
  return 2.f * (float)fmax(fabs(sx - RC(cam.x0 + xw)), fabs(sy - RC(cam.y0 + yw)));
}

// One lane's position in the integration of its current pixel.
//   stage 0: start of a pair (evaluate W and rho at p_in);
//   stages 1..3: the three new right-hand sides of a Bogacki-Shampine step
//   (at q2, q3 and the step end); after an accepted step the samples s_j that
//   fall inside it are visited in order:
//   stage 4: rho at the dense-output point p(s_j) (cubic Hermite through the
//   step's end points and slopes, third order like the pair itself).
//
// BATCH: the queue holds pixels of every request of a batch (BatchArgs); a
// lane looks up its pixel's request when it takes the pixel and from then on
// uses that request's camera, sample distance, transfer function slot and
// image; the block table of the batch's pool carries each block's scalar mode.
//
// The split form of stage 3 (sample points first, shading after) is the
// trace kernel of k_trace.cuh.
template <int P, typename R, bool MIXED, bool STATS, bool BATCH = false>
__global__ void __launch_bounds__(128, 4) k5_integrate(DevVolume V, DevCamera<R> cam, DevTF tf, IntegrateArgs args,
                                                       BatchArgs ba,
                                                       const typename Vec4T<R>::type* __restrict__ pair_in,
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
  if constexpr (!BATCH) {
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
  }
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int nact = *n_active;
  if (nact == 0) return;
  const int npix = args.npix;
  const R tol = R(args.rk_tol), cc = R(args.c), early = R(args.early_alpha);
  R ds = R(args.ds);
  R tail_eps = R(1e-12) * R(V.diag);
  R hmin = R(1e-7) * ds;
  R hmax = R(args.max_step_samples) * ds;
  int rq = 0;             // BATCH: request of the lane's pixel
  unsigned long long c_rhs = 0, c_steps = 0, c_rej = 0, c_samp = 0, c_fp64 = 0, c_cap = 0;
  float max_dp = 0.f;

  // lane state
  int pix = -1;           // -1: needs a pixel; -2: queue drained
  int q = 0, np = 0, stage = 0, j = 0, nsamp = 0, nlast = 0, steps = 0;
  BlockInfo B = V.blocks[0];
  R o[3], d[3], g_in[3], p[3], k1[3], k2[3], k3[3], pn[3], p0[3], k0[3];
  R s = 0, s_last = 0, h = 0, hh = 0, L = 0, rho_prev = 0, rho_end = 0, s0 = 0;
  Acc<R> acc;

  WarpQueue wq(nact, queue_head, nullptr);
  for (;;) {
    if (__ballot_sync(0xffffffffu, pix >= 0) == 0) {     // the whole warp is idle: refill
      if (wq.done()) break;
      const int item = wq.take(lane, queue_head);
      if (pix == -1) {
        if (item < nact) {
          pix = __ldg(active + item);
          if constexpr (BATCH) {
            rq = batch_request(ba, pix);
            const DevRequest& rr = ba.req[rq];
            const int loc = pix - __ldg(ba.pix0 + rq);
            const int xw = loc % rr.cam.w, yw = loc / rr.cam.w;
            make_ray<R>(rr.cam, rr.cam.x0 + xw, rr.cam.y0 + yw, o, d);
            ds = R(rr.ds);
            tail_eps = R(1e-12) * R(rr.diag);
            hmin = R(1e-7) * ds;
            hmax = R(args.max_step_samples) * ds;
          } else {
            const int xw = pix % cam.w, yw = pix / cam.w;
            make_ray<R>(cam, cam.x0 + xw, cam.y0 + yw, o, d);
          }
          acc.C[0] = acc.C[1] = acc.C[2] = acc.a = R(0);
          np = __ldg(pair_count + pix);
          q = -1;
          stage = 0;
        } else {
          pix = -2;                    // the queue is drained
        }
      }
      wq.drained |= __ballot_sync(0xffffffffu, pix == -2);
    }

    // ---- choose this lane's evaluation point
    bool live = pix >= 0;
    if (live && stage == 0) {
      // advance to the next pair with a positive length, or finish the pixel
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
        s = s_last = R(0);
        h = ds;
        j = 1;
        steps = 0;
        found = true;
      }
      if (!found) {
        const float4 res = make_float4((float)acc.C[0], (float)acc.C[1], (float)acc.C[2], (float)acc.a);
        if constexpr (BATCH)
          ba.req[rq].out[pix - __ldg(ba.pix0 + rq)] = res;
        else
          out[pix] = res;
        pix = -1;
        live = false;
      }
    }
    if (!live) continue;                             // idle lanes issue no loads
    R x[3];
    {
      if (stage == 0) {
        x[0] = p[0]; x[1] = p[1]; x[2] = p[2];
      } else if (stage == 1) {
#pragma unroll
        for (int r = 0; r < 3; ++r) x[r] = bs3_q2<R>(p[r], hh, k1[r]);
      } else if (stage == 2) {
#pragma unroll
        for (int r = 0; r < 3; ++r) x[r] = bs3_q3<R>(p[r], hh, k2[r]);
      } else if (stage == 3) {
#pragma unroll
        for (int r = 0; r < 3; ++r) x[r] = pn[r];
      } else {
        // cubic Hermite dense output on the accepted step [s0, s] (length hh)
        const R th = ((j <= nsamp ? R(j) * ds : L) - s0) / hh;
#pragma unroll
        for (int r = 0; r < 3; ++r) x[r] = hermite<R>(th, hh, p0[r], k0[r], p[r], k1[r]);
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) x[r] = x[r] < R(0) ? R(0) : (x[r] > R(1) ? R(1) : x[r]);
    }
    // ---- the one right-hand side of this iteration
    R W[3], rho, phi[3];
    rhs_eval<P, R, MIXED, true>(V, B, x, g_in, d, cc, BATCH ? B.mode : V.mode, W, rho, phi, c_fp64);
    if (STATS) ++c_rhs;
    // ---- advance the lane's state
    bool sample = false;        // rho / phi belong to sample s_j
    if (stage == 0) {
      k1[0] = W[0]; k1[1] = W[1]; k1[2] = W[2];
      rho_prev = rho;
      if (STATS) ++c_samp;
    } else if (stage == 1) {
      k2[0] = W[0]; k2[1] = W[1]; k2[2] = W[2];
    } else if (stage == 2) {
      k3[0] = W[0]; k3[1] = W[1]; k3[2] = W[2];
#pragma unroll
      for (int r = 0; r < 3; ++r)
        pn[r] = bs3_pn<R>(p[r], hh, k1[r], k2[r], k3[r]);
    } else if (stage == 3) {
      R err = R(0);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const R e = bs3_err<R>(hh, bs3_e3<R>(k1[r], k2[r], k3[r]), W[r]);
        const R ae = fabs(e);
        err = ae > err ? ae : err;
      }
      ++steps;
      const bool capped = steps >= args.max_steps;
      if (err <= tol || hh <= hmin || capped) {
        if (STATS) ++c_steps;
        if (capped) ++c_cap;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          p0[r] = p[r];
          k0[r] = k1[r];
          p[r] = x[r];
          k1[r] = W[r];
        }
        s0 = s;
        s = last_end(s, hh, L);
        rho_end = rho;
        R fac = err > R(0) ? R(0.9) * pow_third<R>(tol / err) : R(5);
        fac = fac < R(0.2) ? R(0.2) : (fac > R(5) ? R(5) : fac);
        h = hh * fac;
        if (capped) {
          stage = 0;
          continue;
        }
        stage = 4;           // visit the samples inside (s0, s]
      } else {
        if (STATS) ++c_rej;
        const R fac = R(0.9) * pow_third<R>(tol / err);
        h = hh * (fac < R(0.2) ? R(0.2) : fac);
      }
    } else {
      sample = true;         // stage 4: rho at an interior sample point
    }
    // ---- samples inside the accepted step: composite those that lie at or
    //      before the step end (the end itself reuses the step-end rho)
    if (stage == 4) {
      for (;;) {
        if (j > nlast) break;
        const R s_t = (j <= nsamp) ? R(j) * ds : L;
        R rj;
        if (sample) {
          rj = rho;
          sample = false;
        } else if (s_t >= s) {
          if (s_t > s) break;          // beyond this step
          rj = rho_end;                // the step ends on this sample
          phi[0] = phi[0];
        } else {
          break;                       // needs a dense-output evaluation
        }
        if constexpr (BATCH) {
          const DevTFSlot& ts = ba.tf[rq];
          DevTF t2;
          t2.n = ts.n;
          t2.sigma = ts.sigma;
          t2.lo = ts.lo;
          t2.inv_range = ts.inv_range;
          composite_interval<R>(ts.r, ts.rgba, ts.seg, t2, args.K, rho_prev, rj, s_t - s_last, acc);
        } else {
          composite_interval<R>(s_r, s_rgba, s_seg, tf, args.K, rho_prev, rj, s_t - s_last, acc);
        }
        if (STATS) {
          ++c_samp;
          float dp;
          if constexpr (BATCH) {
            const DevCamera<float>& cm = ba.req[rq].cam;
            const int loc = pix - __ldg(ba.pix0 + rq);
            dp = pixel_error<R>(cm, phi, loc % cm.w, loc / cm.w);
          } else {
            dp = pixel_error<R>(cam, phi, pix % cam.w, pix / cam.w);
          }
          max_dp = fmaxf(max_dp, dp);
        }
        rho_prev = rj;
        s_last = s_t;
        ++j;
        if (acc.a >= early) {
          q = np;                      // early termination ends the pixel
          j = nlast + 1;
        }
      }
      if (j > nlast) {
        stage = 0;                     // pair done
        continue;
      }
      const R s_t = (j <= nsamp) ? R(j) * ds : L;
      if (s_t < s) continue;           // stage 4 again: next interior sample
      // ---- next step
      const R rem = L - s;
      hh = h < hmax ? h : hmax;
      hh = hh < rem ? hh : rem;
      stage = 1;
      continue;
    }
    if (stage == 0) {
      if (j > nlast) {                 // zero-length remainder: pair done
        continue;
      }
      const R rem = L - s;
      hh = h < hmax ? h : hmax;
      hh = hh < rem ? hh : rem;
      stage = 1;
    } else if (stage == 1 || stage == 2) {
      ++stage;
    } else {
      // rejected step (stage 3): retry with the smaller h
      const R rem = L - s;
      hh = h < hmax ? h : hmax;
      hh = hh < rem ? hh : rem;
      stage = 1;
    }
  }
  // counters
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
      c_rej += __shfl_down_sync(0xffffffffu, c_rej, o2);
      c_samp += __shfl_down_sync(0xffffffffu, c_samp, o2);
      c_cap += __shfl_down_sync(0xffffffffu, c_cap, o2);
      max_dp = fmaxf(max_dp, __shfl_down_sync(0xffffffffu, max_dp, o2));
    }
    if (lane == 0) {
      atomicAdd(&st->rhs_evals, c_rhs);
      atomicAdd(&st->rk_steps, c_steps);
      atomicAdd(&st->rk_rejects, c_rej);
      atomicAdd(&st->samples, c_samp);
      atomicAdd(&st->step_cap, c_cap);
      atomic_max_nonneg_float(&st->max_delta_p_bits, max_dp);
    }
  } else if (c_cap) {
    atomicAdd(&st->step_cap, c_cap);               // a cap counter: kept by every render
  }
}

template <int P, typename R, bool MIXED, bool STATS>
void launch_k5(const DevVolume& V, const DevCamera<R>& cam, const DevTF& tf, const IntegrateArgs& a,
               const typename Vec4T<R>::type* pin, const typename Vec4T<R>::type* pout, const int* pblk,
               const int* pcnt, const int* active, const int* n_active, int* queue_head, float4* out, DevStats* st,
               int num_sms, cudaStream_t s) {
  static int blocks_per_sm = -1;
  if (blocks_per_sm < 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k5_integrate<P, R, MIXED, STATS>, 128, 0);
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  int grid = num_sms * blocks_per_sm;
  const int max_useful = (a.npix + 127) / 128;
  if (grid > max_useful) grid = max_useful > 0 ? max_useful : 1;
  BatchArgs none{};
  launch_pdl(k5_integrate<P, R, MIXED, STATS>, dim3(grid), dim3(128), s, V, cam, tf, a, none, pin, pout, pblk, pcnt,
             active, n_active, queue_head, out, st);
}

// ---- split integration: sample shading
// Eight consecutive floats with one 256-bit read-only load (32-byte aligned).
__device__ __forceinline__ void ldg_f8(const float* p, float v[8]) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
      : "l"(p));
}

// The scalar field alone at parameter point p of block B (control-point
// scalars): one contraction of the (P+1)^3 scalar coefficients, read from the
// scalar-only array with 256-bit loads (8 per cubic element, 4 per quadratic
// element), summed in the order of the integrator's fused contraction.
template <int P>
__device__ __forceinline__ float eval_rho_cp(const DevVolume& V, const BlockInfo& B, const float p[3]) {
  constexpr int N = P + 1;
  constexpr int NNN = N * N * N;
  float loc[3];
  int e[3];
#pragma unroll
  for (int dd = 0; dd < 3; ++dd) {
    float x = p[dd];
    x = x < 0.f ? 0.f : (x > 1.f ? 1.f : x);
    if ((B.uniform >> dd) & 1) {
      const float xs = x * (float)B.nseg[dd];
      int k = (int)xs;
      k = k < B.nseg[dd] - 1 ? k : B.nseg[dd] - 1;
      e[dd] = k;
      loc[dd] = xs - (float)k;
    } else {
      float sc;
      e[dd] = locate<float>(V.brk32 + B.brk_off[dd], B.nseg[dd], x, loc[dd], sc);
    }
  }
  const float* cp = V.rho32 + (size_t)(B.elem_off + (e[2] * B.nseg[1] + e[1]) * B.nseg[0] + e[0]) * rho_stride32(P);
  float bu[N], bv[N], bw[N];
  bernstein_v<P, float>(loc[0], bu);
  bernstein_v<P, float>(loc[1], bv);
  bernstein_v<P, float>(loc[2], bw);
  static_assert(NNN <= rho_stride32(P), "padded scalar element");
  float s = 0.f;
  if constexpr (P == 3) {
    // one i-slab (16 scalars, two loads) at a time
#pragma unroll 1
    for (int i = 0; i < N; ++i) {
      float c[16];
      ldg_f8(cp + 16 * i, c);
      ldg_f8(cp + 16 * i + 8, c + 8);
      float si = 0.f;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        float sj = 0.f;
#pragma unroll
        for (int k = 0; k < N; ++k) sj += bw[k] * c[j * N + k];
        si += bv[j] * sj;
      }
      s += pick<N>(bu, i) * si;
    }
  } else {
    float c[rho_stride32(P)];
#pragma unroll
    for (int q = 0; q < rho_stride32(P) / 8; ++q) ldg_f8(cp + 8 * q, c + 8 * q);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      float si = 0.f;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        float sj = 0.f;
#pragma unroll
        for (int k = 0; k < N; ++k) sj += bw[k] * c[(i * N + j) * N + k];
        si += bv[j] * sj;
      }
      s += bu[i] * si;
    }
  }
  return s;
}

// det J with the cofactor expansion of solve3 (same rounding as the fused
// integrator's scalar).
__device__ __forceinline__ float det_cofactor(const float J[3][3]) {
  const float c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  const float c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  const float c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  return J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
}

// Shading and compositing of the split integration: every active pixel's
// sample list is walked front to back (pairs in order, s_j = j ds with the
// last interval partial); the scalar is evaluated at each sample point
// (control points, det J or Eq. 23) and every interval is composited with K
// sub-samples (Alg. 1), stopping at early_alpha.  One sample per lane and
// loop iteration over the flattened (pair, sample) sequence, so lanes whose
// pixels cross pair boundaries at different samples stay converged; lanes
// whose pixel is finished sit out (no loads) until the whole warp is idle,
// and the warp then takes 32 consecutive queue items at once, from a chunk
// of 128 shared by the block's warps while the queue is long: the pixels of
// a block are neighbours that start together, so their control-point loads
// hit the same elements in L1.  With statistics also Delta P (Eq. 5) per
// sample.
// CP: the volume's scalar is its control-point field (a separate instance, so
// the det J / Eq. 23 instance keeps its own register allocation).
// BATCH: pixels of every request of a batch; each takes its request's camera,
// sample distance, transfer-function slot and output image, and each block's
// scalar mode (CP unused); a pixel whose sample list does not fit the list
// (off + cnt > cap) is left to the fused integrator.
// VM: the von Mises scalar of §6.2 (its own instance: the displacement's
// contraction stays out of the other instances' register allocation).
template <int P, bool STATS, bool CP, bool BATCH = false, bool VM = false>
__global__ void __launch_bounds__(128, 4) k_shade_composite(DevVolume V, DevCamera<float> cam, DevTF tf, int K,
                                                         float early, BatchArgs ba, const int* __restrict__ cnt,
                                                         const float4* __restrict__ pair_in,
                                                         const float4* __restrict__ pair_out,
                                                         const int* __restrict__ pair_block,
                                                         const int* __restrict__ pair_count,
                                                         const int* __restrict__ active,
                                                         const int* __restrict__ n_active, int* __restrict__ queue_head,
                                                         const int* __restrict__ off, int npix, float ds,
                                                         float tail_eps, int cap, const float4* __restrict__ sp,
                                                         float4* __restrict__ out, DevStats* __restrict__ st) {
  __shared__ float s_r[BATCH ? 1 : 256];
  __shared__ float4 s_rgba[BATCH ? 1 : 256];
  __shared__ unsigned char s_seg[BATCH ? 1 : kTfTable];
  if constexpr (!BATCH) {
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
  }
  pdl_wait();                                       // (the TF above is the volume's, not a predecessor's)
  const int lane = threadIdx.x & 31;
  const int nact = *n_active;
  if (nact == 0) return;
  __shared__ unsigned long long s_chunk;
  WarpQueue wq(nact, queue_head, &s_chunk);
  const bool excess = BATCH && n_active[3] > 0;     // the sample offsets overflowed
  unsigned long long c_samp = 0, c_rho = 0;
  float max_dp = 0.f;

  // lane state: the pixel (-1: needs one, -2: queue drained), its pair q of
  // np, the sample j of the pair (nlast: its last), k: the sample's index in
  // the list
  int pix = -1, q = 0, np = 0, j = 1, nsamp = 0, nlast = 0, k = 0;
  float L = 0.f, rho_prev = 0.f, s_prev = 0.f;
  Acc<float> acc;
  acc.C[0] = acc.C[1] = acc.C[2] = acc.a = 0.f;
  BlockInfo B = V.blocks[0];
  const float* tr = s_r;
  const float4* trgba = s_rgba;
  const unsigned char* tseg = s_seg;
  DevTF t2 = tf;
  DevCamera<float> cm = cam;
  int loc = 0;            // the pixel's index in its image (and in dst)
  float4* dst = out;

  for (;;) {
    if (__ballot_sync(0xffffffffu, pix >= 0) == 0) {     // the whole warp is idle: refill
      if (wq.done()) break;
      const int item = wq.take(lane, queue_head);
      if (pix == -1) {
        if (item < nact) {
          pix = __ldg(active + item);
          k = __ldg(off + item);
          np = __ldg(pair_count + pix);
          q = -1;
          j = 1;
          nlast = 0;                                // no pair yet: take the first
          acc.C[0] = acc.C[1] = acc.C[2] = acc.a = 0.f;
          loc = pix;
          if constexpr (BATCH) {
            if (excess || k < 0 || k + __ldg(cnt + item) > cap) {
              pix = -1;                             // rendered by the fused integrator
            } else {
              const int rq = batch_request(ba, pix);
              const DevRequest& rr = ba.req[rq];
              const DevTFSlot& ts = ba.tf[rq];
              tr = ts.r;
              trgba = ts.rgba;
              tseg = ts.seg;
              t2.n = ts.n;
              t2.sigma = ts.sigma;
              t2.lo = ts.lo;
              t2.inv_range = ts.inv_range;
              ds = rr.ds;
              tail_eps = 1e-12f * rr.diag;
              loc = pix - __ldg(ba.pix0 + rq);
              dst = rr.out;
              if (STATS) cm = rr.cam;
            }
          }
        } else {
          pix = -2;
        }
      }
      wq.drained |= __ballot_sync(0xffffffffu, pix == -2);
    }

    bool live = pix >= 0;
    if (live && j > nlast) {
      // the next pair with a positive length, or the end of the pixel
      bool found = false;
      while (!found && ++q < np) {
        const size_t slot = (size_t)q * npix + pix;
        const float4 pi = pair_in[slot], po = pair_out[slot];
        L = po.x - pi.x;
        if (!(L > 0.f)) continue;
        B = V.blocks[__ldg(pair_block + slot)];
        const float fl = floorf(L / ds);
        nsamp = (int)fl;
        nlast = nsamp + ((L - fl * ds > tail_eps) ? 1 : 0);
        j = 0;
        rho_prev = 0.f;
        s_prev = 0.f;
        found = true;
      }
      if (!found) live = false;
    }
    if (live && k >= cap) live = false;              // beyond the sample list: the pixel ends here
    if (pix >= 0 && !live) {
      dst[loc] = make_float4(acc.C[0], acc.C[1], acc.C[2], acc.a);
      pix = -1;
    }
    if (!live) continue;                             // idle lanes issue no loads
    // ---- the scalar at this lane's sample
    float p[3];
    {
      const float4 r = sp[k];
      p[0] = r.x; p[1] = r.y; p[2] = r.z;
    }
    float rho;
    const int mode = BATCH ? B.mode : V.mode;
    // single frames: the launch picks the instance of the volume's mode, so
    // CP decides at compile time; batches carry each block's mode
    const bool cp_mode = BATCH ? mode == IVV_SCALAR_CP : CP;
    if (!STATS && !BATCH && CP) {
      rho = eval_rho_cp<P>(V, B, p);
    } else {
      float phi[3], J[3][3], rc;
      // single frames: the contraction fully unrolled (the Eq. 23 bar +1.7 %);
      // the batch instance, which carries every mode, and the von Mises one
      // keep the loop
      if (cp_mode)
        eval_block<P, float, true>(V, B, p, phi, J, rc);
      else
        eval_block<P, float, false, true, (BATCH || VM) ? 1 : P + 1>(V, B, p, phi, J, rc);
      if constexpr (VM) {
        rho = scalar_at<P, float>(V, B, IVV_SCALAR_VONMISES, p, J, rc);
      } else if (cp_mode) {
        rho = rc;
      } else {
        const float det = det_cofactor(J);
        if (mode == IVV_SCALAR_DETJ) {
          rho = det;
        } else {
          float f = 0.f;
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) f += J[a][b] * J[a][b];
          rho = det / sqrtf(f);
        }
      }
      if (STATS) max_dp = fmaxf(max_dp, pixel_error<float>(cm, phi, loc % cm.w, loc / cm.w));
    }
    const float s = j <= nsamp ? (float)j * ds : L;
    if (STATS) {
      ++c_samp;
      ++c_rho;
    }
    if (j > 0) {
      composite_interval<float>(tr, trgba, tseg, t2, K, rho_prev, rho, s - s_prev, acc);
      if (acc.a >= early) {
        dst[loc] = make_float4(acc.C[0], acc.C[1], acc.C[2], acc.a);
        pix = -1;
        continue;
      }
    }
    rho_prev = rho;
    s_prev = s;
    ++j;
    ++k;
  }
  if (STATS) {
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
      c_samp += __shfl_down_sync(0xffffffffu, c_samp, o2);
      c_rho += __shfl_down_sync(0xffffffffu, c_rho, o2);
      max_dp = fmaxf(max_dp, __shfl_down_sync(0xffffffffu, max_dp, o2));
    }
    if (lane == 0) {
      atomicAdd(&st->samples, c_samp);
      atomicAdd(&st->rho_evals, c_rho);
      atomic_max_nonneg_float(&st->max_delta_p_bits, max_dp);
    }
  }
}

template <int P>
void launch_shade_composite_p(const DevVolume& V, const DevCamera<float>& cam, const DevTF& tf, int K, float early,
                              const float4* pin, const float4* pout, const int* pblk, const int* pcnt,
                              const int* active, const int* n_active, int* queue_head, const int* off, int npix,
                              float ds, float tail_eps, const SplitArgs& sa, float4* out, bool stats, DevStats* st,
                              int num_sms, cudaStream_t s) {
  static int per_sm[6] = {-1, -1, -1, -1, -1, -1};
  const bool cp = V.mode == IVV_SCALAR_CP;
  const bool vm = V.mode == IVV_SCALAR_VONMISES;
  const int v = vm ? 4 + (stats ? 1 : 0) : (stats ? 2 : 0) + (cp ? 1 : 0);
  if (per_sm[v] < 0) {
    int n = 1;
    if (v == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_shade_composite<P, false, false>, 128, 0);
    if (v == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_shade_composite<P, false, true>, 128, 0);
    if (v == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_shade_composite<P, true, false>, 128, 0);
    if (v == 3) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_shade_composite<P, true, true>, 128, 0);
    if (v == 4)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_shade_composite<P, false, false, false, true>, 128, 0);
    if (v == 5)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_shade_composite<P, true, false, false, true>, 128, 0);
    per_sm[v] = n < 1 ? 1 : n;
  }
  int grid = num_sms * per_sm[v];                   // persistent: the lanes refill from the queue
  const int useful = (npix + 127) / 128;
  grid = grid < useful ? grid : (useful > 0 ? useful : 1);
#define IVV_SHADE(SS, CC, VV)                                                                               \
  launch_pdl(k_shade_composite<P, SS, CC, false, VV>, dim3(grid), dim3(128), s, V, cam, tf, K, early, BatchArgs{},   \
             (const int*)nullptr, pin, pout, pblk, pcnt, active, n_active, queue_head, off, npix, ds, tail_eps, sa.cap, \
             sa.sp, out, st)
  if (vm) { if (stats) IVV_SHADE(true, false, true); else IVV_SHADE(false, false, true); }
  else if (stats) { if (cp) IVV_SHADE(true, true, false); else IVV_SHADE(true, false, false); }
  else { if (cp) IVV_SHADE(false, true, false); else IVV_SHADE(false, false, false); }
#undef IVV_SHADE
}

template <int P>
void launch_integrate_p(const DevVolume& V, const DevCamera<float>* cam32, const DevCamera<double>* cam64,
                        const DevTF& tf, const IntegrateArgs& a, bool mixed, bool stats, const void* pin,
                        const void* pout, const int* pblk, const int* pcnt, const int* active, const int* n_active,
                        int* queue_head, float4* out, DevStats* st, int num_sms, cudaStream_t s) {
  if (cam32) {
    const float4* i4 = (const float4*)pin;
    const float4* o4 = (const float4*)pout;
    if (mixed) {
      if (stats) launch_k5<P, float, true, true>(V, *cam32, tf, a, i4, o4, pblk, pcnt, active, n_active, queue_head, out, st, num_sms, s);
      else launch_k5<P, float, true, false>(V, *cam32, tf, a, i4, o4, pblk, pcnt, active, n_active, queue_head, out, st, num_sms, s);
    } else {
      if (stats) launch_k5<P, float, false, true>(V, *cam32, tf, a, i4, o4, pblk, pcnt, active, n_active, queue_head, out, st, num_sms, s);
      else launch_k5<P, float, false, false>(V, *cam32, tf, a, i4, o4, pblk, pcnt, active, n_active, queue_head, out, st, num_sms, s);
    }
  } else {
    const Dbl4* i4 = (const Dbl4*)pin;
    const Dbl4* o4 = (const Dbl4*)pout;
    if (stats) launch_k5<P, double, false, true>(V, *cam64, tf, a, i4, o4, pblk, pcnt, active, n_active, queue_head, out, st, num_sms, s);
    else launch_k5<P, double, false, false>(V, *cam64, tf, a, i4, o4, pblk, pcnt, active, n_active, queue_head, out, st, num_sms, s);
  }
}

}  // namespace ivv
