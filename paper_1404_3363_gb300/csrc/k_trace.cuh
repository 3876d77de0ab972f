// Stage 3, first pass of the split integration (FP32 / MIXED, one frame):
// K5t trace -- the Bogacki-Shampine 3(2) integration of the pulled-back view
// ray (Eqs. 10-15, §5.2) with the same error control, step rule, domain clamp
// (§5.4) and cubic Hermite dense output as the fused integrator, but the lane
// only records the parameter point of every sample s_j = j ds (and of the
// exit s = L) in its pixel's slice of the sample list.  The scalar, the
// transfer function and the compositing of Alg. 1 run afterwards in the
// shading pass, so this kernel carries no colour state and no transfer
// function, and evaluates W(p) only: J_phi and phi, not rho.
//
// Lane state between right-hand sides: the ray (d, g_in), the step start p
// with its slope k1 (FSAL), and one stage buffer that holds k2 after the
// first stage and then (pn, e) -- the third-order solution and the partial
// error combination -- after the second, so k2 and k3 are never live
// together.  The dense output of an accepted step is written before p and k1
// move to the step end, so the previous step needs no copy.
//
// BATCH: the queue holds pixels of every request of a batch; a lane looks up
// its pixel's request (camera, sample distance, volume diagonal) when it
// takes the pixel.  A pixel whose sample list would end beyond the list's
// capacity (off + cnt > cap), and every pixel when the scanned total did not
// fit an int (n_active[3] > 0), is skipped here and in the shading pass; the
// batch renders such pixels with the fused integrator.
//
// Resident CTAs: three per SM (up to 168 registers, no spills) for single
// frames of cubic volumes, four otherwise (measured: 1080p bar +1.8 %, bent
// beam -0.7 %, 4K quadratic step -9.5 % at three).
#pragma once

#include "k_integrate.cuh"

namespace ivv {

template <int P, bool MIXED, bool STATS, bool BATCH = false>
__global__ void __launch_bounds__(128, (P == 3 && !BATCH) ? 3 : 4) k5_trace(DevVolume V, DevCamera<float> cam, IntegrateArgs args, BatchArgs ba,
                                                   const int* __restrict__ cnt,
                                                   const float4* __restrict__ pair_in,
                                                   const float4* __restrict__ pair_out,
                                                   const int* __restrict__ pair_block,
                                                   const int* __restrict__ pair_count,
                                                   const int* __restrict__ active, const int* __restrict__ n_active,
                                                   int* __restrict__ queue_head, const int* __restrict__ off,
                                                   float4* __restrict__ sp, int cap, DevStats* __restrict__ st) {
  const int lane = threadIdx.x & 31;
  pdl_wait();
  const int nact = *n_active;
  if (nact == 0) return;
  const bool excess = BATCH && n_active[3] > 0;     // the sample offsets overflowed
  const int npix = args.npix;
  const float tol = args.rk_tol, cc = args.c;
  float ds = args.ds;
  float tail_eps = 1e-12f * V.diag;
  float hmin = 1e-7f * ds;
  float hmax = (float)args.max_step_samples * ds;
  int rq = 0;             // BATCH: request of the lane's pixel
  unsigned long long c_rhs = 0, c_steps = 0, c_rej = 0, c_fp64 = 0, c_cap = 0;

  int pix = -1;           // -1: needs a pixel; -2: queue drained
  int q = 0, np = 0, stage = 0, j = 0, nsamp = 0, nlast = 0, steps = 0, kidx = 0, blk = 0;
  BlockInfo B = V.blocks[0];
  float d[3], g_in[3], p[3], k1[3], ka[3], kb[3];
  float s = 0.f, h = 0.f, hh = 0.f, L = 0.f;

  WarpQueue wq(nact, queue_head, nullptr);
  for (;;) {
    if (__ballot_sync(0xffffffffu, pix >= 0) == 0) {     // the whole warp is idle: refill
      if (wq.done()) break;
      const int item = wq.take(lane, queue_head);
      if (pix == -1) {
        if (item < nact) {
          pix = __ldg(active + item);
          kidx = __ldg(off + item);
          np = __ldg(pair_count + pix);
          q = -1;
          stage = 0;
          if constexpr (BATCH) {
            if (excess || kidx < 0 || kidx + __ldg(cnt + item) > cap) {
              pix = -1;                  // beyond the sample list: the fused integrator's
            } else {
              rq = batch_request(ba, pix);
              const DevRequest& rr = ba.req[rq];
              ds = rr.ds;
              tail_eps = 1e-12f * rr.diag;
              hmin = 1e-7f * ds;
              hmax = (float)args.max_step_samples * ds;
            }
          }
        } else {
          pix = -2;
        }
      }
      wq.drained |= __ballot_sync(0xffffffffu, pix == -2);
    }

    bool live = pix >= 0;
    if (live && stage == 0) {
      // the next pair with a positive length, or the end of the pixel
      bool found = false;
      while (!found && ++q < np) {
        const size_t slot = (size_t)q * npix + pix;
        const float4 pi = pair_in[slot];
        const float4 po = pair_out[slot];
        L = po.x - pi.x;
        if (!(L > 0.f)) continue;
        blk = __ldg(pair_block + slot);
        B = V.blocks[blk];
        float o[3];
        if constexpr (BATCH) {
          const DevCamera<float>& cm = ba.req[rq].cam;
          const int loc = pix - __ldg(ba.pix0 + rq);
          make_ray<float>(cm, cm.x0 + loc % cm.w, cm.y0 + loc / cm.w, o, d);
        } else {
          make_ray<float>(cam, cam.x0 + pix % cam.w, cam.y0 + pix / cam.w, o, d);
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) g_in[r] = o[r] + pi.x * d[r];
        p[0] = pi.y; p[1] = pi.z; p[2] = pi.w;
        const float fl = floorf(L / ds);
        nsamp = (int)fl;
        nlast = nsamp + ((L - fl * ds > tail_eps) ? 1 : 0);
        s = 0.f;
        h = ds;
        j = 1;
        steps = 0;
        found = true;
      }
      if (!found) {
        pix = -1;
        live = false;
      }
    }
    // idle lanes (pixel done, queue drained) sit out the evaluation: they
    // would only add control-point loads of their own to the warp's
    if (!live) continue;
    // ---- this iteration's evaluation point
    float x[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      float v;
      if (stage == 0) v = p[r];
      else if (stage == 1) v = bs3_q2<float>(p[r], hh, k1[r]);
      else if (stage == 2) v = bs3_q3<float>(p[r], hh, ka[r]);
      else v = ka[r];                                   // pn
      x[r] = v < 0.f ? 0.f : (v > 1.f ? 1.f : v);
    }
    float W[3], rho, phi[3];
    // the contraction's outer loop unrolled by two here (measured: 4K
    // backward-facing step +4 %, the beam +1 %, the bar unchanged), and for
    // single frames of cubic volumes (168 registers) without the scalar
    // channel (bar +1.8 %, beam +1.2 %)
    rhs_eval<P, float, MIXED, false, 2, P == 3 && !BATCH>(V, B, x, g_in, d, cc, V.mode, W, rho, phi, c_fp64);
    if (STATS) ++c_rhs;
    if (stage == 0) {
      k1[0] = W[0]; k1[1] = W[1]; k1[2] = W[2];
      if (kidx < cap) sp[kidx] = make_float4(x[0], x[1], x[2], __int_as_float(blk));   // s_0: the entry
      ++kidx;
      if (j > nlast) continue;                          // zero-length remainder: pair done
    } else if (stage == 1) {
      ka[0] = W[0]; ka[1] = W[1]; ka[2] = W[2];         // k2
      stage = 2;
      continue;
    } else if (stage == 2) {
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float k2 = ka[r];
        ka[r] = bs3_pn<float>(p[r], hh, k1[r], k2, W[r]);   // pn
        kb[r] = bs3_e3<float>(k1[r], k2, W[r]);           // error combination, less k4
      }
      stage = 3;
      continue;
    } else {
      float err = 0.f;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float ae = fabsf(bs3_err<float>(hh, kb[r], W[r]));
        err = ae > err ? ae : err;
      }
      ++steps;
      const bool capped = steps >= args.max_steps;
      if (err <= tol || hh <= hmin || capped) {
        if (STATS) ++c_steps;
        if (capped) ++c_cap;
        const float s1 = last_end(s, hh, L);
        // samples inside (s, s1]: cubic Hermite through (p, k1) and (x, W)
        for (; j <= nlast; ++j) {
          const float st_ = (j <= nsamp) ? (float)j * ds : L;
          if (!capped && st_ > s1) break;
          float xs[3];
          if (capped || st_ >= s1) {
            xs[0] = x[0]; xs[1] = x[1]; xs[2] = x[2];
          } else {
            const float th = (st_ - s) / hh;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
              const float v = hermite<float>(th, hh, p[r], k1[r], x[r], W[r]);
              xs[r] = v < 0.f ? 0.f : (v > 1.f ? 1.f : v);
            }
          }
          if (kidx < cap) sp[kidx] = make_float4(xs[0], xs[1], xs[2], __int_as_float(blk));
          ++kidx;
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          p[r] = x[r];
          k1[r] = W[r];
        }
        s = s1;
        float fac = err > 0.f ? 0.9f * pow_third<float>(tol / err) : 5.f;
        fac = fac < 0.2f ? 0.2f : (fac > 5.f ? 5.f : fac);
        h = hh * fac;
        if (j > nlast) {
          stage = 0;                                    // pair done
          continue;
        }
      } else {
        if (STATS) ++c_rej;
        const float fac = 0.9f * pow_third<float>(tol / err);
        h = hh * (fac < 0.2f ? 0.2f : fac);
      }
    }
    // ---- the next step (after s_0, an accepted step or a rejected one)
    const float rem = L - s;
    hh = h < hmax ? h : hmax;
    hh = hh < rem ? hh : rem;
    stage = 1;
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
      c_rej += __shfl_down_sync(0xffffffffu, c_rej, o2);
      c_cap += __shfl_down_sync(0xffffffffu, c_cap, o2);
    }
    if (lane == 0) {
      atomicAdd(&st->rhs_evals, c_rhs);
      atomicAdd(&st->rk_steps, c_steps);
      atomicAdd(&st->rk_rejects, c_rej);
      atomicAdd(&st->step_cap, c_cap);
    }
  } else if (c_cap) {
    atomicAdd(&st->step_cap, c_cap);               // a cap counter: kept by every render
  }
}

template <int P, bool MIXED, bool STATS>
void launch_k5_trace(const DevVolume& V, const DevCamera<float>& cam, const IntegrateArgs& a, const SplitArgs& sa,
                     const float4* pin, const float4* pout, const int* pblk, const int* pcnt, const int* active,
                     const int* n_active, int* queue_head, DevStats* st, int num_sms, cudaStream_t s) {
  static int blocks_per_sm = -1;
  if (blocks_per_sm < 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k5_trace<P, MIXED, STATS>, 128, 0);
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  int grid = num_sms * blocks_per_sm;
  const int max_useful = (a.npix + 127) / 128;
  if (grid > max_useful) grid = max_useful > 0 ? max_useful : 1;
  launch_pdl(k5_trace<P, MIXED, STATS>, dim3(grid), dim3(128), s, V, cam, a, BatchArgs{}, (const int*)nullptr, pin,
             pout, pblk, pcnt, active, n_active, queue_head, sa.off, sa.sp, sa.cap, st);
}

template <int P>
void launch_integrate_split_p(const DevVolume& V, const DevCamera<float>& cam, const IntegrateArgs& a,
                              const SplitArgs& sa, bool mixed, bool stats, const float4* pin, const float4* pout,
                              const int* pblk, const int* pcnt, const int* active, const int* n_active,
                              int* queue_head, DevStats* st, int num_sms, cudaStream_t s) {
#define IVV_K5T(MM, SS) \
  launch_k5_trace<P, MM, SS>(V, cam, a, sa, pin, pout, pblk, pcnt, active, n_active, queue_head, st, num_sms, s)
  if (mixed) { if (stats) IVV_K5T(true, true); else IVV_K5T(true, false); }
  else { if (stats) IVV_K5T(false, true); else IVV_K5T(false, false); }
#undef IVV_K5T
}

}  // namespace ivv
