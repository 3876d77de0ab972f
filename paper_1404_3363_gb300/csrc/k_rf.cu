// Root-finding ray integration (§5.1, Eqs. 6-7), batched over all samples of
// all rays.  Because each sample's preimage is solved from its own initial
// guess, the samples of a ray are independent and the work is spread one
// thread per sample:
//   R1 rf_count     -- samples per active pixel (over its pairs)
//   R2 scan         -- exclusive scan of the counts (per-CTA scan, scan of the
//                      CTA sums, add-back)
//   R3 rf_expand    -- each sample's point g_j = o + (t_in + s_j) d, its block
//                      and an initial guess: the block's parameter centre, or
//                      the chord guess p_in + (s_j / L)(p_out - p_in); the
//                      learned guess overwrites it (K6 in k_mlp.cu)
//   R4 rf_newton    -- damped Newton on F(p) = phi(p) - g_j with a halving
//                      line search and clamping to [0,1]^3, stopped when ||F||
//                      is below rf_tol times the half width of the pixel at the
//                      sample's depth (the paper's pixel-accuracy criterion);
//                      the scalar at the converged point
//   R5 rf_composite -- per pixel, Alg. 1 with supersampling over its samples
//                      in front-to-back order, early termination (also the
//                      compositing pass of the split ODE integrator)
#include <cuda_runtime.h>

#include "ivv_device.cuh"

namespace ivv {

namespace {

constexpr int kScanBlock = 1024;

struct PairView {
  float L, t_in;
  float pin[3], pout[3];
  int blk;
  int nsamp, nlast;
};

__device__ __forceinline__ bool load_pair(const float4* pair_in, const float4* pair_out, const int* pair_block,
                                          size_t slot, float ds, float tail_eps, PairView& v) {
  const float4 pi = pair_in[slot], po = pair_out[slot];
  v.L = po.x - pi.x;
  if (!(v.L > 0.f)) return false;
  v.t_in = pi.x;
  v.pin[0] = pi.y; v.pin[1] = pi.z; v.pin[2] = pi.w;
  v.pout[0] = po.y; v.pout[1] = po.z; v.pout[2] = po.w;
  v.blk = pair_block[slot];
  const float fl = floorf(v.L / ds);
  v.nsamp = (int)fl;
  v.nlast = v.nsamp + ((v.L - fl * ds > tail_eps) ? 1 : 0);
  return true;
}

__global__ void k_rf_count(const float4* __restrict__ pair_in, const float4* __restrict__ pair_out,
                           const int* __restrict__ pair_block, const int* __restrict__ pair_count,
                           const int* __restrict__ active, const int* __restrict__ n_active, int npix, float ds,
                           float tail_eps, int* __restrict__ cnt) {
  pdl_wait();
  const int nact = *n_active;
  for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < nact; item += gridDim.x * blockDim.x) {
    const int pix = active[item];
    const int np = pair_count[pix];
    int c = 0;
    for (int q = 0; q < np; ++q) {
      PairView v;
      if (load_pair(pair_in, pair_out, pair_block, (size_t)q * npix + pix, ds, tail_eps, v)) c += v.nlast + 1;
    }
    cnt[item] = c;
  }
}

// exclusive scan within each CTA of kScanBlock items; CTA totals to sums[]
__global__ void __launch_bounds__(kScanBlock) k_scan_local(const int* __restrict__ in, const int* __restrict__ n_ptr,
                                                           int* __restrict__ out, int* __restrict__ sums) {
  __shared__ int warp_tot[kScanBlock / 32];
  pdl_wait();
  const int n = *n_ptr;
  const int i = blockIdx.x * kScanBlock + threadIdx.x;
  if (blockIdx.x * kScanBlock >= n) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int x = i < n ? in[i] : 0;
  int v = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) warp_tot[warp] = v;
  __syncthreads();
  if (warp == 0) {
    int w = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_tot[lane] = w;
  }
  __syncthreads();
  const int incl = v + (warp > 0 ? warp_tot[warp - 1] : 0);
  if (i < n) out[i] = incl - x;
  if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = incl;
}

// exclusive scan of the CTA sums (one CTA, chunks of kScanBlock) and total;
// the running total is kept in 64 bits, so a total beyond cap (at most
// INT_MAX) is reported as cap with the excess in total[1]
__global__ void __launch_bounds__(kScanBlock) k_scan_sums(int* __restrict__ sums, const int* __restrict__ n_ptr,
                                                          int cap, int* __restrict__ total) {
  __shared__ int warp_tot[kScanBlock / 32];
  __shared__ long long carry;
  pdl_wait();
  const int n = (*n_ptr + kScanBlock - 1) / kScanBlock;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += kScanBlock) {
    const int i = base + threadIdx.x;
    const int x = i < n ? sums[i] : 0;
    int v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane == 31) warp_tot[warp] = v;
    __syncthreads();
    if (warp == 0) {
      int w = warp_tot[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      warp_tot[lane] = w;
    }
    __syncthreads();
    const int incl = v + (warp > 0 ? warp_tot[warp - 1] : 0);
    const long long c = carry;
    if (i < n) sums[i] = (int)(c + incl - x);
    __syncthreads();
    if (threadIdx.x == kScanBlock - 1) carry = c + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *total = carry < (long long)cap ? (int)carry : cap;
    if (carry > (long long)cap) {                                  // overflow count
      const long long ex = carry - cap;
      total[1] = ex < 0x7fffffffll ? (int)ex : 0x7fffffff;
    }
  }
}

__global__ void k_scan_add(int* __restrict__ out, const int* __restrict__ n_ptr, const int* __restrict__ sums) {
  pdl_wait();
  const int n = *n_ptr;
  const int i = blockIdx.x * kScanBlock + threadIdx.x;
  if (i < n) out[i] += sums[blockIdx.x];
}

__global__ void k_rf_expand(DevCamera<float> cam, const float4* __restrict__ pair_in,
                            const float4* __restrict__ pair_out, const int* __restrict__ pair_block,
                            const int* __restrict__ pair_count, const int* __restrict__ active,
                            const int* __restrict__ n_active, const int* __restrict__ off, int npix, float ds,
                            float tail_eps, int guess, int cap, float4* __restrict__ sg, int* __restrict__ sblk,
                            float4* __restrict__ sp) {
  pdl_wait();
  const int nact = *n_active;
  for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < nact; item += gridDim.x * blockDim.x) {
    const int pix = active[item];
    const int xw = pix % cam.w, yw = pix / cam.w;
    float o[3], d[3];
    make_ray<float>(cam, cam.x0 + xw, cam.y0 + yw, o, d);
    const int np = pair_count[pix];
    int k = off[item];
    for (int q = 0; q < np; ++q) {
      PairView v;
      if (!load_pair(pair_in, pair_out, pair_block, (size_t)q * npix + pix, ds, tail_eps, v)) continue;
      for (int j = 0; j <= v.nlast; ++j, ++k) {
        if (k >= cap) return;
        const float s = j <= v.nsamp ? (float)j * ds : v.L;
        const float t = v.t_in + s;
        sg[k] = make_float4(o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2], s);
        sblk[k] = v.blk;
        float p[3];
        if (guess != 0) {
          // the chord point (the learned guess's samples carry it until the
          // inference replaces it: it keys their element sort)
          const float a = s / v.L;
#pragma unroll
          for (int r = 0; r < 3; ++r) p[r] = v.pin[r] + a * (v.pout[r] - v.pin[r]);
        } else {
          p[0] = p[1] = p[2] = 0.5f;
        }
        sp[k] = make_float4(p[0], p[1], p[2], 0.f);
      }
    }
  }
}

// abs_tol > 0: fixed stopping tolerance (point location); otherwise the
// pixel-accuracy rule of the camera.  p_out / it_out are optional.
// MIXED: the 3x3 Newton solve switches to FP64 where |det J| < tau_det.
template <int P, bool STATS, bool MIXED>
__global__ void __launch_bounds__(128) k_rf_newton(DevVolume V, DevCamera<float> cam, float rf_tol, float abs_tol,
                                                   const int* __restrict__ n_ptr, const float4* __restrict__ sg,
                                                   const int* __restrict__ sblk, const float4* __restrict__ sp,
                                                   float* __restrict__ srho, float4* __restrict__ p_out,
                                                   int* __restrict__ it_out, const int* __restrict__ perm,
                                                   DevStats* __restrict__ st) {
  pdl_wait();
  const int n = *n_ptr;
  unsigned long long c_it = 0, c_ev = 0, c_fail = 0, c_64 = 0;
  // half width of a pixel per unit depth (perspective) or absolute (ortho)
  const float px_half = cam.sy / (float)cam.H;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    // perm: the samples in the order of their guesses' elements, so a warp's
    // control-point loads meet few elements
    const int i = perm ? __ldg(perm + k) : k;
    const float4 g4 = sg[i];
    const float g[3] = {g4.x, g4.y, g4.z};
    const BlockInfo B = V.blocks[sblk[i]];
    float tol;
    if (abs_tol > 0.f) {
      tol = abs_tol;
    } else {
      float depth = 1.f;
      if (!cam.ortho)
        depth = (g[0] - cam.eye[0]) * cam.f[0] + (g[1] - cam.eye[1]) * cam.f[1] + (g[2] - cam.eye[2]) * cam.f[2];
      tol = rf_tol * px_half * depth;
    }
    // never below FP32 resolution of the coordinates
    tol = fmaxf(tol, 2e-7f * (fabsf(g[0]) + fabsf(g[1]) + fabsf(g[2]) + V.diag));
    const float4 p4 = sp[i];
    float p[3] = {fminf(fmaxf(p4.x, 0.f), 1.f), fminf(fmaxf(p4.y, 0.f), 1.f), fminf(fmaxf(p4.z, 0.f), 1.f)};
    float phi[3], J[3][3], rc;
    eval_block<P, float, true>(V, B, p, phi, J, rc);
    if (STATS) ++c_ev;
    float F[3] = {phi[0] - g[0], phi[1] - g[1], phi[2] - g[2]};
    float nF = sqrtf(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
    int it = 0;
    for (; it < V.max_newton && nF > tol; ++it) {
      float dx[3];
      const float rhs[3] = {-F[0], -F[1], -F[2]};
      const float det = solve3<float>(J, rhs, dx);
      if constexpr (MIXED) {
        if (fabsf(det) < B.tau_det) {
          double Jd[3][3], bd[3], xd[3];
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            bd[r] = rhs[r];
#pragma unroll
            for (int c = 0; c < 3; ++c) Jd[r][c] = J[r][c];
          }
          solve3<double>(Jd, bd, xd);
#pragma unroll
          for (int r = 0; r < 3; ++r) dx[r] = (float)xd[r];
          ++c_64;
        }
      }
      float lam = 1.f;
      bool moved = false;
      for (int ls = 0; ls < 6; ++ls) {
        float q[3], fq[3], Jq[3][3], rq;
#pragma unroll
        for (int r = 0; r < 3; ++r) q[r] = fminf(fmaxf(p[r] + lam * dx[r], 0.f), 1.f);
        eval_block<P, float, true>(V, B, q, fq, Jq, rq);
        if (STATS) ++c_ev;
        const float G[3] = {fq[0] - g[0], fq[1] - g[1], fq[2] - g[2]};
        const float nG = sqrtf(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
        if (nG < nF || ls == 5) {
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            p[r] = q[r];
            F[r] = G[r];
#pragma unroll
            for (int c = 0; c < 3; ++c) J[r][c] = Jq[r][c];
          }
          rc = rq;
          moved = nG < nF;
          nF = nG;
          break;
        }
        lam *= 0.5f;
      }
      if (!moved) break;
    }
    if (STATS) c_it += it;
    if (nF > tol) ++c_fail;
    if (p_out) p_out[i] = make_float4(p[0], p[1], p[2], nF);
    if (it_out) it_out[i] = nF <= tol ? it : -1 - it;
    const float rho = scalar_at<P, float>(V, B, V.mode, p, J, rc);
    if (srho) srho[i] = rho;
  }
  if (STATS) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      c_it += __shfl_down_sync(0xffffffffu, c_it, o);
      c_ev += __shfl_down_sync(0xffffffffu, c_ev, o);
      c_fail += __shfl_down_sync(0xffffffffu, c_fail, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&st->rf_newton_iters, c_it);
      atomicAdd(&st->rhs_evals, c_ev);
      atomicAdd(&st->rf_unconverged, c_fail);
    }
  } else if (c_fail) {
    atomicAdd(&st->rf_unconverged, c_fail);       // a cap counter: kept by every render
  }
  if (MIXED && c_64) atomicAdd(&st->fp64_solves, c_64);
}

__global__ void k_rf_composite(DevTF tf, int K, float early, const float4* __restrict__ pair_in,
                               const float4* __restrict__ pair_out, const int* __restrict__ pair_block,
                               const int* __restrict__ pair_count, const int* __restrict__ active,
                               const int* __restrict__ n_active, const int* __restrict__ off, int npix, float ds,
                               float tail_eps, int cap, const float* __restrict__ srho,
                               float4* __restrict__ out, DevStats* __restrict__ st, bool stats) {
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
  const int nact = *n_active;
  unsigned long long c_samp = 0;
  for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < nact; item += gridDim.x * blockDim.x) {
    const int pix = active[item];
    const int np = pair_count[pix];
    int k = off[item];
    float C[3] = {0.f, 0.f, 0.f}, a = 0.f;
    bool done = false;
    for (int q = 0; q < np && !done; ++q) {
      PairView v;
      if (!load_pair(pair_in, pair_out, pair_block, (size_t)q * npix + pix, ds, tail_eps, v)) continue;
      float rho_prev = 0.f, s_prev = 0.f;
      for (int j = 0; j <= v.nlast; ++j, ++k) {
        if (k >= cap) {
          done = true;
          break;
        }
        const float rho = srho[k];
        const float s = j <= v.nsamp ? (float)j * ds : v.L;
        ++c_samp;
        if (j > 0 && !done) {
          const float invK = 1.f / (float)K;
          const float dr = rho - rho_prev;
          const float tau = tf.sigma * (s - s_prev) * invK;
          for (int kk = 0; kk < K; ++kk) {
            float x = (rho_prev + ((float)kk + 0.5f) * invK * dr - tf.lo) * tf.inv_range;
            x = fminf(fmaxf(x, 0.f), 1.f);
            const float4 c = tf_eval(s_r, s_rgba, s_seg, tf.n, x);
            const float T = __expf(-tau * c.w);
            const float w = (1.f - T) * (1.f - a);
            C[0] += w * c.x;
            C[1] += w * c.y;
            C[2] += w * c.z;
            a += w;
          }
          if (a >= early) done = true;
        }
        rho_prev = rho;
        s_prev = s;
      }
    }
    out[pix] = make_float4(C[0], C[1], C[2], a);
  }
  if (stats) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c_samp += __shfl_down_sync(0xffffffffu, c_samp, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&st->samples, c_samp);
  }
}

}  // namespace

namespace {
__global__ void k_fill_center(float4* __restrict__ p, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = make_float4(0.5f, 0.5f, 0.5f, 0.f);
}
}  // namespace

void launch_fill_center(float4* p, int n, cudaStream_t s) {
  if (n > 0) k_fill_center<<<(n + 255) / 256, 256, 0, s>>>(p, n);
}

void launch_rf_count(const float4* pin, const float4* pout, const int* pblk, const int* pcnt, const int* active,
                     const int* n_active, int npix, float ds, float tail_eps, int* cnt, int num_sms, cudaStream_t s) {
  launch_pdl(k_rf_count, dim3(num_sms * 8), dim3(256), s, pin, pout, pblk, pcnt, active, n_active, npix, ds, tail_eps,
             cnt);
}

void launch_rf_scan(const int* cnt, const int* n_active, int npix, int* off, int* sums, int cap, int* total,
                    cudaStream_t s) {
  const int blocks = (npix + kScanBlock - 1) / kScanBlock;
  launch_pdl(k_scan_local, dim3(blocks), dim3(kScanBlock), s, cnt, n_active, off, sums);
  launch_pdl(k_scan_sums, dim3(1), dim3(kScanBlock), s, sums, n_active, cap, total);
  launch_pdl(k_scan_add, dim3(blocks), dim3(kScanBlock), s, off, n_active, (const int*)sums);
}

void launch_rf_expand(const DevCamera<float>& cam, const float4* pin, const float4* pout, const int* pblk,
                      const int* pcnt, const int* active, const int* n_active, const int* off, int npix, float ds,
                      float tail_eps, int guess, int cap, float4* sg, int* sblk, float4* sp, int num_sms,
                      cudaStream_t s) {
  launch_pdl(k_rf_expand, dim3(num_sms * 8), dim3(256), s, cam, pin, pout, pblk, pcnt, active, n_active, off, npix, ds,
             tail_eps, guess, cap, sg, sblk, sp);
}

// Sort key of every sample: the global index of the Bezier element that
// holds its Newton start.
__global__ void __launch_bounds__(256) k_rf_elem_key(DevVolume V, const int* __restrict__ n_ptr,
                                                     const int* __restrict__ sblk, const float4* __restrict__ sp,
                                                     int* __restrict__ key) {
  pdl_wait();
  const int n = *n_ptr;
  const float* brk = V.brk32;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const BlockInfo B = V.blocks[__ldg(sblk + i)];
    const float4 p4 = sp[i];
    const float p[3] = {p4.x, p4.y, p4.z};
    int e[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float x = fminf(fmaxf(p[d], 0.f), 1.f);
      if ((B.uniform >> d) & 1) {
        const int k = (int)(x * (float)B.nseg[d]);
        e[d] = k < B.nseg[d] - 1 ? k : B.nseg[d] - 1;
      } else {
        float loc, sc;
        e[d] = locate<float>(brk + B.brk_off[d], B.nseg[d], x, loc, sc);
      }
    }
    key[i] = B.elem_off + (e[2] * B.nseg[1] + e[1]) * B.nseg[0] + e[0];
  }
}

void launch_rf_elem_key(const DevVolume& V, const int* n_ptr, const int* sblk, const float4* sp, int* key, int num_sms,
                        cudaStream_t s) {
  launch_pdl(k_rf_elem_key, dim3(num_sms * 8), dim3(256), s, V, n_ptr, sblk, sp, key);
}

void launch_rf_newton(const DevVolume& V, const DevCamera<float>& cam, float rf_tol, float abs_tol, const int* n_ptr,
                      const float4* sg, const int* sblk, const float4* sp, float* srho, float4* p_out, int* it_out,
                      DevStats* st, bool stats, bool mixed, int num_sms, cudaStream_t s, const int* perm) {
  const int grid = num_sms * 16;
#define IVV_RFN(PP, SS, MM) \
  launch_pdl(k_rf_newton<PP, SS, MM>, dim3(grid), dim3(128), s, V, cam, rf_tol, abs_tol, n_ptr, sg, sblk, sp, srho, \
             p_out, it_out, perm, st)
  if (V.P == 2) {
    if (mixed) { if (stats) IVV_RFN(2, true, true); else IVV_RFN(2, false, true); }
    else { if (stats) IVV_RFN(2, true, false); else IVV_RFN(2, false, false); }
  } else {
    if (mixed) { if (stats) IVV_RFN(3, true, true); else IVV_RFN(3, false, true); }
    else { if (stats) IVV_RFN(3, true, false); else IVV_RFN(3, false, false); }
  }
#undef IVV_RFN
}

void launch_rf_composite(const DevTF& tf, int K, float early, const float4* pin, const float4* pout, const int* pblk,
                         const int* pcnt, const int* active, const int* n_active, const int* off, int npix, float ds,
                         float tail_eps, int cap, const float* srho, float4* out, DevStats* st,
                         bool stats, int num_sms, cudaStream_t s) {
  launch_pdl(k_rf_composite, dim3(num_sms * 8), dim3(128), s, tf, K, early, pin, pout, pblk, pcnt, active, n_active,
             off, npix, ds, tail_eps, cap, srho, out, st, stats);
}

}  // namespace ivv
