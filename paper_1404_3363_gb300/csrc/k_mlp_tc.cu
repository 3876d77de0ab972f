// K6 inference of the learned initial guess on the 5th-generation tensor
// cores: per block a 3-64-64-3 perceptron (ReLU), FP16 weights, FP32
// accumulation.  One CTA of 128 threads takes a contiguous run of tiles of
// 128 listed points (one thread per point = one row of the MMAs); each layer
// is one tcgen05.mma chain (M = 128, issued by one thread, A and B read from
// shared memory through matrix descriptors, the FP32 accumulator in tensor
// memory, 64 columns allocated once per CTA):
//   layer 1 (3 -> 64): A = (x_hi, x_lo, 1) per row, each input split into
//     two FP16 parts so that the products keep FP32 accuracy, against
//     B = (W1, W1, b1): K = 16, N = 64;
//   layer 2 (64 -> 64): A = the ReLU of layer 1 rounded to FP16, B = W2:
//     K = 64 (four K = 16 steps), N = 64;
//   layer 3 (64 -> 3): A = the ReLU of layer 2 (+ b2) rounded to FP16,
//     B = W3 padded to N = 16: K = 64.
// Between layers every thread reads its accumulator row (tcgen05.ld), applies
// bias and ReLU, and writes the next A row.  A tile whose points lie in
// several blocks runs one pass per block with that block's weights (staged
// in shared memory when the block changes); rows of other blocks ride along
// and are not written.  Each MMA chain's completion is awaited on an mbarrier
// with a bounded spin: a wait that gives up counts in
// DevStats::async_timeouts and the CTA writes no further points.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "ivv_device.cuh"
#include "mlp.cuh"

namespace ivv {
namespace {

constexpr int kTcRows = 128;               // points per tile = M of the MMA = threads per CTA
constexpr unsigned kTmemCols = 64;         // accumulator: 128 lanes x 64 FP32 columns
constexpr long long kWaitSpins = 1ll << 22;

// Shared-memory operands in the K-major layout without swizzling: 8 x 8
// "core matrices" (8 rows of 16 bytes, 128 contiguous bytes); along K the
// core matrices of an 8-row group follow each other (leading byte offset
// 128), and the 8-row groups are K / 8 core matrices apart (stride byte
// offset 16 K bytes).
template <int K>
__device__ __forceinline__ int core_off(int row, int k) {
  return (row >> 3) * (16 * K) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}
constexpr int kK1 = 16;                    // layer 1's K: (x_hi, x_lo, 1) padded
constexpr int kN3 = 16;                    // layer 3's N: 3 outputs padded

struct __align__(1024) TcSmem {
  __half a[kTcRows * kMlpH];       // A operand of the current layer (16 KB; layer 1 uses 4 KB)
  __half b2[kMlpH * kMlpH];        // W2 of the loaded block (8 KB)
  __half b1[kMlpH * kK1];          // (W1, W1, b1) (2 KB)
  __half b3[kN3 * kMlpH];          // W3, rows 3..15 zero (2 KB)
  float bias2[kMlpH];
  float bias3[4];
  float nc[3], ninv[3];            // input normalisation of the loaded block
  unsigned long long mbar;
  unsigned tmem;
  int block;                       // block whose weights are loaded (-1: none)
  int next;                        // the tile's next block to run
  int err;
};

// Matrix descriptor of a shared-memory operand starting at p (no swizzle)
// whose 8-row groups are sbo bytes apart.
__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t sbo) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint64_t d = (uint64_t)((a >> 4) & 0x3FFFu);     // start address
  d |= (uint64_t)(128u >> 4) << 16;                // leading byte offset: next core matrix along K
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;     // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                          // descriptor version of tcgen05
  return d;                                        // base offset 0, layout: no swizzle
}

// Instruction descriptor, kind::f16: FP32 accumulator, FP16 A and B, both
// K-major, M = 128 and the given N.
constexpr uint32_t idesc_f16(int n) {
  return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tmem_alloc(unsigned* dst) {       // one whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(kTmemCols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(unsigned taddr) {    // the allocating warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(unsigned d, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned long long* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* mbar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// 16 consecutive FP32 columns of this thread's accumulator row.
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Bounded wait for the phase `parity` of the MMA barrier; false if it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned long long* mbar, unsigned parity) {
  for (long long i = 0; i < kWaitSpins; ++i)
    if (mbar_try_wait(mbar, parity)) return true;
  return false;
}

// One MMA round of the CTA: every thread has written its A row (generic
// proxy); thread 0 issues `issue` and commits; all wait (bounded) for the
// chain.  Returns false (the same on every thread) if a wait gave up.
template <class Issue>
__device__ __forceinline__ bool mma_round(TcSmem& sm, unsigned& phase, Issue issue) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the A rows, for the tensor cores
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    tc_fence_after();
    issue();
    tc_commit(&sm.mbar);
  }
  const bool ok = mbar_wait(&sm.mbar, phase);
  phase ^= 1u;
  if (!ok) atomicOr(&sm.err, 1);
  __syncthreads();
  if (sm.err) return false;
  tc_fence_after();
  return true;
}

// Accumulator row -> bias, ReLU, FP16 -> the next layer's A row (K = 64).
__device__ __forceinline__ void relu_row_to_a(TcSmem& sm, unsigned taddr_row, const float* bias, int row) {
#pragma unroll
  for (int c0 = 0; c0 < kMlpH; c0 += 16) {
    float v[16];
    tmem_ld16(taddr_row + (unsigned)c0, v);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      __align__(16) __half q[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float z = v[8 * h + e] + (bias ? bias[c0 + 8 * h + e] : 0.f);
        q[e] = __float2half_rn(fmaxf(z, 0.f));
      }
      *reinterpret_cast<uint4*>(reinterpret_cast<char*>(sm.a) + core_off<kMlpH>(row, c0 + 8 * h)) =
          *reinterpret_cast<const uint4*>(q);
    }
  }
}

__global__ void __launch_bounds__(kTcRows, 8) k_mlp_infer_tc(const __half* __restrict__ theta16_all,
                                                         const MlpNorm* __restrict__ norms,
                                                         const float4* __restrict__ g, const int* __restrict__ gblk,
                                                         const int* __restrict__ n_ptr, int n_static,
                                                         const int* __restrict__ perm, float4* __restrict__ p_out,
                                                         DevStats* __restrict__ st) {
  __shared__ TcSmem sm;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) tmem_alloc(&sm.tmem);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sm.block = -1;
    sm.err = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = sm.tmem;
  const unsigned trow = tmem + ((unsigned)(warp * 32) << 16);   // this thread's accumulator row (TMEM lane)
  const int n = n_ptr ? *n_ptr : n_static;
  unsigned phase = 0;
  // each CTA takes a contiguous run of tiles: neighbouring list entries
  // mostly share a block, so the staged weights are reused
  const int tiles = (n + kTcRows - 1) / kTcRows;
  const int per_cta = (tiles + (int)gridDim.x - 1) / (int)gridDim.x;
  const int tile0 = blockIdx.x * per_cta, tile1 = min(tiles, tile0 + per_cta);
  for (int tile = tile0; tile < tile1; ++tile) {
    int item = tile * kTcRows + tid;                // the list entry of this row
    if (perm != nullptr && item < n) item = __ldg(perm + item);
    const int myb = item < n ? __ldg(gblk + item) : -1;
    float4 gi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (item < n) gi = __ldg(g + item);
    bool done = myb < 0;
    for (int pass = 0; pass < kTcRows; ++pass) {
      // the smallest block of the tile not yet done
      if (tid == 0) sm.next = INT_MAX;
      __syncthreads();
      if (!done) atomicMin(&sm.next, myb);
      __syncthreads();
      const int bsel = sm.next;
      if (bsel == INT_MAX || sm.err) break;
      if (sm.block != bsel) {
        const __half* th = theta16_all + (size_t)bsel * kMlpStride;
        for (int c = tid; c < kMlpH * (kMlpH / 8); c += kTcRows) {
          const int nrow = c / (kMlpH / 8), kc = c % (kMlpH / 8);
          const uint4 v = *reinterpret_cast<const uint4*>(th + kOffW2 + nrow * kMlpH + kc * 8);
          *reinterpret_cast<uint4*>(reinterpret_cast<char*>(sm.b2) + core_off<kMlpH>(nrow, kc * 8)) = v;
        }
        if (tid < kMlpH) {
          // (W1, W1, b1) of hidden unit tid: pairs with the row (x_hi, x_lo, 1)
          __align__(16) __half r[kK1];
          const __half z = __float2half_rn(0.f);
#pragma unroll
          for (int k = 0; k < kK1; ++k) r[k] = z;
#pragma unroll
          for (int k = 0; k < 3; ++k) r[k] = r[3 + k] = th[kOffW1 + 3 * tid + k];
          r[6] = th[kOffB1 + tid];
          *reinterpret_cast<uint4*>(reinterpret_cast<char*>(sm.b1) + core_off<kK1>(tid, 0)) =
              *reinterpret_cast<const uint4*>(r);
          *reinterpret_cast<uint4*>(reinterpret_cast<char*>(sm.b1) + core_off<kK1>(tid, 8)) =
              *reinterpret_cast<const uint4*>(r + 8);
          sm.bias2[tid] = __half2float(th[kOffB2 + tid]);
        }
        for (int c = tid; c < kN3 * (kMlpH / 8); c += kTcRows) {
          const int nrow = c / (kMlpH / 8), kc = c % (kMlpH / 8);
          uint4 v = make_uint4(0u, 0u, 0u, 0u);
          if (nrow < 3) v = *reinterpret_cast<const uint4*>(th + kOffW3 + nrow * kMlpH + kc * 8);
          *reinterpret_cast<uint4*>(reinterpret_cast<char*>(sm.b3) + core_off<kMlpH>(nrow, kc * 8)) = v;
        }
        if (tid < 3) {
          sm.bias3[tid] = __half2float(th[kOffB3 + tid]);
          sm.nc[tid] = norms[bsel].c[tid];
          sm.ninv[tid] = norms[bsel].inv_h[tid];
        }
        __syncthreads();
        if (tid == 0) sm.block = bsel;
      }
      const bool mine = !done && myb == bsel;
      // layer 1: the row (x_hi, x_lo, 1, 0 ...) of this point (zero for rows
      // of other blocks)
      {
        const float x[3] = {(gi.x - sm.nc[0]) * sm.ninv[0], (gi.y - sm.nc[1]) * sm.ninv[1],
                            (gi.z - sm.nc[2]) * sm.ninv[2]};
        __align__(16) __half r[kK1];
        const __half z = __float2half_rn(0.f);
#pragma unroll
        for (int k = 0; k < kK1; ++k) r[k] = z;
        if (mine) {
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const __half hi = __float2half_rn(x[k]);
            r[k] = hi;
            r[3 + k] = __float2half_rn(x[k] - __half2float(hi));
          }
          r[6] = __float2half_rn(1.f);
        }
        *reinterpret_cast<uint4*>(reinterpret_cast<char*>(sm.a) + core_off<kK1>(tid, 0)) =
            *reinterpret_cast<const uint4*>(r);
        *reinterpret_cast<uint4*>(reinterpret_cast<char*>(sm.a) + core_off<kK1>(tid, 8)) =
            *reinterpret_cast<const uint4*>(r + 8);
      }
      if (!mma_round(sm, phase, [&] {
            tc_mma(tmem, smem_desc(sm.a, 16 * kK1), smem_desc(sm.b1, 16 * kK1), idesc_f16(kMlpH), 0);
          }))
        break;
      relu_row_to_a(sm, trow, nullptr, tid);          // h1 (b1 is in the MMA)
      // layer 2
      if (!mma_round(sm, phase, [&] {
#pragma unroll
            for (int k = 0; k < kMlpH / 16; ++k)
              tc_mma(tmem, smem_desc(reinterpret_cast<const char*>(sm.a) + 256 * k, 16 * kMlpH),
                     smem_desc(reinterpret_cast<const char*>(sm.b2) + 256 * k, 16 * kMlpH), idesc_f16(kMlpH),
                     k > 0);
          }))
        break;
      relu_row_to_a(sm, trow, sm.bias2, tid);         // h2
      // layer 3
      if (!mma_round(sm, phase, [&] {
#pragma unroll
            for (int k = 0; k < kMlpH / 16; ++k)
              tc_mma(tmem, smem_desc(reinterpret_cast<const char*>(sm.a) + 256 * k, 16 * kMlpH),
                     smem_desc(reinterpret_cast<const char*>(sm.b3) + 256 * k, 16 * kMlpH), idesc_f16(kN3), k > 0);
          }))
        break;
      float v[16];
      tmem_ld16(trow, v);
      if (mine) {
        p_out[item] = make_float4(v[0] + sm.bias3[0], v[1] + sm.bias3[1], v[2] + sm.bias3[2], 0.f);
        done = true;
      }
      tc_fence_before();
      __syncthreads();                  // the accumulator and the A rows are free again
    }
    if (sm.err) break;
  }
  __syncthreads();
  if (sm.err) {
    // an MMA chain that did not complete in time: wait once more (bounded)
    // before its tensor memory is released
    if (tid == 0) {
      mbar_wait(&sm.mbar, phase ^ 1u);
      atomicAdd(&st->async_timeouts, 1ull);
    }
    __syncthreads();
  }
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem);
  }
}

// Counting sort of list entries by block (the guess list of the RF method):
// perm lists the entries block after block, so the inference's tiles hold
// one block each and run one pass.  Each CTA takes a contiguous range of the
// list and counts it in shared memory (atomics aggregated per warp over the
// lanes of one block); only its per-block totals go to global memory, so a
// block's global counter sees one atomic per CTA instead of one per warp.
// hist: [n_blocks + 1] ints (zeroed by the caller).  Volumes with more
// blocks than kSortSharedBlocks count with global atomics directly.
constexpr int kSortSharedBlocks = 4096;

__device__ __forceinline__ void cta_range(int n, int& i0, int& i1) {
  const int per = (((n + (int)gridDim.x - 1) / (int)gridDim.x) + 31) & ~31;
  i0 = min(n, (int)blockIdx.x * per);
  i1 = min(n, i0 + per);
}

// Warp-aggregated count of the entries [i0, i1) into cnt (shared or global).
__device__ __forceinline__ void count_range(const int* __restrict__ gblk, int i0, int i1, int* cnt) {
  for (int base = i0; base < i1; base += blockDim.x) {
    const int i = base + (int)threadIdx.x;
    const int b = i < i1 ? __ldg(gblk + i) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    if (b >= 0 && (threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1)) atomicAdd(cnt + b, __popc(peers));
  }
}

template <bool SHARED>
__global__ void k_sort_hist(const int* __restrict__ gblk, const int* __restrict__ n_ptr, int n_blocks,
                            int* __restrict__ hist) {
  extern __shared__ int s_cnt[];
  int i0, i1;
  cta_range(*n_ptr, i0, i1);
  if constexpr (SHARED) {
    for (int b = threadIdx.x; b < n_blocks; b += blockDim.x) s_cnt[b] = 0;
    __syncthreads();
    count_range(gblk, i0, i1, s_cnt);
    __syncthreads();
    for (int b = threadIdx.x; b < n_blocks; b += blockDim.x)
      if (s_cnt[b]) atomicAdd(hist + b, s_cnt[b]);
  } else {
    count_range(gblk, i0, i1, hist);
  }
}

__global__ void k_sort_scan(int* __restrict__ hist, int n_blocks) {
  __shared__ int s_sum[1024];
  // exclusive scan of hist[0..n_blocks) in place by one CTA: per-thread runs,
  // then a scan of the run totals
  const int per = (n_blocks + (int)blockDim.x - 1) / (int)blockDim.x;
  const int b0 = threadIdx.x * per, b1 = min(n_blocks, b0 + per);
  int sum = 0;
  for (int b = b0; b < b1; ++b) sum += hist[b];
  s_sum[threadIdx.x] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (unsigned t = 0; t < blockDim.x; ++t) {
      const int v = s_sum[t];
      s_sum[t] = acc;
      acc += v;
    }
  }
  __syncthreads();
  int acc = s_sum[threadIdx.x];
  for (int b = b0; b < b1; ++b) {
    const int v = hist[b];
    hist[b] = acc;
    acc += v;
  }
}

// cursor: the scanned histogram, advanced as entries are placed.  SHARED:
// the CTA counts its range again, claims one run per block from the global
// cursor, then places its entries inside its runs (shared running offsets).
template <bool SHARED>
__global__ void k_sort_scatter(const int* __restrict__ gblk, const int* __restrict__ n_ptr, int n_blocks,
                               int* __restrict__ cursor, int* __restrict__ perm) {
  extern __shared__ int s_dyn[];
  const int lane = threadIdx.x & 31;
  int i0, i1;
  cta_range(*n_ptr, i0, i1);
  int* off = cursor;
  if constexpr (SHARED) {
    int* s_cnt = s_dyn;
    off = s_dyn + n_blocks;
    for (int b = threadIdx.x; b < n_blocks; b += blockDim.x) s_cnt[b] = 0;
    __syncthreads();
    count_range(gblk, i0, i1, s_cnt);
    __syncthreads();
    for (int b = threadIdx.x; b < n_blocks; b += blockDim.x) off[b] = s_cnt[b] ? atomicAdd(cursor + b, s_cnt[b]) : 0;
    __syncthreads();
  }
  for (int base = i0; base < i1; base += blockDim.x) {
    const int i = base + (int)threadIdx.x;
    const int b = i < i1 ? __ldg(gblk + i) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int leader = __ffs(peers) - 1;
    int at = 0;
    if (b >= 0 && lane == leader) at = atomicAdd(off + b, __popc(peers));
    at = __shfl_sync(0xffffffffu, at, leader);
    if (b >= 0) perm[at + __popc(peers & ((1u << lane) - 1u))] = i;
  }
}

}  // namespace

void launch_block_sort(const int* gblk, const int* n_ptr, int n_blocks, int* hist, int* perm, int num_sms,
                       cudaStream_t s) {
  cudaMemsetAsync(hist, 0, sizeof(int) * (size_t)(n_blocks + 1), s);
  const int grid = num_sms * 8;
  if (n_blocks <= kSortSharedBlocks) {
    k_sort_hist<true><<<grid, 256, sizeof(int) * n_blocks, s>>>(gblk, n_ptr, n_blocks, hist);
    k_sort_scan<<<1, 1024, 0, s>>>(hist, n_blocks);
    k_sort_scatter<true><<<grid, 256, 2 * sizeof(int) * n_blocks, s>>>(gblk, n_ptr, n_blocks, hist, perm);
  } else {
    k_sort_hist<false><<<grid, 256, 0, s>>>(gblk, n_ptr, n_blocks, hist);
    k_sort_scan<<<1, 1024, 0, s>>>(hist, n_blocks);
    k_sort_scatter<false><<<grid, 256, 0, s>>>(gblk, n_ptr, n_blocks, hist, perm);
  }
}

void launch_mlp_infer(const __half* theta16, const MlpNorm* norms, const float4* g, const int* gblk, const int* n_ptr,
                      int n_static, float4* p_out, DevStats* st, int num_sms, cudaStream_t s, const int* perm) {
  int grid = num_sms * 8;         // 8 CTAs of 27 KB shared memory and 64 TMEM columns fill an SM
  if (!n_ptr) {
    const int tiles = (n_static + kTcRows - 1) / kTcRows;
    grid = tiles < grid ? tiles : grid;
    if (grid < 1) return;
  }
  k_mlp_infer_tc<<<grid, kTcRows, 0, s>>>(theta16, norms, g, gblk, n_ptr, n_static, perm, p_out, st);
}

}  // namespace ivv
