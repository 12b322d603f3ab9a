// Weight-stationary BF16 GEMM on the 5th-generation tensor cores for the
// guess network's inference: Y = act(X W^T + b) for one layer, X [M][kp]
// BF16 rows, W [N][kp] BF16 (N <= 256, the whole W fits in shared memory).
//
// Persistent CTAs (one per SM) keep W in shared memory for the whole launch
// and walk the 128-row tiles of X (tile = blockIdx.x + i gridDim.x):
//  * warp 0 (one lane) is the producer: it loads W once and then the tiles'
//    64-column K slices with TMA (cp.async.bulk.tensor, 128-byte swizzle)
//    into a ring of STAGES shared-memory stages, each completing on its own
//    barrier with the copied byte count;
//  * warp 1 (one lane) issues tcgen05.mma kind::f16 (BF16 operands, FP32
//    accumulation) for every slice into one of two accumulators in tensor
//    memory (tile parity), frees the stage with tcgen05.commit and, after a
//    tile's last slice, hands the accumulator to the epilogue;
//  * warps 2..9 read the accumulator with tcgen05.ld (warp w owns lanes
//    32 (w mod 4) ..; two warps per lane quarter, each half of the columns),
//    add the bias (staged in shared memory), apply ReLU, convert and store
//    the rows, and give the accumulator back; so the epilogue of one tile
//    overlaps the MMAs of the next.
// Operands are K-major with the 128-byte swizzle: 8-row x 128-byte atoms
// (64 BF16 values of K per row), 1024 bytes between 8-row groups; the K
// steps of 16 inside an atom advance the descriptor's start address by 32
// bytes.  W is stored as ceil(kp / 64) such column blocks of npad rows.
// Every wait is bounded; a wait that gives up sets *err, the CTA waits once
// more (bounded) for the copies and MMAs it issued, and frees its tensor
// memory.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "device.cuh"

namespace frk {
namespace umws {

constexpr int BM = 128, BK = 64, STAGES = 4, EPI_WARPS = 8, THREADS = 64 + 32 * EPI_WARPS;
constexpr unsigned A_STAGE = BM * BK * 2;  // 16 KB per stage
constexpr unsigned TMEM_COLS = 512;        // two accumulators of up to 256 columns
constexpr size_t kSmemLimit = 227 * 1024;

__host__ __device__ inline int npad_of(int n) { return (n + 15) / 16 * 16; }
__host__ __device__ inline int nkb_of(int kp) { return (kp + BK - 1) / BK; }  // 64-wide column blocks of K
__host__ __device__ inline size_t w_bytes(int n, int kp) { return (size_t)nkb_of(kp) * npad_of(n) * 128; }
// shared memory: W (1024-aligned blocks), the A ring, the bias row, barriers
// and the tensor-memory slot
__host__ __device__ inline size_t smem_bytes(int n, int kp) {
  return w_bytes(n, kp) + (size_t)STAGES * A_STAGE + 4 * (size_t)npad_of(n) + 256 + 1024;  // + alignment slack
}
inline bool fits(int n, int kp) { return n <= 256 && smem_bytes(n, kp) <= kSmemLimit; }

// shared-memory matrix descriptor, K-major, 128-byte swizzle: start address,
// stride byte offset 1024 (8-row groups), descriptor version, layout type 2
__device__ __forceinline__ unsigned long long sdesc_sw128(unsigned saddr) {
  unsigned long long d = 0;
  d |= (unsigned long long)((saddr >> 4) & 0x3FFFu);
  d |= (unsigned long long)(1u) << 16;               // leading byte offset (unused for swizzled K-major)
  d |= (unsigned long long)((1024u >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;                                   // descriptor version
  d |= 2ull << 61;                                   // 128-byte swizzle
  return d;
}
__host__ __device__ constexpr unsigned idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(m >> 4) << 24);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

template <bool RELU, bool OUT_BF16>
__global__ void __launch_bounds__(THREADS, 1)
    k_umma_ws(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap wmap, int M, int N, int kp,
              const float* __restrict__ bias, void* out, int ldo, int* err) {
  extern __shared__ unsigned char usm_raw[];
  // 1024-byte alignment for the swizzled atoms
  unsigned char* usm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(usm_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int npad = npad_of(N), nkb = nkb_of(kp);
  const unsigned wblk = (unsigned)npad * 128u;  // bytes of one 64-wide column block of W
  unsigned char* Ws = usm;
  unsigned char* As = usm + (size_t)nkb * wblk;
  float* bias_s = reinterpret_cast<float*>(As + (size_t)STAGES * A_STAGE);
  unsigned long long* full = reinterpret_cast<unsigned long long*>(bias_s + npad);
  unsigned long long* empty = full + STAGES;
  unsigned long long* tfull = empty + STAGES;
  unsigned long long* tempty = tfull + 2;
  unsigned long long* wbar = tempty + 2;
  unsigned* tslot = reinterpret_cast<unsigned*>(wbar + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = (M + BM - 1) / BM;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], EPI_WARPS);
    }
    mbar_init(wbar, 1);
    mbar_fence_init();
  }
  for (int c = threadIdx.x; c < npad; c += THREADS) bias_s[c] = c < N ? bias[c] : 0.f;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tslot;
  bool ok = true;

  if (warp == 0 && lane == 0) {
    // ---- producer: W once, then the K slices of every tile ----
    mbar_arrive_expect_tx(wbar, (unsigned)(nkb * wblk));
    for (int c = 0; c < nkb; ++c) tma_load_2d(Ws + (size_t)c * wblk, &wmap, c * BK, 0, wbar);
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int s = it % STAGES, u = it / STAGES;
        if (u > 0 && !mbar_wait(&empty[s], (unsigned)((u - 1) & 1), kWaitPolls)) {
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(&full[s], A_STAGE);
        tma_load_2d(As + (size_t)s * A_STAGE, &xmap, kb * BK, tile * BM, &full[s]);
      }
    }
    if (!ok) atomicExch(err, 1);
    // copies still in flight: the last STAGES slices issued
    for (int j = (it > STAGES ? it - STAGES : 0); j < it; ++j)
      (void)mbar_wait(&full[j % STAGES], (unsigned)((j / STAGES) & 1), kWaitPolls);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issue ----
    ok = mbar_wait(wbar, 0, kWaitPolls);
    const unsigned id = idesc_bf16(BM, npad);
    const int k16 = (kp + 15) / 16;  // K steps of 16
    int it = 0, t = 0;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++t) {
      const int b = t & 1, v = t >> 1;
      if (v > 0 && !mbar_wait(&tempty[b], (unsigned)((v - 1) & 1), kWaitPolls)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned acc_addr = tmem + (unsigned)(b * 256);
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int s = it % STAGES, u = it / STAGES;
        if (!mbar_wait(&full[s], (unsigned)(u & 1), kWaitPolls)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned a0 = smem_u32(As + (size_t)s * A_STAGE);
        const unsigned b0 = smem_u32(Ws + (size_t)kb * wblk);
        const int steps = min(BK / 16, k16 - kb * (BK / 16));
        for (int kk = 0; kk < steps; ++kk) {
          const unsigned long long ad = sdesc_sw128(a0 + (unsigned)kk * 32u);
          const unsigned long long bd = sdesc_sw128(b0 + (unsigned)kk * 32u);
          const unsigned acc = (kb > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc_addr),
              "l"(ad), "l"(bd), "r"(id), "r"(acc)
              : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&empty[s]))
                     : "memory");
      }
      if (!ok) break;
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&tfull[b]))
                   : "memory");
    }
    if (!ok) {
      atomicExch(err, 1);
      // MMAs issued before the failure: wait (bounded) for the last commit of each stage
      for (int j = (it > STAGES ? it - STAGES : 0); j < it; ++j)
        (void)mbar_wait(&empty[j % STAGES], (unsigned)((j / STAGES) & 1), kWaitPolls);
    }
  } else if (warp >= 2) {
    // ---- epilogue: two warps per lane quarter, each a contiguous half of
    // the columns, two 16-column accumulator loads in flight per wait ----
    const int q = warp & 3;               // lane quarter of tensor memory
    const int half = (warp - 2) >> 2;     // 0: columns [0, hcol), 1: [hcol, npad)
    const int hcol = (npad / 32) * 16 > 0 ? (npad / 32) * 16 : npad;
    const int cbeg = half ? hcol : 0, cend = half ? npad : hcol;
    const int r_in_tile = q * 32 + lane;  // accumulator row of this thread
    int t = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++t) {
      const int b = t & 1, v = t >> 1;
      if (!mbar_wait(&tfull[b], (unsigned)(v & 1), kWaitPolls)) {
        if (lane == 0) atomicExch(err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const long long row = (long long)tile * BM + r_in_tile;
      const unsigned taddr = tmem + ((unsigned)(q * 32) << 16) + (unsigned)(b * 256);
      for (int c0 = cbeg; c0 < cend; c0 += 32) {
        const bool two = c0 + 16 < cend;
        unsigned vv[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(vv[0]), "=r"(vv[1]), "=r"(vv[2]), "=r"(vv[3]), "=r"(vv[4]), "=r"(vv[5]), "=r"(vv[6]),
              "=r"(vv[7]), "=r"(vv[8]), "=r"(vv[9]), "=r"(vv[10]), "=r"(vv[11]), "=r"(vv[12]), "=r"(vv[13]),
              "=r"(vv[14]), "=r"(vv[15])
            : "r"(taddr + (unsigned)c0));
        if (two)
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(vv[16]), "=r"(vv[17]), "=r"(vv[18]), "=r"(vv[19]), "=r"(vv[20]), "=r"(vv[21]), "=r"(vv[22]),
                "=r"(vv[23]), "=r"(vv[24]), "=r"(vv[25]), "=r"(vv[26]), "=r"(vv[27]), "=r"(vv[28]), "=r"(vv[29]),
                "=r"(vv[30]), "=r"(vv[31])
              : "r"(taddr + (unsigned)(c0 + 16)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row < M) {
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            if (h2 == 1 && !two) break;
            const int cc = c0 + 16 * h2;
            float x[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              x[j] = __uint_as_float(vv[16 * h2 + j]) + bias_s[cc + j];
              if (RELU) x[j] = fmaxf(x[j], 0.f);
            }
            const int ncol = min(16, ldo - cc);  // columns of the output row in this chunk
            if (OUT_BF16) {
              __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(out) + (size_t)row * ldo + cc;
              if (ncol == 16) {
                unsigned w[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
                  w[j] = *reinterpret_cast<const unsigned*>(&h);
                }
                reinterpret_cast<uint4*>(o)[0] = make_uint4(w[0], w[1], w[2], w[3]);
                reinterpret_cast<uint4*>(o)[1] = make_uint4(w[4], w[5], w[6], w[7]);
              } else {
                for (int j = 0; j < ncol; ++j) o[j] = __float2bfloat16_rn(x[j]);
              }
            } else {
              float* o = reinterpret_cast<float*>(out) + (size_t)row * ldo + cc;
              if (ncol == 16 && (ldo % 4) == 0) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                  reinterpret_cast<float4*>(o)[j] = make_float4(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3]);
              } else {
                for (int j = 0; j < ncol; ++j) o[j] = x[j];
              }
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[b])) : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

}  // namespace umws
}  // namespace frk
