// Blocked Gauss-Jordan inversion of one element block (the element-Jacobi
// preconditioner of Sec. 4.5) with the trailing updates on the 5th-generation
// tensor cores.  Used for the reduced-precision blocks (FP32 arithmetic).
//
// In-place Gauss-Jordan with partial pivoting, in panels of BW = 16 columns:
//  * panel factorisation: for each column c of the panel, the pivot row r is
//    the unused row of largest |M[r][c]| (rows are not swapped: pr[c] = r is
//    recorded instead), and the elimination is applied to the panel's
//    columns only (all rows);
//  * the b pivots of a panel act on every other column x as x <- x + U x_P,
//    with x_P the pivot rows' entries of x before the panel and
//    U = (panel columns after the panel) - (unit vectors of the pivot rows):
//    a rank-b update M[:, R] += U X, X = M[pivot rows, R], which is one
//    128 x N x 16 product on the tensor cores (tcgen05.mma kind::tf32,
//    FP32 accumulation in tensor memory);
//  * the result is the inverse with rows and columns permuted:
//    inverse(a, b) = M[pr[a]][ipr[b]], ipr the inverse permutation of pr.
// FP32 accuracy from TF32 operands: every operand is split as x ~ hi + lo,
// hi = x rounded to the nearest TF32 value (10 fraction bits) and lo = the
// difference x - hi (exact in FP32) rounded to TF32 as well, so hi + lo
// carries about 22 bits of x; then U X ~ U_hi X_hi + U_hi X_lo + U_lo X_hi
// (three MMAs per K step), a relative error of about 2^-23 per product.
//
// Operands are K-major without swizzle: 8-row x 16-byte core matrices (four
// TF32 values of K), the two core matrices of one K = 8 step 128 bytes apart,
// 8-row groups 512 bytes apart.  A (U) has 128 rows (zero beyond the block),
// B (X^T) has N = NB rounded up to 16 rows (zero beyond the block).  The
// accumulator occupies lanes 0..127 (row i in lane i) and N columns of tensor
// memory; warp w reads lanes 32 (w % 4) ... with tcgen05.ld.
#pragma once

#include "device.cuh"

namespace frk {
namespace gjtc {

constexpr int BW = 16;      // panel width: two K = 8 steps of kind::tf32
constexpr int MROWS = 128;  // MMA M
constexpr unsigned SBO = (BW / 4) * 128;  // bytes between 8-row groups

template <int NB>
struct Shape {
  static constexpr int N = (NB + 15) / 16 * 16;  // MMA N (multiple of 16 for M = 128)
  static constexpr unsigned A_BYTES = MROWS * BW * 4;
  static constexpr unsigned B_BYTES = N * BW * 4;
  static constexpr unsigned OPS = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr unsigned TMEM_COLS = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
  // scratch after the operands: barrier (8), tensor-memory slot (4), pivot
  // row (4), inverse permutation (4 NB), panel pivot rows (4 BW), scaled
  // pivot row (4 BW), used-row flags (NB)
  static constexpr unsigned OFF_BAR = OPS;
  static constexpr unsigned OFF_SLOT = OFF_BAR + 8;
  static constexpr unsigned OFF_PROW = OFF_SLOT + 4;
  static constexpr unsigned OFF_IPR = OFF_PROW + 4;
  static constexpr unsigned OFF_ROWS = OFF_IPR + 4 * NB;
  static constexpr unsigned OFF_SROW = OFF_ROWS + 4 * BW;
  static constexpr unsigned OFF_USED = OFF_SROW + 4 * BW;
  static constexpr unsigned BYTES = (OFF_USED + NB + 127) / 128 * 128;
};

// blocks whose inversion runs on the tensor cores (one MMA covers <= 128 rows)
template <typename T, int NB>
struct Use {
  static constexpr bool value = std::is_same<T, float>::value && NB <= MROWS;
};

__device__ __forceinline__ unsigned op_off(int row, int k) {
  return (unsigned)(row >> 3) * SBO + (unsigned)(k >> 2) * 128u + (unsigned)(row & 7) * 16u + (unsigned)(k & 3) * 4u;
}

// nearest TF32 value (ties away from zero in magnitude); the tensor cores
// read only these bits of a 32-bit operand
__device__ __forceinline__ float round_tf32(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
// x ~ hi + lo, both TF32 values
__device__ __forceinline__ void split_tf32(float x, float* hi, float* lo) {
  const float h = round_tf32(x);
  *hi = h;
  *lo = round_tf32(x - h);
}

// shared-memory matrix descriptor, no swizzle, K-major
__device__ __forceinline__ unsigned long long sdesc(unsigned saddr, unsigned lbo, unsigned sbo) {
  unsigned long long d = 0;
  d |= (unsigned long long)((saddr >> 4) & 0x3FFFu);
  d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;  // descriptor version
  return d;
}
// instruction descriptor: FP32 accumulate, TF32 A and B, both K-major, M x N
__host__ __device__ constexpr unsigned idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(unsigned tmem, unsigned long long ad, unsigned long long bd, unsigned id,
                                         unsigned acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(id), "r"(acc)
      : "memory");
}

// Invert the NB x NB FP32 matrix M (row stride LD, shared memory) in place
// into the permuted form described above; pr receives the pivot rows and
// scratch (Shape<NB>::BYTES, 128-byte aligned) holds the operands and
// bookkeeping, with ipr at scratch + OFF_IPR.  col: NB floats.  Whole CTA,
// blockDim.x a multiple of 128.  Returns false (on every thread) if a
// tensor-core wait gave up; the tensor memory is freed in every case.
template <int NB, int LD>
__device__ bool invert(float* M, float* col, int* pr, unsigned char* scratch) {
  using Sh = Shape<NB>;
  static_assert(NB <= MROWS, "one MMA covers at most 128 rows");
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nthr = blockDim.x;
  unsigned char* Ahi = scratch;
  unsigned char* Alo = scratch + Sh::A_BYTES;
  unsigned char* Bhi = scratch + 2 * Sh::A_BYTES;
  unsigned char* Blo = Bhi + Sh::B_BYTES;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(scratch + Sh::OFF_BAR);
  unsigned* tslot = reinterpret_cast<unsigned*>(scratch + Sh::OFF_SLOT);
  int* s_prow = reinterpret_cast<int*>(scratch + Sh::OFF_PROW);
  int* ipr = reinterpret_cast<int*>(scratch + Sh::OFF_IPR);
  int* rows = reinterpret_cast<int*>(scratch + Sh::OFF_ROWS);
  float* srow = reinterpret_cast<float*>(scratch + Sh::OFF_SROW);
  unsigned char* used = scratch + Sh::OFF_USED;

  for (int i = tid; i < (int)(Sh::OPS / 16); i += nthr) reinterpret_cast<uint4*>(scratch)[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < NB; i += nthr) used[i] = 0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(Sh::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tslot;
  constexpr unsigned id = idesc_tf32(MROWS, Sh::N);

  bool ok = true;
  int step = 0;
  for (int c0 = 0; c0 < NB; c0 += BW, ++step) {
    const int kb = min(BW, NB - c0);
    // ---- panel factorisation: kb pivots on the panel's columns ----
    for (int k = 0; k < kb; ++k) {
      const int c = c0 + k;
      for (int i = tid; i < NB; i += nthr) col[i] = M[i * LD + c];
      __syncthreads();
      if (warp == 0) {
        float best = -1.f;  // |pivot| (NaN ranks above everything)
        int bi = NB;
        for (int r = lane; r < NB; r += 32) {
          if (used[r]) continue;
          float v = fabsf(col[r]);
          if (v != v) v = __int_as_float(0x7f800000);
          if (v > best) { best = v; bi = r; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float ob = __shfl_down_sync(0xffffffffu, best, o);
          const int oi = __shfl_down_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        bi = __shfl_sync(0xffffffffu, bi, 0);
        const float ip = 1.f / col[bi];
        if (lane < kb) srow[lane] = (lane == k ? 1.f : M[bi * LD + c0 + lane]) * ip;
        if (lane == 0) {
          *s_prow = bi;
          used[bi] = 1;
          pr[c] = bi;
          ipr[bi] = c;
          rows[k] = bi;
        }
      }
      __syncthreads();
      const int r = *s_prow;
      for (int idx = tid; idx < NB * kb; idx += nthr) {
        const int i = idx / kb, t = idx - i * kb;
        float* m = M + i * LD + c0 + t;
        *m = i == r ? srow[t] : (t == k ? 0.f : *m) - col[i] * srow[t];
      }
      __syncthreads();
    }
    // ---- operands: A = U (rows i, K index k), B = X^T (rows j, K index k) ----
    for (int idx = tid; idx < NB * BW; idx += nthr) {
      const int i = idx / BW, k = idx - i * BW;
      float u = 0.f;
      if (k < kb) u = M[i * LD + c0 + k] - (i == rows[k] ? 1.f : 0.f);
      float hi, lo;
      split_tf32(u, &hi, &lo);
      const unsigned o = op_off(i, k);
      *reinterpret_cast<float*>(Ahi + o) = hi;
      *reinterpret_cast<float*>(Alo + o) = lo;
    }
    for (int idx = tid; idx < BW * NB; idx += nthr) {
      const int k = idx / NB, j = idx - k * NB;
      float x = 0.f;
      if (k < kb && (j < c0 || j >= c0 + kb)) x = M[rows[k] * LD + j];
      float hi, lo;
      split_tf32(x, &hi, &lo);
      const unsigned o = op_off(j, k);
      *reinterpret_cast<float*>(Bhi + o) = hi;
      *reinterpret_cast<float*>(Blo + o) = lo;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll
      for (int kk = 0; kk < BW / 8; ++kk) {
        const unsigned ko = (unsigned)kk * 256u;
        mma_tf32(tmem, sdesc(ah + ko, 128, SBO), sdesc(bh + ko, 128, SBO), id, kk > 0 ? 1u : 0u);
        mma_tf32(tmem, sdesc(ah + ko, 128, SBO), sdesc(bl + ko, 128, SBO), id, 1u);
        mma_tf32(tmem, sdesc(al + ko, 128, SBO), sdesc(bh + ko, 128, SBO), id, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(bar))
                   : "memory");
    }
    ok = mbar_wait(bar, (unsigned)(step & 1), kWaitPolls);
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- M[:, j] += (U X)[:, j] outside the panel ----
    {
      const int q = warp & 3, i = q * 32 + lane;
      for (int ch = warp >> 2; ch < Sh::N / 16; ch += nthr >> 7) {
        unsigned v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(tmem + ((unsigned)(q * 32) << 16) + (unsigned)(ch * 16)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (i < NB) {
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const int j = ch * 16 + t;
            if (j < NB && (j < c0 || j >= c0 + kb)) M[i * LD + j] += __uint_as_float(v[t]);
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  // a wait that gave up: give the MMAs one more bounded wait before the
  // tensor memory they write is released
  if (!ok) (void)mbar_wait(bar, (unsigned)(step & 1), kWaitPolls);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Sh::TMEM_COLS) : "memory");
  return ok;
}

}  // namespace gjtc
}  // namespace frk
