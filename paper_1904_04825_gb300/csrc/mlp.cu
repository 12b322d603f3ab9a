// Per-element MLP that predicts a stage solve's initial Krylov guess (not in
// the paper; the GMRES solve still tests the guess and converges to the
// same tolerance).
//
// Network 3nb -> 256 -> 256 -> nb, ReLU, FP32 master weights.
//  * training path (forward with stored activations, backward, Adam): FP32
//    tiled GEMMs on the CUDA cores, so the gradients can be checked against
//    the FP64 oracle;
//  * inference path: BF16 operands on the 5th-generation tensor cores
//    (tcgen05.mma, FP32 accumulator in tensor memory) with bias + ReLU fused
//    into the epilogue that reads the accumulator back.
// Loss: mean of (y - t)^2 / 2 over all outputs; Adam with bias correction.
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstring>
#include <new>

#include "device.cuh"
#include "umma_ws.cuh"

struct fr_mlp {
  int n[4] = {0, 0, 0, 0};  // layer widths: in, hidden, hidden, out
  int max_batch = 0;
  long long nparam = 0;
  float* P = nullptr;       // FP32 master parameters [W1 b1 W2 b2 W3 b3]
  float* G = nullptr;       // gradients (same layout)
  float* Mo = nullptr;      // Adam first moments
  float* Vo = nullptr;      // Adam second moments
  float* Z[3] = {};         // pre-activations [M x n[l+1]]
  float* A[2] = {};         // hidden activations [M x n[l+1]]
  float* D[3] = {};         // loss gradients w.r.t. Z
  float* part = nullptr;    // split-M partial weight gradients
  __nv_bfloat16* X16 = nullptr;   // BF16 input / hidden activations for inference,
  __nv_bfloat16* H16[2] = {};     //   rows padded to kp[l] (16-byte rows, zero pad)
  __nv_bfloat16* W16[3] = {};     // BF16 weights [n[l+1]][kp[l]], zero-padded columns
  int kp[3] = {0, 0, 0};          // padded widths of the layer inputs
  int* derr = nullptr;            // device flag: a bounded wait of the GEMM gave up
  // TMA tensor maps of the inference operands (input rows, hidden rows, weights)
  // for the weight-stationary GEMM; ws = 1 when every layer's weights fit in
  // shared memory and the maps were built
  CUtensorMap amap[3] = {};       // layer l input: X16 (l = 0), H16[l-1]
  CUtensorMap wmap[3] = {};
  int ws = 0;
  int* herr = nullptr;            // pinned host copy, refreshed after every inference
  double* loss = nullptr;   // device scalar
  int step = 0;
  char err[256] = {0};
};

namespace frk {
namespace {

constexpr int kSplitRows = 4096;  // rows per partial in the weight-gradient reduction

long long off_W(const fr_mlp* m, int l) {
  long long o = 0;
  for (int i = 0; i < l; ++i) o += (long long)m->n[i + 1] * m->n[i] + m->n[i + 1];
  return o;
}
long long off_b(const fr_mlp* m, int l) { return off_W(m, l) + (long long)m->n[l + 1] * m->n[l]; }

// ---- FP32 tiled GEMM: C[i][j] = sum_k A(i,k) B(k,j) (+ bias[j]) (ReLU) ----
// A(i,k) = A[i*sai + k*sak], B(k,j) = B[k*sbk + j*sbj], C row-major ldc.
// 64x64 tile, 16-deep k slices, 256 threads x (4x4) outputs.
template <bool RELU>
__global__ void __launch_bounds__(256) k_sgemm(int M, int N, int K, const float* __restrict__ A,
                                               long long sai, long long sak, const float* __restrict__ B,
                                               long long sbk, long long sbj, float* __restrict__ C, int ldc,
                                               const float* __restrict__ bias, float* __restrict__ Zout,
                                               int kbeg, int kend) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  float acc[4][4] = {};
  if (kend < 0) kend = K;
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
    for (int t = threadIdx.x; t < 16 * 64; t += 256) {
      const int kk = t / 64, r = t % 64;
      const int i = i0 + r, k = k0 + kk, j = j0 + r;
      As[kk][r] = (i < M && k < kend) ? A[i * sai + k * sak] : 0.f;
      Bs[kk][r] = (j < N && k < kend) ? B[k * sbk + j * sbj] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[kk][ty + 16 * u];
        b[u] = Bs[kk][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
      if (i < M && j < N) {
        float c = acc[u][v] + (bias ? bias[j] : 0.f);
        if (Zout) Zout[(long long)i * ldc + j] = c;
        if (RELU) c = fmaxf(c, 0.f);
        C[(long long)i * ldc + j] = c;
      }
    }
}

// ---- BF16 tensor-core GEMM for inference: Y = act(X W^T + b) ----
// 5th-generation tensor cores: one thread issues tcgen05.mma (kind::f16,
// BF16 operands, FP32 accumulator in tensor memory), the CTA stages the
// operands in shared memory, and the epilogue reads the accumulator back
// with tcgen05.ld.
//  * CTA tile 128 rows x BN (<= 256) columns, 128 threads (4 warps);
//    K in 64-wide slices through a 2-stage shared-memory ring filled with
//    16-byte cp.async copies (zero-filled outside the matrices), so padded
//    rows/columns contribute exact zeros;
//  * operands K-major without swizzle: 8-row x 16-byte core matrices, the
//    two core matrices of one K=16 step 128 bytes apart (leading byte
//    offset), consecutive 8-row groups 1024 bytes apart (stride byte offset);
//  * one MMA group per slice is committed to that stage's mbarrier; a stage
//    is refilled only after its MMAs completed; every wait is bounded and a
//    wait that gives up sets *err, and the tensor memory is always freed.
// X [M][kp] and W [N][kp] row-major BF16 with kp % 8 == 0 (16-byte rows).
namespace umma {
constexpr int BM = 128, BK = 64, STAGES = 2, MAXN = 256;
constexpr unsigned A_BYTES = BM * BK * 2;        // 16 KB
constexpr unsigned B_BYTES = MAXN * BK * 2;      // 32 KB
constexpr unsigned STAGE_BYTES = A_BYTES + B_BYTES;
constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 64;
constexpr unsigned TMEM_COLS = 256;

// shared-memory matrix descriptor, no swizzle, K-major
__device__ __forceinline__ unsigned long long sdesc(unsigned saddr, unsigned lbo, unsigned sbo) {
  unsigned long long d = 0;
  d |= (unsigned long long)((saddr >> 4) & 0x3FFFu);
  d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;  // descriptor version (fixed 0b001 at bits 46-48)
  return d;         // base offset 0, absolute-offset mode off, layout 0 = no swizzle
}
// instruction descriptor: FP32 accumulate, BF16 A and B, both K-major, M x N
__host__ __device__ constexpr unsigned idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(m >> 4) << 24);
}
__device__ __forceinline__ void cp16(unsigned dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}
}  // namespace umma

template <bool RELU, bool OUT_BF16>
__global__ void __launch_bounds__(128) k_umma_gemm(int M, int N, int kp, const __nv_bfloat16* __restrict__ X,
                                                   const __nv_bfloat16* __restrict__ W,
                                                   const float* __restrict__ bias, void* out, int ldo,
                                                   int* err) {
  using namespace umma;
  extern __shared__ __align__(1024) unsigned char usm[];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(usm + STAGES * STAGE_BYTES);
  unsigned* tslot = reinterpret_cast<unsigned*>(usm + STAGES * STAGE_BYTES + 32);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * MAXN;
  const int ncol = min(MAXN, N - n0);           // output columns of this tile
  const int bn = (ncol + 15) / 16 * 16;         // MMA N (multiple of 16)
  const int nk = (kp + BK - 1) / BK;
  const unsigned sbase = smem_u32(usm);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int q = 0; q < STAGES; ++q) mbar_init(&bar[q], 1);
    mbar_fence_init();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tslot;

  // fill stage st with K slice kt: A rows m0.., B rows n0.. (16-byte chunks)
  auto load = [&](int kt, int st) {
    const unsigned a_s = sbase + st * STAGE_BYTES, b_s = a_s + A_BYTES;
    const int k0 = kt * BK;
    for (int c = tid; c < BM * (BK / 8); c += 128) {
      const int row = c / (BK / 8), kc = c % (BK / 8);
      const int gi = m0 + row, gk = k0 + kc * 8;
      const bool ok = gi < M && gk < kp;
      cp16(a_s + (row / 8) * 1024 + kc * 128 + (row % 8) * 16, ok ? (const void*)(X + (size_t)gi * kp + gk) : (const void*)X, ok);
    }
    for (int c = tid; c < bn * (BK / 8); c += 128) {
      const int row = c / (BK / 8), kc = c % (BK / 8);
      const int gj = n0 + row, gk = k0 + kc * 8;
      const bool ok = gj < N && gk < kp;
      cp16(b_s + (row / 8) * 1024 + kc * 128 + (row % 8) * 16, ok ? (const void*)(W + (size_t)gj * kp + gk) : (const void*)W, ok);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  bool ok = true;
  load(0, 0);
  for (int kt = 0; kt < nk && ok; ++kt) {
    const int st = kt % STAGES;
    if (kt + 1 < nk) {
      const int nst = (kt + 1) % STAGES;
      if (kt + 1 >= STAGES) {  // MMAs of slice kt+1-STAGES must be done with stage nst
        const int u = (kt + 1 - STAGES) / STAGES;
        ok = mbar_wait(&bar[nst], (unsigned)(u & 1), kWaitPolls);
      }
      if (!__syncthreads_and(ok)) break;
      load(kt + 1, nst);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    // generic-proxy writes -> visible to the tensor cores' async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned a_s = sbase + st * STAGE_BYTES, b_s = a_s + A_BYTES;
      const unsigned id = idesc_bf16(BM, bn);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const unsigned long long ad = sdesc(a_s + kk * 256, 128, 1024);
        const unsigned long long bd = sdesc(b_s + kk * 256, 128, 1024);
        const unsigned acc = (kt > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(id), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&bar[st]))
                   : "memory");
    }
  }
  // all MMAs done: the last commit tracks every MMA issued before it
  if (ok && nk > 0) {
    const int last = nk - 1;
    ok = mbar_wait(&bar[last % STAGES], (unsigned)((last / STAGES) & 1), kWaitPolls);
  }
  ok = __syncthreads_and(ok);
  if (!ok) {
    asm volatile("cp.async.wait_all;" ::: "memory");  // no copy may land after the CTA leaves
    if (tid == 0) atomicExch(err, 1);
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // Accumulator -> bias, activation, output type -> a row-major tile of 64
    // rows in the (now idle) stage buffers, then coalesced 16-byte row
    // stores; two passes (warps 0-1, then warps 2-3) keep the staged tile
    // within the stage buffers for FP32 output too.
    using OutT = typename std::conditional<OUT_BF16, __nv_bfloat16, float>::type;
    constexpr int ES = (int)sizeof(OutT);
    const int pitch = bn * ES + 16;  // bytes per staged row (+16 spreads the banks)
    unsigned char* tile = usm;
    const int wcols = min(bn, ldo - n0);  // output columns of this tile
    const bool vec = ((ldo * ES) % 16 == 0) && ((wcols * ES) % 16 == 0);
    for (int pass = 0; pass < 2; ++pass) {
      if ((warp >> 1) == pass) {
        const int lrow = (warp & 1) * 32 + lane;  // row within the pass
        for (int c0 = 0; c0 < bn; c0 += 16) {
          unsigned v[16];
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          float x[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int j = n0 + c0 + q;
            x[q] = __uint_as_float(v[q]) + (j < N ? bias[j] : 0.f);
            if (RELU) x[q] = fmaxf(x[q], 0.f);
          }
          uint4* dst = reinterpret_cast<uint4*>(tile + (size_t)lrow * pitch + (size_t)c0 * ES);
          if (OUT_BF16) {
            unsigned w[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
              w[q] = *reinterpret_cast<const unsigned*>(&h);
            }
            dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
            dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
              dst[q] = make_uint4(__float_as_uint(x[4 * q]), __float_as_uint(x[4 * q + 1]), __float_as_uint(x[4 * q + 2]),
                                  __float_as_uint(x[4 * q + 3]));
          }
        }
      }
      __syncthreads();
      const int r0 = m0 + pass * 64;
      const int rows = max(0, min(64, M - r0));
      if (vec) {
        const int cpr = wcols * ES / 16;  // 16-byte chunks per row
        for (int c = tid; c < rows * cpr; c += 128) {
          const int r = c / cpr, k = c % cpr;
          const uint4 val = *reinterpret_cast<const uint4*>(tile + (size_t)r * pitch + k * 16);
          *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(out) + ((size_t)(r0 + r) * ldo + n0) * ES +
                                    k * 16) = val;
        }
      } else {
        for (int c = tid; c < rows * wcols; c += 128) {
          const int r = c / wcols, k = c % wcols;
          reinterpret_cast<OutT*>(out)[(size_t)(r0 + r) * ldo + n0 + k] =
              reinterpret_cast<const OutT*>(tile + (size_t)r * pitch)[k];
        }
      }
      __syncthreads();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// x [M][k] FP32 -> y [M][kp] BF16, zero in the padding columns
__global__ void k_f2bf_pad(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, long long M, int k, int kp) {
  const long long n = M * kp;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long i = t / kp;
    const int j = (int)(t % kp);
    y[t] = j < k ? __float2bfloat16_rn(x[i * k + j]) : __float2bfloat16_rn(0.f);
  }
}


// dZ_out = (y - t) / (M * n_out), loss partial sums (FP64)
__global__ void k_loss_grad(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ d,
                            long long n, double* loss, Reduce red) {
  __shared__ double sh[32];
  double s = 0.0;
  const float inv = 1.0f / (float)n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float e = y[i] - t[i];
    d[i] = e * inv;
    s += 0.5 * (double)e * (double)e;
  }
  const double bs = block_sum(s, sh);
  if (threadIdx.x == 0) red.partials[(size_t)blockIdx.x * kMaxVec] = bs;
  if (last_block(red.counter)) {
    finish_sums(red, 1, loss);
    if (threadIdx.x == 0) *loss /= (double)n;
  }
}

// d = d * (z > 0)
__global__ void k_relu_back(float* __restrict__ d, const float* __restrict__ z, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (!(z[i] > 0.f)) d[i] = 0.f;
}

// sum of the split-M partials (fixed order) into the weight gradient; bias
// gradient = column sums of dZ (fixed order)
__global__ void k_sum_parts(const float* __restrict__ part, int nparts, long long n, float* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int p = 0; p < nparts; ++p) s += part[(long long)p * n + i];
    out[i] = s;
  }
}

__global__ void k_colsum(const float* __restrict__ d, int M, int N, float* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.f;
  for (int i = 0; i < M; ++i) s += d[(long long)i * N + j];
  out[j] = s;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

int mlp_err(fr_mlp* m, int code, const char* msg) {
  if (m) {
    std::strncpy(m->err, msg, sizeof(m->err) - 1);
    m->err[sizeof(m->err) - 1] = 0;
  }
  return code;
}

#define MLP_CUDA(m, call)                                                  \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) return mlp_err((m), FR_ERR_CUDA, cudaGetErrorString(e_)); \
  } while (0)

unsigned grid_for(long long n) {
  long long g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  return (unsigned)(g < 1 ? 1 : g);
}

// BF16 copies of the weights with rows padded to 16 bytes (biases stay FP32)
int refresh_bf16(fr_mlp* m, cudaStream_t s) {
  for (int l = 0; l < 3; ++l) {
    const long long n = (long long)m->n[l + 1] * m->kp[l];
    count_launch();
    k_f2bf_pad<<<grid_for(n), 256, 0, s>>>(m->P + off_W(m, l), m->W16[l], m->n[l + 1], m->n[l], m->kp[l]);
  }
  MLP_CUDA(m, cudaGetLastError());
  return FR_OK;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2D BF16 row-major [rows][ld] (cols <= ld valid), boxes of 64 columns x box_rows
// rows, 128-byte swizzle, zero fill outside
bool make_map(CUtensorMap* map, const void* base, long long rows, int cols, int ld, int box_rows) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)umws::BK, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// tensor maps of the weight-stationary inference (all three layers, or none)
void build_maps(fr_mlp* m) {
  m->ws = 0;
  for (int l = 0; l < 3; ++l)
    if (!umws::fits(m->n[l + 1], m->kp[l])) return;
  for (int l = 0; l < 3; ++l) {
    const void* in = l == 0 ? (const void*)m->X16 : (const void*)m->H16[l - 1];
    if (!make_map(&m->amap[l], in, m->max_batch, m->kp[l], m->kp[l], umws::BM)) return;
    if (!make_map(&m->wmap[l], m->W16[l], m->n[l + 1], m->kp[l], m->kp[l], umws::npad_of(m->n[l + 1]))) return;
  }
  m->ws = 1;
}

void free_mlp(fr_mlp* m) {
  if (!m) return;
  cudaFree(m->P); cudaFree(m->G); cudaFree(m->Mo); cudaFree(m->Vo);
  for (auto* p : m->W16) cudaFree(p);
  cudaFree(m->derr);
  cudaFreeHost(m->herr);
  for (auto* p : m->Z) cudaFree(p);
  for (auto* p : m->A) cudaFree(p);
  for (auto* p : m->D) cudaFree(p);
  cudaFree(m->part); cudaFree(m->X16);
  for (auto* p : m->H16) cudaFree(p);
  cudaFree(m->loss);
  delete m;
}

// Reduction scratch for the loss (own copy, independent of any fr_ctx).
struct MlpRed {
  double* partials = nullptr;
  unsigned* counter = nullptr;
};
MlpRed g_mlp_red[64];

}  // namespace
}  // namespace frk

using namespace frk;

extern "C" int fr_mlp_create(int n_in, int n_hidden, int n_out, int max_batch, fr_mlp** out) {
  if (!out) return FR_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_in < 1 || n_hidden < 1 || n_out < 1 || max_batch < 1) return FR_ERR_INVALID_ARG;
  fr_mlp* m = new (std::nothrow) fr_mlp();
  if (!m) return FR_ERR_CUDA;
  m->n[0] = n_in; m->n[1] = n_hidden; m->n[2] = n_hidden; m->n[3] = n_out;
  m->max_batch = max_batch;
  m->nparam = off_b(m, 2) + n_out;
  auto fail = [&](cudaError_t e) { free_mlp(m); return e == cudaSuccess ? FR_OK : FR_ERR_CUDA; };
  cudaError_t e = cudaSuccess;
  const size_t np = (size_t)m->nparam;
  if (e == cudaSuccess) e = cudaMalloc(&m->P, np * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->G, np * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->Mo, np * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->Vo, np * sizeof(float));
  for (int l = 0; l < 3; ++l) m->kp[l] = (m->n[l] + 7) / 8 * 8;
  for (int l = 0; l < 3 && e == cudaSuccess; ++l)
    e = cudaMalloc(&m->W16[l], (size_t)m->n[l + 1] * m->kp[l] * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&m->derr, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(m->derr, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&m->herr, sizeof(int));
  if (e == cudaSuccess) *m->herr = 0;
  for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
    e = cudaMalloc(&m->Z[l], (size_t)max_batch * m->n[l + 1] * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->D[l], (size_t)max_batch * m->n[l + 1] * sizeof(float));
  }
  for (int l = 0; l < 2 && e == cudaSuccess; ++l) {
    e = cudaMalloc(&m->A[l], (size_t)max_batch * m->n[l + 1] * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->H16[l], (size_t)max_batch * m->kp[l + 1] * sizeof(__nv_bfloat16));
  }
  const int nparts = (max_batch + kSplitRows - 1) / kSplitRows;
  long long maxw = 0;
  for (int l = 0; l < 3; ++l) maxw = std::max(maxw, (long long)m->n[l + 1] * m->n[l]);
  if (e == cudaSuccess) e = cudaMalloc(&m->part, (size_t)nparts * maxw * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->X16, (size_t)max_batch * m->kp[0] * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&m->loss, sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(m->Mo, 0, np * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->Vo, 0, np * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->P, 0, np * sizeof(float));
  int dev = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess && dev >= 0 && dev < 64 && !g_mlp_red[dev].partials) {
    e = cudaMalloc(&g_mlp_red[dev].partials, (size_t)kRedBlocks * kMaxVec * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&g_mlp_red[dev].counter, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(g_mlp_red[dev].counter, 0, sizeof(unsigned));
  }
  if (e != cudaSuccess) return fail(e);
  build_maps(m);
  *out = m;
  return FR_OK;
}

extern "C" int fr_mlp_destroy(fr_mlp* m) {
  free_mlp(m);
  return FR_OK;
}

extern "C" const char* fr_mlp_last_error(const fr_mlp* m) { return m ? m->err : "invalid model"; }

extern "C" long long fr_mlp_num_params(const fr_mlp* m) { return m ? m->nparam : 0; }

extern "C" int fr_mlp_set_params(fr_mlp* m, const float* host, void* stream) {
  if (!m || !host) return FR_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  MLP_CUDA(m, cudaMemcpyAsync(m->P, host, m->nparam * sizeof(float), cudaMemcpyHostToDevice, s));
  MLP_CUDA(m, cudaMemsetAsync(m->Mo, 0, m->nparam * sizeof(float), s));
  MLP_CUDA(m, cudaMemsetAsync(m->Vo, 0, m->nparam * sizeof(float), s));
  m->step = 0;
  FRK_TRY(refresh_bf16(m, s));
  MLP_CUDA(m, cudaStreamSynchronize(s));
  return FR_OK;
}

extern "C" int fr_mlp_get_params(fr_mlp* m, float* host, void* stream) {
  if (!m || !host) return FR_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  MLP_CUDA(m, cudaMemcpyAsync(host, m->P, m->nparam * sizeof(float), cudaMemcpyDeviceToHost, s));
  MLP_CUDA(m, cudaStreamSynchronize(s));
  return FR_OK;
}

extern "C" int fr_mlp_get_grads(fr_mlp* m, float* host, void* stream) {
  if (!m || !host) return FR_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  MLP_CUDA(m, cudaMemcpyAsync(host, m->G, m->nparam * sizeof(float), cudaMemcpyDeviceToHost, s));
  MLP_CUDA(m, cudaStreamSynchronize(s));
  return FR_OK;
}

extern "C" int fr_mlp_forward(fr_mlp* m, const float* X, int M, float* Y, int bf16, void* stream) {
  if (!m || !X || !Y || M < 1 || M > m->max_batch) return mlp_err(m, FR_ERR_INVALID_ARG, "bad forward arguments");
  if (*m->herr) return mlp_err(m, FR_ERR_TIMEOUT, "an earlier tensor-core GEMM gave up a bounded wait");
  cudaStream_t s = as_stream(stream);
  if (!bf16) {
    const float* in = X;
    for (int l = 0; l < 3; ++l) {
      const int K = m->n[l], N = m->n[l + 1];
      const dim3 grid((N + 63) / 64, (M + 63) / 64);
      float* C = l < 2 ? m->A[l] : Y;
      count_launch();
      if (l < 2)
        k_sgemm<true><<<grid, 256, 0, s>>>(M, N, K, in, K, 1, m->P + off_W(m, l), 1, K, C, N,
                                           m->P + off_b(m, l), m->Z[l], 0, -1);
      else
        k_sgemm<false><<<grid, 256, 0, s>>>(M, N, K, in, K, 1, m->P + off_W(m, l), 1, K, C, N,
                                            m->P + off_b(m, l), m->Z[l], 0, -1);
      in = C;
    }
  } else {
    static bool attr = false;  // dynamic shared memory above 48 KB, set once per process
    if (!attr) {
      MLP_CUDA(m, cudaFuncSetAttribute(k_umma_gemm<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)umma::SMEM));
      MLP_CUDA(m, cudaFuncSetAttribute(k_umma_gemm<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)umma::SMEM));
      attr = true;
    }
    count_launch();
    k_f2bf_pad<<<grid_for((long long)M * m->kp[0]), 256, 0, s>>>(X, m->X16, M, m->n[0], m->kp[0]);
    if (m->ws) {
      // weight-stationary persistent GEMMs: one CTA per SM (at most one per 128-row tile)
      static int sms = 0;
      if (sms == 0) {
        int dev = 0;
        MLP_CUDA(m, cudaGetDevice(&dev));
        MLP_CUDA(m, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        MLP_CUDA(m, cudaFuncSetAttribute(umws::k_umma_ws<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)umws::kSmemLimit));
        MLP_CUDA(m, cudaFuncSetAttribute(umws::k_umma_ws<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)umws::kSmemLimit));
      }
      const int tiles = (M + umws::BM - 1) / umws::BM;
      const unsigned grid = (unsigned)std::min(tiles, sms);
      for (int l = 0; l < 3; ++l) {
        const int N = m->n[l + 1];
        const size_t smem = umws::smem_bytes(N, m->kp[l]);
        count_launch();
        if (l < 2)
          umws::k_umma_ws<true, true><<<grid, umws::THREADS, smem, s>>>(m->amap[l], m->wmap[l], M, N, m->kp[l],
                                                                        m->P + off_b(m, l), m->H16[l], m->kp[l + 1],
                                                                        m->derr);
        else
          umws::k_umma_ws<false, false><<<grid, umws::THREADS, smem, s>>>(m->amap[l], m->wmap[l], M, N, m->kp[l],
                                                                          m->P + off_b(m, l), Y, N, m->derr);
      }
      MLP_CUDA(m, cudaGetLastError());
      MLP_CUDA(m, cudaMemcpyAsync(m->herr, m->derr, sizeof(int), cudaMemcpyDeviceToHost, s));
      return FR_OK;
    }
    const __nv_bfloat16* in = m->X16;
    for (int l = 0; l < 3; ++l) {
      const int N = m->n[l + 1];
      const dim3 grid((M + umma::BM - 1) / umma::BM, (N + umma::MAXN - 1) / umma::MAXN);
      count_launch();
      if (l < 2)
        k_umma_gemm<true, true><<<grid, 128, umma::SMEM, s>>>(M, N, m->kp[l], in, m->W16[l], m->P + off_b(m, l),
                                                              m->H16[l], m->kp[l + 1], m->derr);
      else
        k_umma_gemm<false, false><<<grid, 128, umma::SMEM, s>>>(M, N, m->kp[l], in, m->W16[l], m->P + off_b(m, l),
                                                                Y, N, m->derr);
      in = l < 2 ? m->H16[l] : nullptr;
    }
  }
  MLP_CUDA(m, cudaGetLastError());
  // the GEMMs' error flag reaches the host with the stream; the next call reports it
  if (bf16) MLP_CUDA(m, cudaMemcpyAsync(m->herr, m->derr, sizeof(int), cudaMemcpyDeviceToHost, s));
  return FR_OK;
}

extern "C" int fr_mlp_backward(fr_mlp* m, const float* X, const float* T, int M, double* loss_host,
                               void* stream) {
  if (!m || !X || !T || M < 1 || M > m->max_batch) return mlp_err(m, FR_ERR_INVALID_ARG, "bad backward arguments");
  cudaStream_t s = as_stream(stream);
  int dev = 0;
  MLP_CUDA(m, cudaGetDevice(&dev));
  Reduce red{g_mlp_red[dev].partials, g_mlp_red[dev].counter};
  const long long nout = (long long)M * m->n[3];
  // output: Y = Z[2] (forward_train stored it)
  count_launch();
  k_loss_grad<<<grid_for(nout) > 1024 ? 1024 : grid_for(nout), 256, 0, s>>>(m->Z[2], T, m->D[2], nout, m->loss, red);
  const int nparts = (M + kSplitRows - 1) / kSplitRows;
  for (int l = 2; l >= 0; --l) {
    const int K = m->n[l], N = m->n[l + 1];
    const float* in = l == 0 ? X : m->A[l - 1];
    // dW[N x K] = sum over rows of D[l]^T (rows) x in (rows): split by rows
    for (int p = 0; p < nparts; ++p) {
      const int r0 = p * kSplitRows, r1 = std::min(M, r0 + kSplitRows);
      const dim3 grid((K + 63) / 64, (N + 63) / 64);
      count_launch();
      // C[i=n][j=k] = sum_r D[r][n] in[r][k]; A(i,kr) = D[kr*N + i], B(kr,j) = in[kr*K + j]
      k_sgemm<false><<<grid, 256, 0, s>>>(N, K, r1, m->D[l], 1, N, in, K, 1,
                                          m->part + (long long)p * N * K, K, nullptr, nullptr, r0, r1);
    }
    count_launch();
    k_sum_parts<<<grid_for((long long)N * K), 256, 0, s>>>(m->part, nparts, (long long)N * K, m->G + off_W(m, l));
    count_launch();
    k_colsum<<<(N + 127) / 128, 128, 0, s>>>(m->D[l], M, N, m->G + off_b(m, l));
    if (l > 0) {
      // D[l-1] = (D[l] W_l) * relu'(Z[l-1]);  D[l] [M x N], W_l [N x K]
      const dim3 grid((K + 63) / 64, (M + 63) / 64);
      count_launch();
      k_sgemm<false><<<grid, 256, 0, s>>>(M, K, N, m->D[l], N, 1, m->P + off_W(m, l), K, 1, m->D[l - 1], K,
                                          nullptr, nullptr, 0, -1);
      count_launch();
      k_relu_back<<<grid_for((long long)M * K), 256, 0, s>>>(m->D[l - 1], m->Z[l - 1], (long long)M * K);
    }
  }
  MLP_CUDA(m, cudaGetLastError());
  if (loss_host) {
    MLP_CUDA(m, cudaMemcpyAsync(loss_host, m->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    MLP_CUDA(m, cudaStreamSynchronize(s));
  }
  return FR_OK;
}

extern "C" int fr_mlp_adam(fr_mlp* m, float lr, float beta1, float beta2, float eps, void* stream) {
  if (!m) return FR_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  m->step += 1;
  const float c1 = 1.f - std::pow(beta1, (float)m->step);
  const float c2 = 1.f - std::pow(beta2, (float)m->step);
  count_launch();
  k_adam<<<grid_for(m->nparam), 256, 0, s>>>(m->P, m->G, m->Mo, m->Vo, m->nparam, lr, beta1, beta2, eps, c1, c2);
  MLP_CUDA(m, cudaGetLastError());
  return refresh_bf16(m, s);
}
