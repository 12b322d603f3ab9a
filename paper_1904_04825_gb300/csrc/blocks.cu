// Element-Jacobi preconditioner (Sec. 4.5): form M_e = shift*I - dR_e/dq_e by
// element-local forward differences with the neighbour traces frozen, invert
// it in shared memory by Gauss-Jordan elimination with partial pivoting, and
// apply the inverse blocks as batched matrix-vector products.
//
// Block formation exploits the FR stencil inside one element: perturbing the
// state at point (a, b) changes the pointwise flux there, the x-face traces
// of row b and the y-face traces of column a, so only the residual on row b
// and column a changes.  Each thread forms one column from those changes
// (mathematically the same forward difference R_e(q + eps e_j) - R_e(q)
// over eps; entries outside the cross are exactly zero in both forms).
#include <cuda_bf16.h>

#include <type_traits>

#include "device.cuh"
#include "gj_cluster.cuh"
#include "gj_tc.cuh"

namespace frk {
namespace {

struct FactorArgs {
  const double* U;
  void* blocks;      // [ne][nb][nb] of S, column-major inverse per element: Minv[k*nb + i]
  double* mst;       // staged M = shift I - J_ee before inversion, [ne][c][row] (FP64)
  const double* hx;
  const double* hy;
  long long ne;
  int nx, ny;
  double gam;
  double shift;
  double beps;       // block_eps_rel
  int riemann;       // common flux: 0 Rusanov, 1 Roe
  int* err;          // set when a tensor-core wait gave up
  Tables tab;
};

template <int P, typename T>
struct FactorLayout {
  static constexpr int N = P + 1, NP = N * N, NB = 4 * NP, LD = NB + 1;
  static constexpr int THREADS = NB <= 64 ? 128 : 256;
  // shared memory: doubles first, then the block (type T), its pivot column and pivots
  static constexpr int OFF_Q = 0;                       // 4 x NP state
  static constexpr int OFF_F = OFF_Q + 4 * NP;          // 4 x NP  (hy/2) f
  static constexpr int OFF_G = OFF_F + 4 * NP;          // 4 x NP  (hx/2) g
  static constexpr int OFF_TR = OFF_G + 4 * NP;         // own traces [4 faces][4 vars][N]
  static constexpr int OFF_NT = OFF_TR + 16 * N;        // neighbour traces [4][4][N]
  static constexpr int OFF_FN = OFF_NT + 16 * N;        // base common fluxes [4][4][N] (scaled)
  static constexpr int DOUBLES = OFF_FN + 16 * N;
  static constexpr bool TC = gjtc::Use<T, NB>::value;  // inversion on the tensor cores
  // block, pivot column and pivots, then (TC) the tensor-core scratch, 128-byte aligned
  static constexpr size_t GJ_END = DOUBLES * sizeof(double) + (size_t)(NB * LD + NB) * sizeof(T) + NB * sizeof(int);
  static constexpr size_t OFF_TC = (GJ_END + 127) / 128 * 128;
  static constexpr size_t BYTES = TC ? OFF_TC + gjtc::Shape<NB>::BYTES : GJ_END + 64;
};

constexpr size_t kSmemMax = 227 * 1024;  // opt-in shared memory per CTA

template <typename S> struct StoreT;
template <> struct StoreT<double> { __device__ static double to(double x) { return x; } };
template <> struct StoreT<float> { __device__ static float to(float x) { return x; } };
template <> struct StoreT<__nv_bfloat16> {
  __device__ static __nv_bfloat16 to(float x) { return __float2bfloat16_rn(x); }
};
__device__ __forceinline__ double load_acc(const double* p) { return *p; }
__device__ __forceinline__ float load_acc(const float* p) { return *p; }
__device__ __forceinline__ float load_acc(const __nv_bfloat16* p) { return __bfloat162float(*p); }

template <int N>
__device__ __forceinline__ double tsum(const double* x, int stride, const double* c) {
  double s = c[0] * x[0];
#pragma unroll
  for (int k = 1; k < N; ++k) s = fma(c[k], x[k * stride], s);
  return s;
}

// In-place Gauss-Jordan inversion with partial (row) pivoting of the NB x NB
// matrix M (row stride LD) in shared memory, by the whole CTA; col holds the
// pivot column, piv the row exchanges (undone on the columns at the end).
template <typename T, int NB, int LD>
__device__ void gauss_jordan(T* M, T* col, int* piv) {
  __shared__ int s_prow;
  for (int k = 0; k < NB; ++k) {
    if (threadIdx.x < 32) {
      T best = (T)-1;
      int bi = k;
      for (int r = k + (int)threadIdx.x; r < NB; r += 32) {
        const T val = fabs(M[r * LD + k]);
        if (val > best) { best = val; bi = r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) { s_prow = bi; piv[k] = bi; }
    }
    __syncthreads();
    const int r = s_prow;
    if (r != k) {
      for (int jj = threadIdx.x; jj < NB; jj += blockDim.x) {
        const T tmp = M[k * LD + jj];
        M[k * LD + jj] = M[r * LD + jj];
        M[r * LD + jj] = tmp;
      }
    }
    __syncthreads();
    for (int ii = threadIdx.x; ii < NB; ii += blockDim.x) col[ii] = M[ii * LD + k];
    __syncthreads();
    const T pinv = (T)1 / col[k];
    for (int jj = threadIdx.x; jj < NB; jj += blockDim.x)
      M[k * LD + jj] = (jj == k ? (T)1 : M[k * LD + jj]) * pinv;
    __syncthreads();
    for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
      const int ii = idx / NB, jj = idx % NB;
      if (ii == k) continue;
      M[ii * LD + jj] = (jj == k ? (T)0 : M[ii * LD + jj]) - col[ii] * M[k * LD + jj];
    }
    __syncthreads();
  }
  for (int k = NB - 1; k >= 0; --k) {
    const int r = piv[k];
    if (r != k) {
      for (int ii = threadIdx.x; ii < NB; ii += blockDim.x) {
        const T tmp = M[ii * LD + k];
        M[ii * LD + k] = M[ii * LD + r];
        M[ii * LD + r] = tmp;
      }
    }
    __syncthreads();
  }
}

// T: arithmetic of the Gauss-Jordan inversion (double, or float for the
// reduced-precision preconditioner); S: storage type of the inverse blocks.
// The finite-difference columns are always formed in FP64.
template <int P, typename T, typename S>
__global__ void __launch_bounds__(FactorLayout<P, T>::THREADS) k_factor(const FactorArgs a) {
  using L = FactorLayout<P, T>;
  constexpr int N = L::N, NP = L::NP, NB = L::NB, LD = L::LD;
  extern __shared__ double smem[];
  double* q = smem + L::OFF_Q;
  double* F = smem + L::OFF_F;
  double* G = smem + L::OFF_G;
  double* tr = smem + L::OFF_TR;
  double* nt = smem + L::OFF_NT;
  double* fn = smem + L::OFF_FN;
  T* M = reinterpret_cast<T*>(smem + L::DOUBLES);
  T* col = M + NB * LD;
  int* piv = reinterpret_cast<int*>(col + NB);

  const long long e = blockIdx.x;
  const int ix = (int)(e % a.nx), iy = (int)(e / a.nx);
  const double hx = a.hx[ix], hy = a.hy[iy];
  const double sJ = 4.0 / (hx * hy);
  const Tables& T_ = a.tab;

  // ---- base state, pointwise fluxes ----
  for (int t = threadIdx.x; t < NP; t += blockDim.x) {
    double qq[4], f[4], g[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      qq[v] = a.U[e * NB + v * NP + t];
      q[v * NP + t] = qq[v];
    }
    euler_fluxes(qq, a.gam, f, g);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      F[v * NP + t] = 0.5 * hy * f[v];
      G[v * NP + t] = 0.5 * hx * g[v];
    }
  }
  __syncthreads();
  // ---- own and neighbour traces, base common fluxes ----
  for (int fp = threadIdx.x; fp < 4 * N; fp += blockDim.x) {
    const int face = fp / N, k = fp % N;
    long long nbr;
    if (face == 0) nbr = (long long)((ix + a.nx - 1) % a.nx) + (long long)a.nx * iy;
    else if (face == 1) nbr = (long long)((ix + 1) % a.nx) + (long long)a.nx * iy;
    else if (face == 2) nbr = (long long)ix + (long long)a.nx * ((iy + a.ny - 1) % a.ny);
    else nbr = (long long)ix + (long long)a.nx * ((iy + 1) % a.ny);
    const int off = face < 2 ? N * k : k;
    const int stride = face < 2 ? 1 : N;
    const double* co = (face == 0 || face == 2) ? T_.lm : T_.lp;
    const double* cn = (face == 0 || face == 2) ? T_.lp : T_.lm;
    double qo[4], qn[4], fc[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      qo[v] = tsum<N>(q + v * NP + off, stride, co);
      qn[v] = tsum<N>(a.U + nbr * NB + v * NP + off, stride, cn);
      tr[(face * 4 + v) * N + k] = qo[v];
      nt[(face * 4 + v) * N + k] = qn[v];
    }
    const int dir = face < 2 ? 0 : 1;
    if (face == 0 || face == 2) riemann_flux(a.riemann, qn, qo, dir, a.gam, fc);
    else riemann_flux(a.riemann, qo, qn, dir, a.gam, fc);
    const double sc = face < 2 ? 0.5 * hy : 0.5 * hx;
#pragma unroll
    for (int v = 0; v < 4; ++v) fn[(face * 4 + v) * N + k] = sc * fc[v];
  }
  __syncthreads();

  // ---- columns of M = shift*I - J_ee ----
  for (int c = threadIdx.x; c < NB; c += blockDim.x) {
    const int vv = c / NP, pt = c % NP, ia = pt % N, jb = pt / N;
    T* Mc = M + c;  // column c, row stride LD
    for (int r = 0; r < NB; ++r) Mc[r * LD] = (r == c) ? (T)a.shift : (T)0;
    const double eps = a.beps * (1.0 + fabs(q[vv * NP + pt]));
    const double inv = 1.0 / eps;
    double qp[4], f[4], g[4], dF[4], dG[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) qp[v] = q[v * NP + pt];
    qp[vv] += eps;
    euler_fluxes(qp, a.gam, f, g);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      dF[v] = 0.5 * hy * f[v] - F[v * NP + pt];
      dG[v] = 0.5 * hx * g[v] - G[v * NP + pt];
    }
    // perturbed common fluxes on the four faces touched: W/E at row jb, S/N at column ia
    double dFn[4][4];
#pragma unroll
    for (int face = 0; face < 4; ++face) {
      const int k = face < 2 ? jb : ia;
      const double cf = face == 0 ? T_.lm[ia] : face == 1 ? T_.lp[ia] : face == 2 ? T_.lm[jb] : T_.lp[jb];
      double qo[4], qn[4], fc[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        qo[v] = tr[(face * 4 + v) * N + k];
        qn[v] = nt[(face * 4 + v) * N + k];
      }
      qo[vv] = fma(cf, eps, qo[vv]);
      const int dir = face < 2 ? 0 : 1;
      if (face == 0 || face == 2) riemann_flux(a.riemann, qn, qo, dir, a.gam, fc);
      else riemann_flux(a.riemann, qo, qn, dir, a.gam, fc);
      const double sc = face < 2 ? 0.5 * hy : 0.5 * hx;
#pragma unroll
      for (int v = 0; v < 4; ++v) dFn[face][v] = sc * fc[v] - fn[(face * 4 + v) * N + k];
    }
    // M = shift I - J with J = -sJ d / eps: row jb (x-direction change) and
    // column ia (y-direction change); the point (ia, jb) gets both.  Each
    // entry is formed in FP64 and stored once.
    for (int i = 0; i < N; ++i) {
      const int pnt = i + N * jb;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double d = T_.Dt[i][ia] * dF[v];
        d = fma(T_.dgL[i], dFn[0][v], d);
        d = fma(T_.dgR[i], dFn[1][v], d);
        if (i == ia) {
          d = fma(T_.Dt[jb][jb], dG[v], d);
          d = fma(T_.dgL[jb], dFn[2][v], d);
          d = fma(T_.dgR[jb], dFn[3][v], d);
        }
        const int row = v * NP + pnt;
        Mc[row * LD] = (T)((row == c ? a.shift : 0.0) + sJ * d * inv);
      }
    }
    for (int j = 0; j < N; ++j) {
      if (j == jb) continue;
      const int pnt = ia + N * j;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double d = T_.Dt[j][jb] * dG[v];
        d = fma(T_.dgL[j], dFn[2][v], d);
        d = fma(T_.dgR[j], dFn[3][v], d);
        Mc[(v * NP + pnt) * LD] = (T)(sJ * d * inv);
      }
    }
  }
  __syncthreads();

  // stage M (column-major) so a later shift change only re-inverts
  {
    double* st = a.mst + e * (long long)NB * NB;
    for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
      const int c = idx / NB, r = idx % NB;
      st[idx] = (double)M[r * LD + c];
    }
  }
  __syncthreads();
  S* out = reinterpret_cast<S*>(a.blocks) + e * (long long)NB * NB;
  if constexpr (L::TC) {
    unsigned char* tcs = reinterpret_cast<unsigned char*>(smem) + L::OFF_TC;
    const bool ok = gjtc::invert<NB, LD>(M, col, piv, tcs);
    if (!ok && threadIdx.x == 0) atomicExch(a.err, 1);
    // ---- store column-major: inverse(i, k) = M[pr[i]][ipr[k]] ----
    const int* ipr = reinterpret_cast<const int*>(tcs + gjtc::Shape<NB>::OFF_IPR);
    for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
      const int kk = idx / NB, ii = idx % NB;
      out[idx] = StoreT<S>::to(M[piv[ii] * LD + ipr[kk]]);
    }
  } else {
    gauss_jordan<T, NB, LD>(M, col, piv);
    // ---- store column-major: Minv[k*NB + i] = inverse(i, k) ----
    for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
      const int kk = idx / NB, ii = idx % NB;
      out[idx] = StoreT<S>::to(M[ii * LD + kk]);
    }
  }
}

// Invert staged FP64 blocks (column-major per element: mst[e][c][row]) into
// the preconditioner storage; one CTA per element.
template <int NB, typename T>
struct InvertLayout {
  static constexpr int LD = NB + 1;
  static constexpr bool TC = gjtc::Use<T, NB>::value;
  static constexpr size_t GJ_END = (size_t)(NB * LD + NB) * sizeof(T) + NB * sizeof(int);
  static constexpr size_t OFF_TC = (GJ_END + 127) / 128 * 128;
  static constexpr size_t BYTES = TC ? OFF_TC + gjtc::Shape<NB>::BYTES : GJ_END + 64;
};

template <int NB, typename T, typename S>
__global__ void __launch_bounds__(256) k_invert(const double* __restrict__ mst, void* blocks, long long e0,
                                                double dshift, int* err) {
  using L = InvertLayout<NB, T>;
  constexpr int LD = L::LD;
  extern __shared__ double smem_inv[];
  T* M = reinterpret_cast<T*>(smem_inv);
  T* col = M + NB * LD;
  int* piv = reinterpret_cast<int*>(col + NB);
  const long long e = e0 + blockIdx.x;
  const double* src = mst + (long long)blockIdx.x * NB * NB;
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
    const int c = idx / NB, r = idx % NB;
    M[r * LD + c] = (T)(r == c ? src[idx] + dshift : src[idx]);
  }
  __syncthreads();
  S* out = reinterpret_cast<S*>(blocks) + e * (long long)NB * NB;
  if constexpr (L::TC) {
    unsigned char* tcs = reinterpret_cast<unsigned char*>(smem_inv) + L::OFF_TC;
    const bool ok = gjtc::invert<NB, LD>(M, col, piv, tcs);
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
    const int* ipr = reinterpret_cast<const int*>(tcs + gjtc::Shape<NB>::OFF_IPR);
    for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
      const int kk = idx / NB, ii = idx % NB;
      out[idx] = StoreT<S>::to(M[piv[ii] * LD + ipr[kk]]);
    }
  } else {
    gauss_jordan<T, NB, LD>(M, col, piv);
    for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
      const int kk = idx / NB, ii = idx % NB;
      out[idx] = StoreT<S>::to(M[ii * LD + kk]);
    }
  }
}

// z = Minv r (optionally r scaled by *scale first and written back), optional
// sum of squares of z.  EPC elements per CTA, one thread per block row.
// S: block storage type; A: accumulation type (FP64 for FP64 blocks, FP32 otherwise).
// Shape of the staged apply per block size and storage type: KS threads
// share one row's dot product (threads = KS nb), NS elements in flight per
// CTA (element block + its r, one bulk copy each, in a ring of stages).
template <int NB, typename S> struct ApplyShape;
template <> struct ApplyShape<36, double> { static constexpr int KS = 4, NS = 6; };
template <> struct ApplyShape<64, double> { static constexpr int KS = 1, NS = 1; };  // swept: (KS, NS) = (1, 1) 192 us, (1, 2) 197, (2, 2) 201, (2, 3) 218, (4, 3) 231 at 160^2 p=3
template <> struct ApplyShape<100, double> { static constexpr int KS = 2, NS = 2; };
template <> struct ApplyShape<36, float> { static constexpr int KS = 4, NS = 8; };
template <> struct ApplyShape<64, float> { static constexpr int KS = 2, NS = 4; };
template <> struct ApplyShape<100, float> { static constexpr int KS = 2, NS = 3; };
template <> struct ApplyShape<36, __nv_bfloat16> { static constexpr int KS = 4, NS = 8; };
template <> struct ApplyShape<64, __nv_bfloat16> { static constexpr int KS = 2, NS = 6; };
template <> struct ApplyShape<100, __nv_bfloat16> { static constexpr int KS = 2, NS = 4; };
template <> struct ApplyShape<40, double> { static constexpr int KS = 4, NS = 6; };
template <> struct ApplyShape<40, float> { static constexpr int KS = 4, NS = 8; };
template <> struct ApplyShape<40, __nv_bfloat16> { static constexpr int KS = 4, NS = 8; };
template <> struct ApplyShape<144, double> { static constexpr int KS = 1, NS = 1; };
template <> struct ApplyShape<144, float> { static constexpr int KS = 1, NS = 2; };
template <> struct ApplyShape<144, __nv_bfloat16> { static constexpr int KS = 1, NS = 4; };
template <> struct ApplyShape<196, double> { static constexpr int KS = 1, NS = 1; };  // does not fit: rejected
template <> struct ApplyShape<196, float> { static constexpr int KS = 1, NS = 1; };
template <> struct ApplyShape<196, __nv_bfloat16> { static constexpr int KS = 1, NS = 2; };

template <int NB, typename S, typename A>
struct ApplyLayout {
  static constexpr int KS = ApplyShape<NB, S>::KS, NS = ApplyShape<NB, S>::NS;
  static constexpr int WORKERS = KS * NB;                   // threads with a (row, k-range)
  static constexpr int THREADS = (WORKERS + 31) / 32 * 32;  // whole warps (the reductions shuffle)
  static constexpr unsigned MB = (unsigned)(NB * NB * sizeof(S));  // one block (multiple of 16)
  static constexpr unsigned RB = (unsigned)(NB * sizeof(double));  // its r (multiple of 16)
  static constexpr unsigned STAGE = (MB + RB + 127) / 128 * 128;
  static constexpr size_t BYTES = (size_t)NS * STAGE + (size_t)(1 + KS) * NB * sizeof(A) + 32 * sizeof(double) +
                                  NS * sizeof(unsigned long long);
};

// z_e = M_e^-1 (s r_e) per element (optionally r_e *= s written back), and the
// sum of squares of z.  Persistent CTAs walk the elements e = blockIdx.x +
// t gridDim.x; thread 0 keeps NS elements' block and r in flight with bulk
// copies (TMA engine) completing on per-stage mbarriers, so the block bytes
// stream from HBM while the previous elements are multiplied out of shared
// memory (column-major blocks: thread i reads consecutive addresses).  Each
// row's dot product is split over KS threads and summed in a fixed order.
// A wait that gives up sets *kerr, waits (bounded) for the copies it issued
// and leaves.
template <int NB, typename S, typename A>
__device__ __forceinline__ void apply_body(const S* __restrict__ Minv, double* r, const double* scale,
                                           double* __restrict__ z, long long ne, double* sumsq, const Reduce& red,
                                           const int* done, const EpsArgs& ea, int* kerr, unsigned polls,
                                           int skip_first_copy, int bid, int nblk) {
  using L = ApplyLayout<NB, S, A>;
  constexpr int KS = L::KS, NS = L::NS, KP = NB / KS;
  extern __shared__ __align__(128) double smem_d[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(smem_d);
  A* rs = reinterpret_cast<A*>(smem + (size_t)NS * L::STAGE);
  A* part = rs + NB;
  double* sh = reinterpret_cast<double*>(part + KS * NB);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(sh + 32);
  if (done && *done) return;
  const int tid = threadIdx.x, i = tid % NB, ks = tid / NB;  // ks == KS: padding thread
  const long long G = nblk;
  const long long nloc = ne > (long long)bid ? (ne - 1 - bid) / G + 1 : 0;
  if (tid == 0) {
    for (int q = 0; q < NS; ++q) mbar_init(&bar[q], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](long long t) {
    // test hook: CTA 0 leaves its first element's copies unissued, so its
    // bounded wait for them runs out
    if (skip_first_copy && bid == 0 && t == 0) return;
    const int q = (int)(t % NS);
    const long long e = bid + t * G;
    unsigned char* st = smem + (size_t)q * L::STAGE;
    mbar_arrive_expect_tx(&bar[q], L::MB + L::RB);
    bulk_g2s(st, Minv + e * NB * NB, L::MB, &bar[q]);
    bulk_g2s(st + L::MB, r + e * NB, L::RB, &bar[q]);
  };
  if (tid == 0)
    for (long long t = 0; t < NS && t < nloc; ++t) issue(t);
  const double sc = scale ? *scale : 1.0;
  double ss = 0.0;
  long long t = 0;
  for (; t < nloc; ++t) {
    const int q = (int)(t % NS);
    const bool ok = mbar_wait(&bar[q], (unsigned)((t / NS) & 1), polls);
    if (!__syncthreads_and(ok)) break;
    const long long e = bid + t * G;
    const S* Ms = reinterpret_cast<const S*>(smem + (size_t)q * L::STAGE);
    const double* rsrc = reinterpret_cast<const double*>(smem + (size_t)q * L::STAGE + L::MB);
    if (ks == 0) {
      double v = rsrc[i];
      if (scale) {
        v *= sc;
        r[e * NB + i] = v;
      }
      rs[i] = (A)v;
    }
    __syncthreads();
    if (ks < KS) {
      const S* Mk = Ms + (size_t)(ks * KP) * NB + i;
      const A* rk = rs + ks * KP;
      A acc0 = 0, acc1 = 0;
#pragma unroll
      for (int k = 0; k < KP; k += 2) {
        acc0 = fma(load_acc(Mk + k * NB), rk[k], acc0);
        if (k + 1 < KP) acc1 = fma(load_acc(Mk + (k + 1) * NB), rk[k + 1], acc1);
      }
      part[ks * NB + i] = acc0 + acc1;
    }
    __syncthreads();  // stage q consumed, partial sums visible
    if (tid == 0 && t + NS < nloc) issue(t + NS);
    if (ks == 0) {
      A zz = part[i];
#pragma unroll
      for (int u = 1; u < KS; ++u) zz += part[u * NB + i];
      const double zi = (double)zz;
      z[e * NB + i] = zi;
      ss = fma(zi, zi, ss);
    }
  }
  if (t < nloc && tid == 0) {  // a copy never completed: flag it and drain what was issued
    atomicExch(kerr, 1);
    for (long long u = t; u < nloc && u < t + NS; ++u)
      (void)mbar_wait(&bar[u % NS], (unsigned)((u / NS) & 1), polls);
  }
  if (sumsq) {  // every CTA takes part, so the reduction's counter stays consistent
    const double bs = block_sum(ss, sh);
    if (threadIdx.x == 0) red.partials[(size_t)bid * kMaxVec] = bs;
    if (last_block(red.counter, nblk)) {
      finish_sums(red, 1, sumsq, nblk);
      if (threadIdx.x == 0) write_eps(ea, *sumsq);
    }
  }
}

template <int NB, typename S, typename A>
__global__ void __launch_bounds__(ApplyLayout<NB, S, A>::THREADS)
    k_apply(const S* __restrict__ Minv, double* r, const double* scale, double* __restrict__ z, long long ne,
            double* sumsq, Reduce red, const int* done, EpsArgs ea, int* kerr, unsigned polls,
            int skip_first_copy) {
  apply_body<NB, S, A>(Minv, r, scale, z, ne, sumsq, red, done, ea, kerr, polls, skip_first_copy, blockIdx.x,
                       gridDim.x);
}

}  // namespace

// Per-instance arguments of the batched apply (Arnoldi iteration j: r = V_j,
// scale = 1/||v_j|| = invh[j]).
struct BatchApply {
  const void* Minv;
  double* V;
  long long n;
  const double* invh;
  double* z;
  long long ne;
  double* sumsq;
  Reduce red;
  const int* done;
  EpsArgs ea;
  int* kerr;
  unsigned polls;
  int skip;
};

namespace {

// z = M^-1 v_j of every instance (of one block size) in one grid; instance k
// owns blocks [start[k], start[k+1]), the partition of its own launch.
template <int NB, typename S, typename A>
__global__ void __launch_bounds__(ApplyLayout<NB, S, A>::THREADS)
    kb_apply(const BatchApply* __restrict__ tab, const int* __restrict__ start, int ninst, int j) {
  const int k = batch_instance(start, ninst, blockIdx.x);
  const BatchApply& t = tab[k];
  const int bid = blockIdx.x - start[k], nblk = start[k + 1] - start[k];
  apply_body<NB, S, A>(reinterpret_cast<const S*>(t.Minv), t.V + (size_t)j * t.n, t.invh + j, t.z, t.ne, t.sumsq,
                       t.red, t.done, t.ea, t.kerr, t.polls, t.skip, bid, nblk);
}

// Elements per pass and threads of the one-thread-per-row kernels.
template <int NB> struct RowsShape {
  static constexpr int EPC = NB >= 256 ? 1 : 256 / NB;
  static constexpr int THREADS = (EPC * NB + 31) / 32 * 32;
};

// z_e = M_e^-1 (s r_e) for blocks whose rows are not 16-byte multiples (3D
// degree 2: nb = 135) or too large to stage in shared memory (3D degree 3:
// nb = 320), without bulk copies: EPC elements per pass, one thread per row,
// column-major blocks so thread i reads consecutive addresses; optional
// r_e *= s written back and sum of squares of z.
template <int NB, typename S, typename A>
__global__ void __launch_bounds__(RowsShape<NB>::THREADS) k_apply_rows(const S* __restrict__ Minv, double* r,
                                                                       const double* scale, double* z, long long ne,
                                                                       double* sumsq, Reduce red, const int* done,
                                                                       EpsArgs ea) {
  constexpr int EPC = RowsShape<NB>::EPC;
  __shared__ A rs[EPC][NB];
  __shared__ double sh[32];
  if (done && *done) return;
  const double sc = scale ? *scale : 1.0;
  const int el = threadIdx.x / NB, i = threadIdx.x % NB;
  double ss = 0.0;
  for (long long e0 = (long long)blockIdx.x * EPC; e0 < ne; e0 += (long long)gridDim.x * EPC) {
    const long long e = e0 + el;
    const bool act = el < EPC && e < ne;
    __syncthreads();
    if (act) {
      double v = r[e * NB + i];
      if (scale) {
        v *= sc;
        r[e * NB + i] = v;
      }
      rs[el][i] = (A)v;
    }
    __syncthreads();
    if (act) {
      const S* Me = Minv + e * (long long)NB * NB;
      A acc = 0;
#pragma unroll 16
      for (int kk = 0; kk < NB; ++kk) acc = fma(load_acc(Me + kk * NB + i), rs[el][kk], acc);
      const double zi = (double)acc;
      z[e * NB + i] = zi;
      ss = fma(zi, zi, ss);
    }
  }
  if (sumsq) {
    const double bs = block_sum(ss, sh);
    if (threadIdx.x == 0) red.partials[(size_t)blockIdx.x * kMaxVec] = bs;
    if (last_block(red.counter)) {
      finish_sums(red, 1, sumsq);
      if (threadIdx.x == 0) write_eps(ea, *sumsq);
    }
  }
}

// The row apply for BF16 blocks of even, large nb (3D degree 3: nb = 320):
// each thread two adjacent rows, so one 4-byte load brings the bf16 pair of
// a column and a warp request covers 128 bytes (2-byte loads left the apply
// at two thirds of HBM bandwidth).  Two elements per CTA, nb threads.  Each
// row's sum runs over the columns in the same order as in k_apply_rows.
template <int NB>
__global__ void __launch_bounds__(NB) k_apply_rows_bf2(const __nv_bfloat16* __restrict__ Minv, double* r,
                                                       const double* scale, double* z, long long ne,
                                                       double* sumsq, Reduce red, const int* done, EpsArgs ea) {
  static_assert(NB % 64 == 0, "two rows per thread, whole warps per element");
  constexpr int HALF = NB / 2, EPC = 2;
  __shared__ float rs[EPC][NB];
  __shared__ double sh[32];
  if (done && *done) return;
  const double sc = scale ? *scale : 1.0;
  const int el = threadIdx.x / HALF, i2 = threadIdx.x % HALF;
  double ss = 0.0;
  for (long long e0 = (long long)blockIdx.x * EPC; e0 < ne; e0 += (long long)gridDim.x * EPC) {
    const long long e = e0 + el;
    const bool act = e < ne;
    __syncthreads();
    if (act) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        double v = r[e * NB + 2 * i2 + h];
        if (scale) {
          v *= sc;
          r[e * NB + 2 * i2 + h] = v;
        }
        rs[el][2 * i2 + h] = (float)v;
      }
    }
    __syncthreads();
    if (act) {
      const __nv_bfloat162* Me = reinterpret_cast<const __nv_bfloat162*>(Minv + e * (long long)NB * NB);
      float a0 = 0.f, a1 = 0.f;
#pragma unroll 16
      for (int kk = 0; kk < NB; ++kk) {
        const float2 m = __bfloat1622float2(Me[kk * HALF + i2]);
        const float x = rs[el][kk];
        a0 = fmaf(m.x, x, a0);
        a1 = fmaf(m.y, x, a1);
      }
      const double z0 = (double)a0, z1 = (double)a1;
      z[e * NB + 2 * i2] = z0;
      z[e * NB + 2 * i2 + 1] = z1;
      ss = fma(z0, z0, ss);
      ss = fma(z1, z1, ss);
    }
  }
  if (sumsq) {
    const double bs = block_sum(ss, sh);
    if (threadIdx.x == 0) red.partials[(size_t)blockIdx.x * kMaxVec] = bs;
    if (last_block(red.counter)) {
      finish_sums(red, 1, sumsq);
      if (threadIdx.x == 0) write_eps(ea, *sumsq);
    }
  }
}

// z = s * r (no preconditioner), optional r *= s written back, optional sum of squares.
__global__ void k_scale_copy(double* r, const double* scale, double* z, long long n,
                             double* sumsq, Reduce red, const int* done, EpsArgs ea) {
  __shared__ double sh[32];
  if (done && *done) return;
  const double s = scale ? *scale : 1.0;
  double ss = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double v = r[i];
    if (scale) {
      v *= s;
      r[i] = v;
    }
    if (z != r) z[i] = v;
    ss = fma(v, v, ss);
  }
  if (sumsq) {
    const double bs = block_sum(ss, sh);
    if (threadIdx.x == 0) red.partials[(size_t)blockIdx.x * kMaxVec] = bs;
    if (last_block(red.counter)) {
      finish_sums(red, 1, sumsq);
      if (threadIdx.x == 0) write_eps(ea, *sumsq);
    }
  }
}

// x += Minv (sum_{l<k} y_l V_l) per element (precond) -- right-preconditioned update.
template <int NB, typename S, typename A>
__global__ void __launch_bounds__(RowsShape<NB>::THREADS) k_solupdate(const S* __restrict__ Minv,
                                                                      const double* __restrict__ V, long long ldv,
                                                                      const double* y, const int* kp, double* x,
                                                                      long long ne) {
  constexpr int EPC = RowsShape<NB>::EPC;
  __shared__ A ts[EPC][NB];
  __shared__ double ys[kMaxVec];
  const int k = *kp;
  if (k <= 0) return;
  if (threadIdx.x < k) ys[threadIdx.x] = y[threadIdx.x];
  const int el = threadIdx.x / NB, i = threadIdx.x % NB;
  for (long long e0 = (long long)blockIdx.x * EPC; e0 < ne; e0 += (long long)gridDim.x * EPC) {
    const long long e = e0 + el;
    const bool act = el < EPC && e < ne;
    __syncthreads();
    if (act) {
      double t = 0.0;
      for (int l = 0; l < k; ++l) t = fma(ys[l], V[l * ldv + e * NB + i], t);
      ts[el][i] = (A)t;
    }
    __syncthreads();
    if (act) {
      const S* Me = Minv + e * (long long)NB * NB;
      A acc = 0;
#pragma unroll 16
      for (int kk = 0; kk < NB; ++kk) acc = fma(load_acc(Me + kk * NB + i), ts[el][kk], acc);
      x[e * NB + i] += (double)acc;
    }
  }
}

// x += sum_{l<k} y_l V_l (no preconditioner)
__global__ void k_solupdate_plain(const double* __restrict__ V, long long ldv, const double* y,
                                  const int* kp, double* x, long long n) {
  __shared__ double ys[kMaxVec];
  const int k = *kp;
  if (k <= 0) return;
  if (threadIdx.x < k) ys[threadIdx.x] = y[threadIdx.x];
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int l = 0; l < k; ++l) t = fma(ys[l], V[l * ldv + i], t);
    x[i] += t;
  }
}

template <int P, typename T, typename S>
int factor_pts(fr_ctx* ctx, const FactorArgs& a, cudaStream_t s) {
  using L = FactorLayout<P, T>;
  if constexpr (L::BYTES > kSmemMax) {
    return set_error(ctx, FR_ERR_UNSUPPORTED, "FP64 element blocks of degree %d exceed shared memory; "
                     "use block_precision 1 or 2", P);
  }
  FRK_CUDA(ctx, cudaFuncSetAttribute(k_factor<P, T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)L::BYTES));
  // work: read U (8 B/DOF), write ne nb^2 entries of S; flops per element as counted
  const double fb = 8.0 * (double)ctx->ndof + (double)sizeof(S) * (double)ctx->ne * L::NB * L::NB;
  const double ff = factor_flops_per_element(P) * (double)ctx->ne;
  { ProfScope ps_(ctx, FR_KF_FACTOR, s, fb, ff); k_factor<P, T, S><<<(unsigned)ctx->ne, L::THREADS, L::BYTES, s>>>(a); }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

template <int P>
int factor_p(fr_ctx* ctx, const FactorArgs& a, cudaStream_t s) {
  switch (ctx->opts.block_precision) {
    case 1: return factor_pts<P, float, float>(ctx, a, s);
    case 2: return factor_pts<P, float, __nv_bfloat16>(ctx, a, s);
    default: return factor_pts<P, double, double>(ctx, a, s);
  }
}

template <int NB>
unsigned apply_grid(long long ne) {
  constexpr int EPC = RowsShape<NB>::EPC;
  long long g = (ne + EPC - 1) / EPC;
  if (g > kRedBlocks) g = kRedBlocks;
  return (unsigned)(g < 1 ? 1 : g);
}

// persistent grid of the staged apply: resident CTAs per SM x SMs, at most
// one CTA per element (the function attributes are set once per process)
template <int NB, typename S, typename A>
int apply_grid_nbs(fr_ctx* ctx, long long* grid_out) {
  using L = ApplyLayout<NB, S, A>;
  static int per_sm = 0;
  if (per_sm == 0) {
    FRK_CUDA(ctx, cudaFuncSetAttribute(k_apply<NB, S, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES));
    FRK_CUDA(ctx, cudaFuncSetAttribute(kb_apply<NB, S, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES));
    int occ = 0;
    FRK_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_apply<NB, S, A>, L::THREADS, L::BYTES));
    per_sm = occ > 0 ? occ : 1;
  }
  long long grid = (long long)per_sm * ctx->num_sms;
  if (grid > ctx->ne) grid = ctx->ne;
  if (grid > kRedBlocks) grid = kRedBlocks;
  if (grid < 1) grid = 1;
  *grid_out = grid;
  return FR_OK;
}

template <int NB, typename S, typename A>
int apply_nbs(fr_ctx* ctx, double* r, const double* scale, double* z, double* sumsq,
              const int* done, cudaStream_t s, bool with_eps) {
  // work: ne nb^2 block entries, r in, z out (and r written back when scaled):
  // 2 nb flops per DOF.  Inside a GMRES cycle it is booked per finished iteration.
  const bool in_cycle = done != nullptr;
  const double nd = (double)ctx->ndof;
  const double wb = in_cycle ? 0.0 : (double)sizeof(S) * (double)ctx->ne * NB * NB + 16.0 * nd + (scale ? 8.0 * nd : 0.0);
  const double wf = in_cycle ? 0.0 : 2.0 * NB * nd;
  using L = ApplyLayout<NB, S, A>;
  if constexpr (L::BYTES > kSmemMax) {
    return set_error(ctx, FR_ERR_UNSUPPORTED, "element blocks of %d rows in this precision exceed shared memory", NB);
  }
  // the staged apply copies r with the bulk-copy engine: 16-byte aligned rows
  if (reinterpret_cast<uintptr_t>(r) % 16 != 0)
    return set_error(ctx, FR_ERR_INVALID_ARG, "ejacobi_apply: r must be 16-byte aligned");
  long long grid = 0;
  FRK_TRY((apply_grid_nbs<NB, S, A>(ctx, &grid)));
  { ProfScope ps_(ctx, FR_KF_APPLY, s, wb, wf); k_apply<NB, S, A><<<(unsigned)grid, L::THREADS, L::BYTES, s>>>(reinterpret_cast<const S*>(ctx->blocks), r, scale, z, ctx->ne,
                                                                  sumsq, ctx->red, done, eps_args(ctx, with_eps), ctx->kerr,
                                                                  ctx->wait_polls, ctx->test_skip_copy); }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

template <int NB, typename S, typename A>
int apply_rows_nbs(fr_ctx* ctx, double* r, const double* scale, double* z, double* sumsq,
                   const int* done, cudaStream_t s, bool with_eps) {
  const bool in_cycle = done != nullptr;
  const double nd = (double)ctx->ndof;
  const double wb = in_cycle ? 0.0 : (double)sizeof(S) * (double)ctx->ne * NB * NB + 16.0 * nd + (scale ? 8.0 * nd : 0.0);
  const double wf = in_cycle ? 0.0 : 2.0 * NB * nd;
  constexpr int threads = RowsShape<NB>::THREADS;  // whole warps (the reduction shuffles)
  if constexpr (std::is_same<S, __nv_bfloat16>::value && NB % 64 == 0) {
    long long g = (ctx->ne + 1) / 2;
    if (g > kRedBlocks) g = kRedBlocks;
    { ProfScope ps_(ctx, FR_KF_APPLY, s, wb, wf);
      k_apply_rows_bf2<NB><<<(unsigned)g, NB, 0, s>>>(reinterpret_cast<const S*>(ctx->blocks), r, scale, z, ctx->ne,
                                                      sumsq, ctx->red, done, eps_args(ctx, with_eps)); }
  } else {
    ProfScope ps_(ctx, FR_KF_APPLY, s, wb, wf);
    k_apply_rows<NB, S, A><<<apply_grid<NB>(ctx->ne), threads, 0, s>>>(reinterpret_cast<const S*>(ctx->blocks), r, scale, z,
                                                                       ctx->ne, sumsq, ctx->red, done, eps_args(ctx, with_eps));
  }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

template <int NB>
int apply_rows_nb(fr_ctx* ctx, double* r, const double* scale, double* z, double* sumsq,
                  const int* done, cudaStream_t s, bool with_eps) {
  switch (ctx->opts.block_precision) {
    case 1: return apply_rows_nbs<NB, float, float>(ctx, r, scale, z, sumsq, done, s, with_eps);
    case 2: return apply_rows_nbs<NB, __nv_bfloat16, float>(ctx, r, scale, z, sumsq, done, s, with_eps);
    default: return apply_rows_nbs<NB, double, double>(ctx, r, scale, z, sumsq, done, s, with_eps);
  }
}

template <int NB>
int apply_nb(fr_ctx* ctx, double* r, const double* scale, double* z, double* sumsq,
             const int* done, cudaStream_t s, bool with_eps) {
  switch (ctx->opts.block_precision) {
    case 1: return apply_nbs<NB, float, float>(ctx, r, scale, z, sumsq, done, s, with_eps);
    case 2: return apply_nbs<NB, __nv_bfloat16, float>(ctx, r, scale, z, sumsq, done, s, with_eps);
    default: return apply_nbs<NB, double, double>(ctx, r, scale, z, sumsq, done, s, with_eps);
  }
}

template <int NB, typename S, typename A>
int solupdate_nbs(fr_ctx* ctx, double* x, cudaStream_t s) {
  { ProfScope ps_(ctx, FR_KF_SOLUPDATE, s); k_solupdate<NB, S, A><<<apply_grid<NB>(ctx->ne), RowsShape<NB>::THREADS, 0, s>>>(
      reinterpret_cast<const S*>(ctx->blocks), ctx->V, ctx->ndof, ctx->gd.y, ctx->gd.k, x, ctx->ne); }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

template <int NB>
int solupdate_nb(fr_ctx* ctx, double* x, cudaStream_t s) {
  switch (ctx->opts.block_precision) {
    case 1: return solupdate_nbs<NB, float, float>(ctx, x, s);
    case 2: return solupdate_nbs<NB, __nv_bfloat16, float>(ctx, x, s);
    default: return solupdate_nbs<NB, double, double>(ctx, x, s);
  }
}

unsigned vec_grid(const fr_ctx* ctx, long long n) {
  long long g = (n + kThreads - 1) / kThreads;
  if (g > ctx->vec_blocks) g = ctx->vec_blocks;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

template <int NB, typename T, typename S>
int invert_nbts(fr_ctx* ctx, const double* mst, double dshift, long long e0, long long n, cudaStream_t s) {
  constexpr size_t bytes = InvertLayout<NB, T>::BYTES;
  if constexpr (bytes > kSmemMax) {
    return set_error(ctx, FR_ERR_UNSUPPORTED, "element blocks of %d rows in this precision exceed shared memory", NB);
  }
  FRK_CUDA(ctx, cudaFuncSetAttribute(k_invert<NB, T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)bytes));
  { ProfScope ps_(ctx, FR_KF_INVERT, s, 0.0, 2.0 * NB * NB * (double)NB * (double)n);
    k_invert<NB, T, S><<<(unsigned)n, NB <= 64 ? 128 : 256, bytes, s>>>(mst, ctx->blocks, e0, dshift, ctx->kerr); }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

// blocks larger than one SM's shared memory: FP32 Gauss-Jordan over a
// cluster of two CTAs (gj_cluster.cuh), stored in S
template <int NB, typename S>
int invert_cluster_nbs(fr_ctx* ctx, const double* mst, double dshift, long long e0, long long n, cudaStream_t s) {
  using Sh = gjcl::Shape<NB>;
  static_assert(Sh::BYTES <= kSmemMax, "one CTA's half of the block fits shared memory");
  auto kern = gjcl::k_invert_cluster<NB, S, StoreT<S>>;
  FRK_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::BYTES));
  { ProfScope ps_(ctx, FR_KF_INVERT, s, 0.0, 2.0 * NB * NB * (double)NB * (double)n);
    kern<<<(unsigned)(n * gjcl::CL), gjcl::THREADS, Sh::BYTES, s>>>(mst, reinterpret_cast<S*>(ctx->blocks), e0,
                                                                   dshift); }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

template <int NB>
int invert_nb(fr_ctx* ctx, const double* mst, double dshift, long long e0, long long n, cudaStream_t s) {
  switch (ctx->opts.block_precision) {
    case 1: return invert_nbts<NB, float, float>(ctx, mst, dshift, e0, n, s);
    case 2: return invert_nbts<NB, float, __nv_bfloat16>(ctx, mst, dshift, e0, n, s);
    default: return invert_nbts<NB, double, double>(ctx, mst, dshift, e0, n, s);
  }
}

int launch_block_invert_range(fr_ctx* ctx, const double* mst, double dshift, long long e0, long long n,
                              cudaStream_t s) {
  if (n <= 0) return FR_OK;
  switch (ctx->nb) {
    case 36: return invert_nb<36>(ctx, mst, dshift, e0, n, s);
    case 40: return invert_nb<40>(ctx, mst, dshift, e0, n, s);
    case 135: return invert_nb<135>(ctx, mst, dshift, e0, n, s);
    case 64: return invert_nb<64>(ctx, mst, dshift, e0, n, s);
    case 100: return invert_nb<100>(ctx, mst, dshift, e0, n, s);
    case 144: return invert_nb<144>(ctx, mst, dshift, e0, n, s);
    case 196: return invert_nb<196>(ctx, mst, dshift, e0, n, s);
    case 320:
      switch (ctx->opts.block_precision) {
        case 1: return invert_cluster_nbs<320, float>(ctx, mst, dshift, e0, n, s);
        case 2: return invert_cluster_nbs<320, __nv_bfloat16>(ctx, mst, dshift, e0, n, s);
        default: return set_error(ctx, FR_ERR_UNSUPPORTED, "320-row element blocks are stored in FP32 or BF16");
      }
    default: return set_error(ctx, FR_ERR_UNSUPPORTED, "block size %d not compiled", ctx->nb);
  }
}

int launch_block_invert(fr_ctx* ctx, const double* mst, double dshift, cudaStream_t s) {
  return launch_block_invert_range(ctx, mst, dshift, 0, ctx->ne, s);
}

int launch_block_reshift(fr_ctx* ctx, double shift, cudaStream_t s) {
  if (ctx->blk_chunk < ctx->ne)
    return set_error(ctx, FR_ERR_UNSUPPORTED, "the staged blocks are kept per chunk only; form them again");
  FRK_TRY(launch_block_invert(ctx, ctx->mst, shift - ctx->staged_shift, s));
  ctx->blocks_valid = 1;
  return FR_OK;
}

int launch_block_factor(fr_ctx* ctx, const double* U, double shift, cudaStream_t s) {
  ctx->staged_shift = shift;
  if (ctx->dim3) return launch_f3_factor(ctx, U, shift, s);
  if (ctx->viscous) return launch_ns_factor(ctx, U, shift, s);
  FactorArgs a;
  a.U = U; a.blocks = ctx->blocks; a.mst = ctx->mst; a.hx = ctx->hx; a.hy = ctx->hy;
  a.ne = ctx->ne; a.nx = ctx->nx; a.ny = ctx->ny;
  a.gam = ctx->opts.gamma; a.shift = shift; a.beps = ctx->opts.block_eps_rel;
  a.riemann = ctx->opts.riemann;
  a.err = ctx->kerr;
  a.tab = ctx->tab;
  switch (ctx->p) {
    case 2: return factor_p<2>(ctx, a, s);
    case 3: return factor_p<3>(ctx, a, s);
    case 4: return factor_p<4>(ctx, a, s);
    case 5: return factor_p<5>(ctx, a, s);
    case 6: return factor_p<6>(ctx, a, s);
    default: return set_error(ctx, FR_ERR_UNSUPPORTED, "degree %d not compiled", ctx->p);
  }
}

int launch_block_apply(fr_ctx* ctx, double* r, const double* scale, double* z, double* sumsq,
                       const int* done, cudaStream_t s, bool with_eps) {
  if (!ctx->opts.precond) {
    { ProfScope ps_(ctx, FR_KF_APPLY, s); k_scale_copy<<<vec_grid(ctx, ctx->ndof), kThreads, 0, s>>>(r, scale, z, ctx->ndof, sumsq, ctx->red,
                                                          done, eps_args(ctx, with_eps)); }
    FRK_LAUNCHED(ctx);
    return FR_OK;
  }
  switch (ctx->nb) {
    case 36: return apply_nb<36>(ctx, r, scale, z, sumsq, done, s, with_eps);
    case 40: return apply_nb<40>(ctx, r, scale, z, sumsq, done, s, with_eps);
    case 135: return apply_rows_nb<135>(ctx, r, scale, z, sumsq, done, s, with_eps);
    case 320: return apply_rows_nb<320>(ctx, r, scale, z, sumsq, done, s, with_eps);
    case 64: return apply_nb<64>(ctx, r, scale, z, sumsq, done, s, with_eps);
    case 100: return apply_nb<100>(ctx, r, scale, z, sumsq, done, s, with_eps);
    case 144: return apply_nb<144>(ctx, r, scale, z, sumsq, done, s, with_eps);
    case 196: return apply_nb<196>(ctx, r, scale, z, sumsq, done, s, with_eps);
    default: return set_error(ctx, FR_ERR_UNSUPPORTED, "block size %d not compiled", ctx->nb);
  }
}

int launch_solution_update(fr_ctx* ctx, double* x, cudaStream_t s) {
  if (!ctx->opts.precond) {
    { ProfScope ps_(ctx, FR_KF_SOLUPDATE, s); k_solupdate_plain<<<vec_grid(ctx, ctx->ndof), kThreads, 0, s>>>(ctx->V, ctx->ndof, ctx->gd.y,
                                                               ctx->gd.k, x, ctx->ndof); }
    FRK_LAUNCHED(ctx);
    return FR_OK;
  }
  switch (ctx->nb) {
    case 36: return solupdate_nb<36>(ctx, x, s);
    case 40: return solupdate_nb<40>(ctx, x, s);
    case 135: return solupdate_nb<135>(ctx, x, s);
    case 320: return solupdate_nb<320>(ctx, x, s);
    case 64: return solupdate_nb<64>(ctx, x, s);
    case 100: return solupdate_nb<100>(ctx, x, s);
    case 144: return solupdate_nb<144>(ctx, x, s);
    case 196: return solupdate_nb<196>(ctx, x, s);
    default: return set_error(ctx, FR_ERR_UNSUPPORTED, "block size %d not compiled", ctx->nb);
  }
}

}  // namespace frk

namespace frk {

size_t batch_apply_bytes() { return sizeof(BatchApply); }

unsigned apply_grid_of(fr_ctx* ctx) {
  long long g = 1;
  int rc = FR_OK;
  const int prec = ctx->opts.block_precision;
  switch (ctx->nb) {
    case 36: rc = prec == 1 ? apply_grid_nbs<36, float, float>(ctx, &g) : prec == 2 ? apply_grid_nbs<36, __nv_bfloat16, float>(ctx, &g) : apply_grid_nbs<36, double, double>(ctx, &g); break;
    case 64: rc = prec == 1 ? apply_grid_nbs<64, float, float>(ctx, &g) : prec == 2 ? apply_grid_nbs<64, __nv_bfloat16, float>(ctx, &g) : apply_grid_nbs<64, double, double>(ctx, &g); break;
    case 100: rc = prec == 1 ? apply_grid_nbs<100, float, float>(ctx, &g) : prec == 2 ? apply_grid_nbs<100, __nv_bfloat16, float>(ctx, &g) : apply_grid_nbs<100, double, double>(ctx, &g); break;
    default: return 0;
  }
  return rc == FR_OK ? (unsigned)g : 0u;
}

int fill_batch_apply(fr_ctx* ctx, BatchApply* t) {
  t->Minv = ctx->blocks;
  t->V = ctx->V;
  t->n = ctx->ndof;
  t->invh = ctx->gd.invh;
  t->z = ctx->z;
  t->ne = ctx->ne;
  t->sumsq = ctx->scal + S_NZ2;
  t->red = ctx->red;
  t->done = ctx->gd.done;
  t->ea = eps_args(ctx, true);
  t->kerr = ctx->kerr;
  t->polls = ctx->wait_polls;
  t->skip = ctx->test_skip_copy;
  return FR_OK;
}

namespace {
template <int NB, typename S, typename A>
int batch_apply_nbs(const BatchApply* tab, const int* start, int ninst, int nblocks, int j, cudaStream_t s) {
  using L = ApplyLayout<NB, S, A>;
  count_launch();
  kb_apply<NB, S, A><<<nblocks, L::THREADS, L::BYTES, s>>>(tab, start, ninst, j);
  return cudaGetLastError() == cudaSuccess ? FR_OK : FR_ERR_CUDA;
}
}  // namespace

int launch_batch_apply(int nb, int prec, const BatchApply* tab, const int* start, int ninst, int nblocks, int j,
                       cudaStream_t s) {
  switch (nb) {
    case 36: return prec == 1 ? batch_apply_nbs<36, float, float>(tab, start, ninst, nblocks, j, s) : prec == 2 ? batch_apply_nbs<36, __nv_bfloat16, float>(tab, start, ninst, nblocks, j, s) : batch_apply_nbs<36, double, double>(tab, start, ninst, nblocks, j, s);
    case 64: return prec == 1 ? batch_apply_nbs<64, float, float>(tab, start, ninst, nblocks, j, s) : prec == 2 ? batch_apply_nbs<64, __nv_bfloat16, float>(tab, start, ninst, nblocks, j, s) : batch_apply_nbs<64, double, double>(tab, start, ninst, nblocks, j, s);
    case 100: return prec == 1 ? batch_apply_nbs<100, float, float>(tab, start, ninst, nblocks, j, s) : prec == 2 ? batch_apply_nbs<100, __nv_bfloat16, float>(tab, start, ninst, nblocks, j, s) : batch_apply_nbs<100, double, double>(tab, start, ninst, nblocks, j, s);
    default: return FR_ERR_UNSUPPORTED;
  }
}

}  // namespace frk
