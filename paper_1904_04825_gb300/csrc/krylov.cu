// Restarted GMRES(m) of Sec. 4.5 on the device.
//
// Arnoldi uses classical Gram-Schmidt with one re-orthogonalisation pass
// (CGS2): every pass is one multi-dot kernel and one multi-AXPY kernel over
// the whole basis slice, with deterministic two-stage reductions.  The
// Hessenberg column, the Givens rotation and the convergence test run in a
// one-warp kernel, so a cycle of m iterations is launched without any host
// round trip: once the device sets `done`, the remaining kernels of the
// cycle return at once.  The host reads the cycle status once per restart.
#include <cmath>

#include "device.cuh"

namespace frk {
namespace {

unsigned vgrid(const fr_ctx* ctx, long long n) {
  long long g = (n + kThreads - 1) / kThreads;
  if (g > ctx->vec_blocks) g = ctx->vec_blocks;
  return (unsigned)(g < 1 ? 1 : g);
}

__global__ void k_sumsq(const double* __restrict__ x, long long n, double* out, Reduce red,
                        EpsArgs ea) {
  __shared__ double sh[32];
  double ss = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    ss = fma(x[i], x[i], ss);
  const double bs = block_sum(ss, sh);
  if (threadIdx.x == 0) red.partials[(size_t)blockIdx.x * kMaxVec] = bs;
  if (last_block(red.counter)) {
    finish_sums(red, 1, out);
    if (threadIdx.x == 0) write_eps(ea, *out);
  }
}

struct Lincomb {
  const double* x[8];
  double c[8];
  int n;
};

// out = sum_t c_t x_t (out may alias any x_t), optional sum of squares of out
__global__ void k_lincomb(double* out, long long len, const Lincomb lc, double* sumsq, Reduce red) {
  __shared__ double sh[32];
  double ss = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x) {
    double v = lc.c[0] * lc.x[0][i];
    for (int t = 1; t < lc.n; ++t) v = fma(lc.c[t], lc.x[t][i], v);
    out[i] = v;
    ss = fma(v, v, ss);
  }
  if (sumsq) {
    const double bs = block_sum(ss, sh);
    if (threadIdx.x == 0) red.partials[(size_t)blockIdx.x * kMaxVec] = bs;
    if (last_block(red.counter)) finish_sums(red, 1, sumsq);
  }
}

// One sweep over the rows accumulating NC dot products against w; the
// basis pointers are resolved outside the row loop so every row costs
// exactly NC fused multiply-adds on the FP64 pipe.  UR rows are in flight per
// thread (NC x UR independent accumulation chains hide the FMA latency).
template <int NC>
__device__ __forceinline__ void dots_chunk(const double* const* ptr, const double* __restrict__ w,
                                           long long n, double* acc, int bid, int nblk) {
  constexpr int UR = NC >= 8 ? 1 : (NC >= 4 ? 2 : 4);
  double a[NC][UR];
#pragma unroll
  for (int i = 0; i < NC; ++i)
#pragma unroll
    for (int u = 0; u < UR; ++u) a[i][u] = 0.0;
  const long long S = (long long)nblk * blockDim.x;
  for (long long r0 = (long long)bid * blockDim.x + threadIdx.x; r0 < n; r0 += UR * S) {
    double wr[UR];
#pragma unroll
    for (int u = 0; u < UR; ++u) wr[u] = (r0 + u * S < n) ? w[r0 + u * S] : 0.0;
#pragma unroll
    for (int i = 0; i < NC; ++i)
#pragma unroll
      for (int u = 0; u < UR; ++u)
        if (r0 + u * S < n) a[i][u] = fma(ptr[i][r0 + u * S], wr[u], a[i][u]);
  }
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    double s = a[i][0];
#pragma unroll
    for (int u = 1; u < UR; ++u) s += a[i][u];
    acc[i] = s;
  }
}

// out[i] = <V_i, w> for i < nvec, and out[nvec] = <w, w> when with_self,
// in chunks of up to 8 values per sweep.  Skipped when the cycle is done or
// when `gate` points at a zero flag.
__device__ __forceinline__ void dots_body(const double* __restrict__ V, long long ldv, int nvec,
                                          const double* __restrict__ w, long long n, double* out,
                                          int with_self, const Reduce& red, const int* done,
                                          const int* gate, int bid, int nblk) {
  __shared__ double sred[8][kThreads / 32];
  if ((done && *done) || (gate && !*gate)) return;
  const int total = nvec + (with_self ? 1 : 0);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c0 = 0; c0 < total; c0 += 8) {
    const int nc = min(8, total - c0);
    const double* ptr[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int idx = c0 + i;
      ptr[i] = idx < nvec ? V + (size_t)idx * ldv : w;
    }
    double acc[8];
    switch (nc) {
      case 1: dots_chunk<1>(ptr, w, n, acc, bid, nblk); break;
      case 2: dots_chunk<2>(ptr, w, n, acc, bid, nblk); break;
      case 3: dots_chunk<3>(ptr, w, n, acc, bid, nblk); break;
      case 4: dots_chunk<4>(ptr, w, n, acc, bid, nblk); break;
      case 5: dots_chunk<5>(ptr, w, n, acc, bid, nblk); break;
      case 6: dots_chunk<6>(ptr, w, n, acc, bid, nblk); break;
      case 7: dots_chunk<7>(ptr, w, n, acc, bid, nblk); break;
      default: dots_chunk<8>(ptr, w, n, acc, bid, nblk); break;
    }
    // Warp sums of the (up to) 8 values by recursive halving: each exchange
    // sends half of the values still held to the partner lane and keeps the
    // other half, so lane l ends with the warp sum of value
    // 4 b4 + 2 b3 + b2 (b = bits of l) after 9 additions instead of 8 x 5.
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (i >= nc) acc[i] = 0.0;
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double send = b4 ? acc[q] : acc[q + 4];
      const double keep = b4 ? acc[q + 4] : acc[q];
      acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const double send = b3 ? acc[q] : acc[q + 2];
      const double keep = b3 ? acc[q + 2] : acc[q];
      acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    {
      const double send = b2 ? acc[0] : acc[1];
      const double keep = b2 ? acc[1] : acc[0];
      acc[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 2);
    acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
    const int vi = (b4 ? 4 : 0) + (b3 ? 2 : 0) + (b2 ? 1 : 0);
    if ((lane & 3) == 0 && vi < nc) sred[vi][wid] = acc[0];
    __syncthreads();
    if ((int)threadIdx.x < nc) {
      double t = 0.0;
      for (int q = 0; q < nw; ++q) t += sred[threadIdx.x][q];
      red.partials[(size_t)bid * kMaxVec + c0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
  if (last_block(red.counter, nblk)) finish_sums(red, total, out, nblk);
}

__global__ void __launch_bounds__(256) k_dots(const double* __restrict__ V, long long ldv, int nvec,
                                              const double* __restrict__ w, long long n, double* out,
                                              int with_self, Reduce red, const int* done,
                                              const int* gate) {
  dots_body(V, ldv, nvec, w, n, out, with_self, red, done, gate, blockIdx.x, gridDim.x);
}

// w -= sum_i h_i V_i as one FMA chain per row (exactly nvec FP64 FMAs); optional sum of
// squares of the new w.  With `self2` (the first Gram-Schmidt pass) the last
// block also decides whether iteration j needs the second pass: it does when
// ||w_new|| < eta ||w_old|| (the test of Daniel, Gragg, Kaufman and Stewart;
// one classical pass leaves an orthogonality error of about
// u ||w_old|| / ||w_new||, so eta = 1/64 keeps it below ~64 u), recorded in
// rflag[j]; otherwise h2 is cleared.
struct Reorth {
  const double* self2;  // ||w||^2 before the first pass, or nullptr
  double eta2;          // second pass when ||w_new||^2 < eta2 ||w_old||^2
  int* rflag;           // &rflag[j]
  double* h2;
};

__device__ __forceinline__ void update_body(double* __restrict__ w, const double* __restrict__ V,
                                            long long ldv, int nvec, const double* h,
                                            long long n, double* sumsq, const Reduce& red,
                                            const int* done, const int* gate, const Reorth& ro,
                                            int bid, int nblk) {
  __shared__ double sh[32];
  __shared__ double hs[kMaxVec];
  if ((done && *done) || (gate && !*gate)) return;
  if (threadIdx.x < nvec) hs[threadIdx.x] = -h[threadIdx.x];
  __syncthreads();
  // four rows per thread in flight: four independent FMA chains of length nvec
  constexpr int UR = 4;
  double ss[UR] = {0.0, 0.0, 0.0, 0.0};
  const long long S = (long long)nblk * blockDim.x;
  for (long long r0 = (long long)bid * blockDim.x + threadIdx.x; r0 < n; r0 += UR * S) {
    double v[UR];
#pragma unroll
    for (int u = 0; u < UR; ++u) v[u] = (r0 + u * S < n) ? w[r0 + u * S] : 0.0;
    for (int i = 0; i < nvec; ++i) {
      const double hi = hs[i];
      const double* Vi = V + i * ldv;
#pragma unroll
      for (int u = 0; u < UR; ++u)
        if (r0 + u * S < n) v[u] = fma(hi, Vi[r0 + u * S], v[u]);
    }
#pragma unroll
    for (int u = 0; u < UR; ++u) {
      if (r0 + u * S < n) {
        w[r0 + u * S] = v[u];
        if (sumsq) ss[u] = fma(v[u], v[u], ss[u]);
      }
    }
  }
  if (sumsq) {
    const double bs = block_sum((ss[0] + ss[1]) + (ss[2] + ss[3]), sh);
    if (threadIdx.x == 0) red.partials[(size_t)bid * kMaxVec] = bs;
    if (last_block(red.counter, nblk)) {
      finish_sums(red, 1, sumsq, nblk);
      if (ro.self2 && threadIdx.x == 0) {
        const int need = (*sumsq < ro.eta2 * *ro.self2) ? 1 : 0;
        *ro.rflag = need;
        if (!need)
          for (int q = 0; q < nvec; ++q) ro.h2[q] = 0.0;
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_update(double* __restrict__ w, const double* __restrict__ V,
                                                long long ldv, int nvec, const double* h,
                                                long long n, double* sumsq, Reduce red,
                                                const int* done, const int* gate, Reorth ro) {
  update_body(w, V, ldv, nvec, h, n, sumsq, red, done, gate, ro, blockIdx.x, gridDim.x);
}

// start of a cycle: beta = ||r||, g = beta e_1, done if beta <= rtol ||b||
__global__ void k_cycle_init(GmresDev gd, const double* nr2, const double* nb2, double rtol, int m,
                             const int* fin) {
  if (threadIdx.x != 0) return;
  if (fin && *fin) {  // solve already finished: the whole cycle is skipped
    *gd.k = 0;
    *gd.done = 1;
    return;
  }
  const double beta = sqrt(*nr2);
  const double target = rtol * sqrt(*nb2);
  for (int i = 0; i <= m; ++i) gd.g[i] = 0.0;
  gd.g[0] = beta;
  *gd.target = target;
  *gd.res = beta;
  *gd.k = 0;
  *gd.done = (beta <= target) ? 1 : 0;
  for (int i = 0; i < m; ++i) gd.rflag[i] = 0;
  gd.invh[0] = beta > 0.0 ? 1.0 / beta : 0.0;
}

// Hessenberg column j, Givens rotations, residual estimate, convergence.
// One warp: the lanes bring the column's Gram-Schmidt coefficients and the
// earlier rotations into shared memory together (one round of independent
// loads instead of a chain of dependent ones), lane 0 applies the rotations
// in order, and the lanes write the column back.
__device__ __forceinline__ void givens_body(const GmresDev& gd, int j, const double* nw2) {
  __shared__ double hs[kMaxVec + 1], cs_s[kMaxVec], sn_s[kMaxVec];
  if (*gd.done) return;
  const int lane = threadIdx.x & 31;
  for (int i = lane; i <= j; i += 32) hs[i] = gd.h1[i] + gd.h2[i];
  for (int i = lane; i < j; i += 32) {
    cs_s[i] = gd.cs[i];
    sn_s[i] = gd.sn[i];
  }
  __syncwarp();
  if (lane == 0) {
    const double hn = sqrt(*nw2);
    hs[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
      const double t = cs_s[i] * hs[i] + sn_s[i] * hs[i + 1];
      hs[i + 1] = -sn_s[i] * hs[i] + cs_s[i] * hs[i + 1];
      hs[i] = t;
    }
    const double den = hypot(hs[j], hs[j + 1]);
    const double c = den > 0.0 ? hs[j] / den : 1.0;
    const double s = den > 0.0 ? hs[j + 1] / den : 0.0;
    gd.cs[j] = c;
    gd.sn[j] = s;
    hs[j] = den;
    hs[j + 1] = 0.0;
    gd.g[j + 1] = -s * gd.g[j];
    gd.g[j] = c * gd.g[j];
    *gd.k = j + 1;
    const double res = fabs(gd.g[j + 1]);
    *gd.res = res;
    gd.invh[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
    if (res <= *gd.target || hn == 0.0 || !(res == res)) *gd.done = 1;
  }
  __syncwarp();
  double* Hj = gd.H + (size_t)j * gd.ldh;
  for (int i = lane; i <= j + 1; i += 32) Hj[i] = hs[i];
}

__global__ void k_givens(GmresDev gd, int j, const double* nw2) {
  givens_body(gd, j, nw2);
}

// y = H(0:k,0:k)^{-1} g(0:k); one warp loads the triangle, lane 0 solves
__global__ void k_backsub(GmresDev gd) {
  __shared__ double Hs[kMaxVec][kMaxVec];
  __shared__ double ys[kMaxVec];
  const int k = *gd.k;
  const int lane = threadIdx.x & 31;
  for (int idx = lane; idx < k * k; idx += 32) {
    const int l = idx / k, i = idx % k;   // column l, row i
    if (i <= l) Hs[l][i] = gd.H[(size_t)l * gd.ldh + i];
  }
  for (int i = lane; i < k; i += 32) ys[i] = gd.g[i];
  __syncwarp();
  if (lane == 0) {
    for (int i = k - 1; i >= 0; --i) {
      double s = ys[i];
      for (int l = i + 1; l < k; ++l) s -= Hs[l][i] * ys[l];
      ys[i] = s / Hs[i][i];
    }
  }
  __syncwarp();
  for (int i = lane; i < k; i += 32) gd.y[i] = ys[i];
}

// cycle status for the host: [k, |g_k|, rtol ||b||, ||b||]; marks the
// solve finished once the residual met the target
__global__ void k_status(GmresDev gd, const double* nb2, double* out, int* fin, const int* kerr) {
  if (threadIdx.x != 0) return;
  if (*kerr) {  // a bounded wait gave up in this cycle
    out[0] = -1.0;
    return;
  }
  if (fin) {
    if (*fin) {
      out[0] = 0.0;
      return;
    }
    if (*gd.res <= *gd.target) *fin = 1;
  }
  out[0] = (double)*gd.k;
  out[1] = *gd.res;
  out[2] = *gd.target;
  out[3] = sqrt(*nb2);
}

__global__ void k_copy(double* dst, const double* src, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

__global__ void k_fill(double* dst, double v, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = v;
}

// ---- batched Arnoldi-step kernels: the CTAs of every instance in one grid,
// instance k owning blocks [start[k], start[k+1]) (the same partition as its
// single-instance launch, so every reduction sums in the same order) ----
__global__ void __launch_bounds__(256) kb_dots(const BatchKrylov* __restrict__ tab, const int* __restrict__ start,
                                               int ninst, int j, int second) {
  const int k = batch_instance(start, ninst, blockIdx.x);
  const BatchKrylov& t = tab[k];
  const int bid = blockIdx.x - start[k], nblk = start[k + 1] - start[k];
  const long long n = t.n;
  dots_body(t.V, n, j + 1, t.V + (size_t)(j + 1) * n, n, second ? t.gd.h2 : t.gd.h1, second ? 0 : 1, t.red,
            t.gd.done, second ? t.gd.rflag + j : nullptr, bid, nblk);
}

__global__ void __launch_bounds__(256) kb_update(const BatchKrylov* __restrict__ tab, const int* __restrict__ start,
                                                 int ninst, int j, int second) {
  const int k = batch_instance(start, ninst, blockIdx.x);
  const BatchKrylov& t = tab[k];
  const int bid = blockIdx.x - start[k], nblk = start[k + 1] - start[k];
  const long long n = t.n;
  const Reorth none{nullptr, 0.0, nullptr, nullptr};
  const Reorth first{t.gd.h1 + (j + 1), t.eta2, t.gd.rflag + j, t.gd.h2};
  update_body(t.V + (size_t)(j + 1) * n, t.V, n, j + 1, second ? t.gd.h2 : t.gd.h1, n, t.nw2, t.red, t.gd.done,
              second ? t.gd.rflag + j : nullptr, second ? none : first, bid, nblk);
}

__global__ void kb_givens(const BatchKrylov* __restrict__ tab, int j) {
  const BatchKrylov& t = tab[blockIdx.x];
  givens_body(t.gd, j, t.nw2);
}

}  // namespace

BatchKrylov batch_krylov_args(fr_ctx* ctx) {
  BatchKrylov t;
  t.V = ctx->V;
  t.n = ctx->ndof;
  t.gd = ctx->gd;
  t.red = ctx->red;
  t.nw2 = ctx->scal + S_NW2;
  t.eta2 = ctx->opts.reorth_eta * ctx->opts.reorth_eta;
  return t;
}

unsigned vec_grid_of(const fr_ctx* ctx) { return vgrid(ctx, ctx->ndof); }

// The Gram-Schmidt passes and the Givens step of Arnoldi iteration j of every
// instance of a batch: tab / start describe the instances (device arrays),
// nblocks = start[ninst].
int launch_batch_gs_givens(const BatchKrylov* tab, const int* start, int ninst, int nblocks, int j, cudaStream_t s) {
  count_launches(5);
  kb_dots<<<nblocks, kThreads, 0, s>>>(tab, start, ninst, j, 0);
  kb_update<<<nblocks, kThreads, 0, s>>>(tab, start, ninst, j, 0);
  kb_dots<<<nblocks, kThreads, 0, s>>>(tab, start, ninst, j, 1);
  kb_update<<<nblocks, kThreads, 0, s>>>(tab, start, ninst, j, 1);
  kb_givens<<<ninst, 32, 0, s>>>(tab, j);
  return cudaGetLastError() == cudaSuccess ? FR_OK : FR_ERR_CUDA;
}

EpsArgs eps_args(fr_ctx* ctx, bool on) {
  EpsArgs ea{ctx->scal + S_NU2, ctx->opts.eps_rel, ctx->opts.eps_fixed, on ? ctx->scal + S_EPS : nullptr};
  return ea;
}

int launch_sumsq(fr_ctx* ctx, const double* x, double* out, cudaStream_t s, bool with_eps) {
  { ProfScope ps_(ctx, FR_KF_OTHER, s); k_sumsq<<<vgrid(ctx, ctx->ndof), kThreads, 0, s>>>(x, ctx->ndof, out, ctx->red, eps_args(ctx, with_eps)); }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

int launch_lincomb(fr_ctx* ctx, double* out, int nterms, const double* const* xs,
                   const double* coefs, double* sumsq, cudaStream_t s) {
  if (nterms < 1 || nterms > 8) return set_error(ctx, FR_ERR_INVALID_ARG, "lincomb of %d terms", nterms);
  Lincomb lc{};
  lc.n = nterms;
  for (int t = 0; t < nterms; ++t) {
    lc.x[t] = xs[t];
    lc.c[t] = coefs[t];
  }
  { ProfScope ps_(ctx, FR_KF_OTHER, s); k_lincomb<<<vgrid(ctx, ctx->ndof), kThreads, 0, s>>>(out, ctx->ndof, lc, sumsq, ctx->red); }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

int launch_copy(fr_ctx* ctx, double* dst, const double* src, cudaStream_t s) {
  { ProfScope ps_(ctx, FR_KF_OTHER, s); k_copy<<<vgrid(ctx, ctx->ndof), kThreads, 0, s>>>(dst, src, ctx->ndof); }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

int launch_fill(fr_ctx* ctx, double* dst, double v, cudaStream_t s) {
  { ProfScope ps_(ctx, FR_KF_OTHER, s); k_fill<<<vgrid(ctx, ctx->ndof), kThreads, 0, s>>>(dst, v, ctx->ndof); }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

// One whole GMRES cycle enqueued without any host synchronisation (for CUDA
// graph capture): r = b - A x (exactly b for x = 0), m Arnoldi iterations
// that stop on the device, the solution update, and the status
// [k, |g_k|, target, ||b||] written to status (device, 4 doubles).  The three
// parts are also enqueued separately by batches, whose Arnoldi iterations
// run as batched launches over all instances.
int gmres_cycle_prologue(fr_ctx* ctx, const double* U, const double* R0, double shift, const double* b,
                         double* x, int m, double rtol, int* fin, cudaStream_t s) {
  double* sc = ctx->scal;
  FRK_TRY(launch_linearize(ctx, U, s));
  FRK_TRY(launch_sumsq(ctx, U, sc + S_NU2, s));
  FRK_TRY(launch_sumsq(ctx, b, sc + S_NB2, s));
  FRK_TRY(launch_sumsq(ctx, x, sc + S_NZ2, s, true));
  FRK_TRY(launch_residual(ctx, 2, U, x, R0, b, ctx->V, shift, sc + S_EPS, fin, s));
  FRK_TRY(launch_sumsq(ctx, ctx->V, sc + S_NR2, s));
  { ProfScope ps_(ctx, FR_KF_OTHER, s); k_cycle_init<<<1, 32, 0, s>>>(ctx->gd, sc + S_NR2, sc + S_NB2, rtol, m, fin); }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

int gmres_cycle_epilogue(fr_ctx* ctx, double* x, double* status, int* fin, cudaStream_t s) {
  GmresDev& gd = ctx->gd;
  { ProfScope ps_(ctx, FR_KF_OTHER, s); k_backsub<<<1, 32, 0, s>>>(gd); }
  FRK_LAUNCHED(ctx);
  FRK_TRY(launch_solution_update(ctx, x, s));
  { ProfScope ps_(ctx, FR_KF_OTHER, s); k_status<<<1, 32, 0, s>>>(gd, ctx->scal + S_NB2, status, fin, ctx->kerr); }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

int gmres_cycle_enqueue(fr_ctx* ctx, const double* U, const double* R0, double shift, const double* b,
                        double* x, int m, double rtol, double* status, int* fin, cudaStream_t s) {
  const long long n = ctx->ndof;
  double* sc = ctx->scal;
  GmresDev& gd = ctx->gd;
  double* V = ctx->V;
  FRK_TRY(gmres_cycle_prologue(ctx, U, R0, shift, b, x, m, rtol, fin, s));
  for (int j = 0; j < m; ++j) {
    double* vj = V + (size_t)j * n;
    double* w = V + (size_t)(j + 1) * n;
    FRK_TRY(launch_block_apply(ctx, vj, gd.invh + j, ctx->z, sc + S_NZ2, gd.done, s, true));
    FRK_TRY(launch_residual(ctx, 1, U, ctx->z, R0, nullptr, w, shift, sc + S_EPS, gd.done, s));
    const Reorth none{nullptr, 0.0, nullptr, nullptr};
    const Reorth first{gd.h1 + (j + 1), ctx->opts.reorth_eta * ctx->opts.reorth_eta, gd.rflag + j, gd.h2};
    { ProfScope ps_(ctx, FR_KF_DOTS, s); k_dots<<<vgrid(ctx, n), kThreads, 0, s>>>(V, n, j + 1, w, n, gd.h1, 1, ctx->red, gd.done, nullptr); }
    { ProfScope ps_(ctx, FR_KF_UPDATE, s); k_update<<<vgrid(ctx, n), kThreads, 0, s>>>(w, V, n, j + 1, gd.h1, n, sc + S_NW2, ctx->red, gd.done, nullptr, first); }
    { ProfScope ps_(ctx, FR_KF_DOTS, s); k_dots<<<vgrid(ctx, n), kThreads, 0, s>>>(V, n, j + 1, w, n, gd.h2, 0, ctx->red, gd.done, gd.rflag + j); }
    { ProfScope ps_(ctx, FR_KF_UPDATE, s); k_update<<<vgrid(ctx, n), kThreads, 0, s>>>(w, V, n, j + 1, gd.h2, n, sc + S_NW2, ctx->red, gd.done, gd.rflag + j, none); }
    { ProfScope ps_(ctx, FR_KF_OTHER, s); k_givens<<<1, 32, 0, s>>>(gd, j, sc + S_NW2); }
    FRK_LAUNCHED(ctx);
  }
  return gmres_cycle_epilogue(ctx, x, status, fin, s);
}

int gmres_impl(fr_ctx* ctx, const double* U, const double* R0, double shift, const double* b,
               double* x, int m, double rtol, int max_restarts, bool x_is_zero,
               fr_gmres_info* info, cudaStream_t s) {
  const long long n = ctx->ndof;
  double* sc = ctx->scal;
  GmresDev& gd = ctx->gd;
  double* V = ctx->V;
  fr_gmres_info loc{};
  FRK_TRY(launch_linearize(ctx, U, s));
  // ||U|| for the FD step, ||b|| for the stopping test
  FRK_TRY(launch_sumsq(ctx, U, sc + S_NU2, s));
  FRK_TRY(launch_sumsq(ctx, b, sc + S_NB2, s));
  if (!x_is_zero) {
    FRK_TRY(launch_sumsq(ctx, x, sc + S_NX2, s));
    FRK_CUDA(ctx, cudaMemcpyAsync(ctx->h_scal, sc + S_NB2, sizeof(double), cudaMemcpyDeviceToHost, s));
    FRK_CUDA(ctx, cudaMemcpyAsync(ctx->h_scal + 1, sc + S_NX2, sizeof(double),
                                  cudaMemcpyDeviceToHost, s));
    FRK_CUDA(ctx, cudaStreamSynchronize(s));
    if (ctx->h_scal[0] == 0.0) {  // b = 0: the solution is x = 0
      FRK_TRY(launch_fill(ctx, x, 0.0, s));
      loc.converged = 1;
      if (info) *info = loc;
      return FR_OK;
    }
    x_is_zero = ctx->h_scal[1] == 0.0;
  }
  int cycles_iterated = 0;
  int status = FR_ERR_NOT_CONVERGED;
  for (int cycle = 0; cycle <= max_restarts; ++cycle) {
    // r = b - A x into V[0]
    if (cycle == 0 && x_is_zero) {
      FRK_TRY(launch_copy(ctx, V, b, s));
    } else {
      FRK_TRY(launch_sumsq(ctx, x, sc + S_NZ2, s, true));
      FRK_TRY(launch_residual(ctx, 2, U, x, R0, b, V, shift, sc + S_EPS, nullptr, s));
    }
    FRK_TRY(launch_sumsq(ctx, V, sc + S_NR2, s));
    { ProfScope ps_(ctx, FR_KF_OTHER, s); k_cycle_init<<<1, 32, 0, s>>>(gd, sc + S_NR2, sc + S_NB2, rtol, m, nullptr); }
    FRK_LAUNCHED(ctx);
    // Launch the cycle in chunks of kChunk iterations; after launching chunk
    // c, wait for the finished-flag copied after chunk c-1, so the device
    // always has queued work and at most one chunk runs past convergence.
    constexpr int kChunk = 4;
    int launched = 0, chunk = 0;
    while (launched < m) {
      const int jend = launched + kChunk < m ? launched + kChunk : m;
      for (int j = launched; j < jend; ++j) {
        double* vj = V + (size_t)j * n;
        double* w = V + (size_t)(j + 1) * n;
        // v_j = r_j / ||r_j|| (written back), z = M^{-1} v_j, ||z||^2
        FRK_TRY(launch_block_apply(ctx, vj, gd.invh + j, ctx->z, sc + S_NZ2, gd.done, s, true));
        // w = A z
        FRK_TRY(launch_residual(ctx, 1, U, ctx->z, R0, nullptr, w, shift, sc + S_EPS, gd.done, s));
        // Gram-Schmidt: one classical pass, a second one only when the
        // first shrank ||w|| below reorth_eta ||w|| (decided on the device)
        const Reorth none{nullptr, 0.0, nullptr, nullptr};
        const Reorth first{gd.h1 + (j + 1), ctx->opts.reorth_eta * ctx->opts.reorth_eta, gd.rflag + j, gd.h2};
        { ProfScope ps_(ctx, FR_KF_DOTS, s); k_dots<<<vgrid(ctx, n), kThreads, 0, s>>>(V, n, j + 1, w, n, gd.h1, 1, ctx->red, gd.done, nullptr); }
        { ProfScope ps_(ctx, FR_KF_UPDATE, s); k_update<<<vgrid(ctx, n), kThreads, 0, s>>>(w, V, n, j + 1, gd.h1, n, sc + S_NW2, ctx->red, gd.done, nullptr, first); }
        { ProfScope ps_(ctx, FR_KF_DOTS, s); k_dots<<<vgrid(ctx, n), kThreads, 0, s>>>(V, n, j + 1, w, n, gd.h2, 0, ctx->red, gd.done, gd.rflag + j); }
        { ProfScope ps_(ctx, FR_KF_UPDATE, s); k_update<<<vgrid(ctx, n), kThreads, 0, s>>>(w, V, n, j + 1, gd.h2, n, sc + S_NW2, ctx->red, gd.done, gd.rflag + j, none); }
        { ProfScope ps_(ctx, FR_KF_OTHER, s); k_givens<<<1, 32, 0, s>>>(gd, j, sc + S_NW2); }
        FRK_LAUNCHED(ctx);
      }
      launched = jend;
      const int slot = chunk & 1;
      FRK_CUDA(ctx, cudaMemcpyAsync(ctx->h_stat + 2 + slot, gd.done, sizeof(int), cudaMemcpyDeviceToHost, s));
      FRK_CUDA(ctx, cudaEventRecord(ctx->chunk_ev[slot], s));
      ++chunk;
      if (chunk >= 2) {
        const int prev = (chunk - 2) & 1;
        FRK_CUDA(ctx, cudaEventSynchronize(ctx->chunk_ev[prev]));
        if (ctx->h_stat[2 + prev]) break;
      }
    }
    { ProfScope ps_(ctx, FR_KF_OTHER, s); k_backsub<<<1, 32, 0, s>>>(gd); }
    FRK_LAUNCHED(ctx);
    FRK_TRY(launch_solution_update(ctx, x, s));
    FRK_CUDA(ctx, cudaMemcpyAsync(ctx->h_stat, gd.k, sizeof(int), cudaMemcpyDeviceToHost, s));
    FRK_CUDA(ctx, cudaMemcpyAsync(ctx->h_stat + 4, gd.rflag, m * sizeof(int), cudaMemcpyDeviceToHost, s));
    FRK_CUDA(ctx, cudaMemcpyAsync(ctx->h_scal, gd.res, sizeof(double), cudaMemcpyDeviceToHost, s));
    FRK_CUDA(ctx, cudaMemcpyAsync(ctx->h_scal + 1, gd.target, sizeof(double), cudaMemcpyDeviceToHost, s));
    FRK_CUDA(ctx, cudaMemcpyAsync(ctx->h_scal + 2, sc + S_NB2, sizeof(double), cudaMemcpyDeviceToHost, s));
    FRK_CUDA(ctx, cudaMemcpyAsync(ctx->h_stat + 1, ctx->kerr, sizeof(int), cudaMemcpyDeviceToHost, s));
    FRK_CUDA(ctx, cudaStreamSynchronize(s));
    if (ctx->h_stat[1]) return set_error(ctx, FR_ERR_TIMEOUT, "a kernel's bounded wait for its copies gave up");
    const int k = ctx->h_stat[0];
    const double res = ctx->h_scal[0], target = ctx->h_scal[1], bn = std::sqrt(ctx->h_scal[2]);
    {  // launches of this cycle that found it finished (for per-launch timing),
       // and the algorithmic work of the k iterations that ran: apply (blocks +
       // r in, r and z out), A z (U, z, R0 in, w out), CGS2 (two multi-dots
       // reading j+1 basis vectors and w, two updates reading them and
       // reading/writing w)
      const long long sk = launched - k;
      const double nd = (double)n;
      long long second = 0;
      for (int j = 0; j < k; ++j) {
        const double kv = j + 1;
        const int re = ctx->h_stat[4 + j];
        second += re;
        if (ctx->opts.precond)
          prof_work(ctx, FR_KF_APPLY, 8.0 * (double)ctx->ne * ctx->nb * ctx->nb + 24.0 * nd, 2.0 * ctx->nb * nd);
        else
          prof_work(ctx, FR_KF_APPLY, 24.0 * nd, 3.0 * nd);
        prof_work(ctx, FR_KF_JV, 32.0 * nd, jv_flops_per_element(ctx) * (double)ctx->ne + 6.0 * nd);
        // pass 1: dots of j+1 basis vectors and w with w; update reads them and w, writes w
        prof_work(ctx, FR_KF_DOTS, 8.0 * (kv + 1) * nd, 2.0 * (kv + 1) * nd);
        prof_work(ctx, FR_KF_UPDATE, 8.0 * (kv + 2) * nd, 2.0 * kv * nd + 2.0 * nd);
        if (re) {
          prof_work(ctx, FR_KF_DOTS, 8.0 * (kv + 1) * nd, 2.0 * kv * nd);
          prof_work(ctx, FR_KF_UPDATE, 8.0 * (kv + 2) * nd, 2.0 * kv * nd + 2.0 * nd);
        }
      }
      Prof& P = ctx->prof;
      P.skipped[FR_KF_APPLY] += sk;
      P.skipped[FR_KF_JV] += sk;
      P.skipped[FR_KF_DOTS] += 2 * sk + (k - second);
      P.skipped[FR_KF_UPDATE] += 2 * sk + (k - second);
      P.skipped[FR_KF_OTHER] += sk;
    }
    if (!std::isfinite(res) || !std::isfinite(bn)) {
      if (info) *info = loc;
      return set_error(ctx, FR_ERR_NONFINITE, "GMRES residual is not finite");
    }
    if (bn == 0.0) {  // b = 0 and x = 0 on entry
      loc.converged = 1;
      loc.relres = 0.0;
      status = FR_OK;
      break;
    }
    loc.iters += k;
    if (k > 0) ++cycles_iterated;
    loc.relres = res / bn;
    if (res <= target) {
      loc.converged = 1;
      status = FR_OK;
      break;
    }
  }
  loc.restarts = cycles_iterated > 0 ? cycles_iterated - 1 : 0;
  if (info) *info = loc;
  if (status != FR_OK)
    set_error(ctx, FR_ERR_NOT_CONVERGED, "GMRES stopped after %d iterations at relres %.3e",
              loc.iters, loc.relres);
  return status;
}

}  // namespace frk
