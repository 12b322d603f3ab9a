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
#include "device.cuh"

namespace frk {
namespace {

struct FactorArgs {
  const double* U;
  double* blocks;    // [ne][nb][nb], column-major inverse per element: Minv[k*nb + i]
  const double* hx;
  const double* hy;
  long long ne;
  int nx, ny;
  double gam;
  double shift;
  double beps;       // block_eps_rel
  Tables tab;
};

template <int P>
struct FactorLayout {
  static constexpr int N = P + 1, NP = N * N, NB = 4 * NP, LD = NB + 1;
  static constexpr int THREADS = NB <= 64 ? 128 : 256;
  // shared memory (doubles)
  static constexpr int OFF_M = 0;                       // NB x LD
  static constexpr int OFF_Q = OFF_M + NB * LD;         // 4 x NP state
  static constexpr int OFF_F = OFF_Q + 4 * NP;          // 4 x NP  (hy/2) f
  static constexpr int OFF_G = OFF_F + 4 * NP;          // 4 x NP  (hx/2) g
  static constexpr int OFF_TR = OFF_G + 4 * NP;         // own traces [4 faces][4 vars][N]
  static constexpr int OFF_NT = OFF_TR + 16 * N;        // neighbour traces [4][4][N]
  static constexpr int OFF_FN = OFF_NT + 16 * N;        // base common fluxes [4][4][N] (scaled)
  static constexpr int OFF_COL = OFF_FN + 16 * N;       // pivot column NB
  static constexpr int TOTAL = OFF_COL + NB;
  static constexpr size_t BYTES = TOTAL * sizeof(double) + 2 * NB * sizeof(int) + 64;
};

template <int N>
__device__ __forceinline__ double tsum(const double* x, int stride, const double* c) {
  double s = c[0] * x[0];
#pragma unroll
  for (int k = 1; k < N; ++k) s = fma(c[k], x[k * stride], s);
  return s;
}

template <int P>
__global__ void __launch_bounds__(FactorLayout<P>::THREADS) k_factor(const FactorArgs a) {
  using L = FactorLayout<P>;
  constexpr int N = L::N, NP = L::NP, NB = L::NB, LD = L::LD;
  extern __shared__ double smem[];
  double* M = smem + L::OFF_M;
  double* q = smem + L::OFF_Q;
  double* F = smem + L::OFF_F;
  double* G = smem + L::OFF_G;
  double* tr = smem + L::OFF_TR;
  double* nt = smem + L::OFF_NT;
  double* fn = smem + L::OFF_FN;
  double* col = smem + L::OFF_COL;
  int* piv = reinterpret_cast<int*>(smem + L::TOTAL);
  __shared__ int s_prow;

  const long long e = blockIdx.x;
  const int ix = (int)(e % a.nx), iy = (int)(e / a.nx);
  const double hx = a.hx[ix], hy = a.hy[iy];
  const double sJ = 4.0 / (hx * hy);
  const Tables& T = a.tab;

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
    const double* co = (face == 0 || face == 2) ? T.lm : T.lp;
    const double* cn = (face == 0 || face == 2) ? T.lp : T.lm;
    double qo[4], qn[4], fc[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      qo[v] = tsum<N>(q + v * NP + off, stride, co);
      qn[v] = tsum<N>(a.U + nbr * NB + v * NP + off, stride, cn);
      tr[(face * 4 + v) * N + k] = qo[v];
      nt[(face * 4 + v) * N + k] = qn[v];
    }
    const int dir = face < 2 ? 0 : 1;
    if (face == 0 || face == 2) rusanov(qn, qo, dir, a.gam, fc);
    else rusanov(qo, qn, dir, a.gam, fc);
    const double sc = face < 2 ? 0.5 * hy : 0.5 * hx;
#pragma unroll
    for (int v = 0; v < 4; ++v) fn[(face * 4 + v) * N + k] = sc * fc[v];
  }
  __syncthreads();

  // ---- columns of M = shift*I - J_ee ----
  for (int c = threadIdx.x; c < NB; c += blockDim.x) {
    const int vv = c / NP, pt = c % NP, ia = pt % N, jb = pt / N;
    double* Mc = M + c;  // column c, row stride LD
    for (int r = 0; r < NB; ++r) Mc[r * LD] = (r == c) ? a.shift : 0.0;
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
      const double cf = face == 0 ? T.lm[ia] : face == 1 ? T.lp[ia] : face == 2 ? T.lm[jb] : T.lp[jb];
      double qo[4], qn[4], fc[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        qo[v] = tr[(face * 4 + v) * N + k];
        qn[v] = nt[(face * 4 + v) * N + k];
      }
      qo[vv] = fma(cf, eps, qo[vv]);
      const int dir = face < 2 ? 0 : 1;
      if (face == 0 || face == 2) rusanov(qn, qo, dir, a.gam, fc);
      else rusanov(qo, qn, dir, a.gam, fc);
      const double sc = face < 2 ? 0.5 * hy : 0.5 * hx;
#pragma unroll
      for (int v = 0; v < 4; ++v) dFn[face][v] = sc * fc[v] - fn[(face * 4 + v) * N + k];
    }
    // row jb: points (i, jb), x-direction change
    for (int i = 0; i < N; ++i) {
      const int pnt = i + N * jb;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double d = T.Dt[i][ia] * dF[v];
        d = fma(T.dgL[i], dFn[0][v], d);
        d = fma(T.dgR[i], dFn[1][v], d);
        Mc[(v * NP + pnt) * LD] += sJ * d * inv;   // M = shift I - J, J = -sJ * d / eps
      }
    }
    // column ia: points (ia, j), y-direction change
    for (int j = 0; j < N; ++j) {
      const int pnt = ia + N * j;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double d = T.Dt[j][jb] * dG[v];
        d = fma(T.dgL[j], dFn[2][v], d);
        d = fma(T.dgR[j], dFn[3][v], d);
        Mc[(v * NP + pnt) * LD] += sJ * d * inv;
      }
    }
  }
  __syncthreads();

  // ---- in-place Gauss-Jordan inversion with partial (row) pivoting ----
  for (int k = 0; k < NB; ++k) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = k;
      for (int r = k + (int)threadIdx.x; r < NB; r += 32) {
        const double val = fabs(M[r * LD + k]);
        if (val > best) { best = val; bi = r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) { s_prow = bi; piv[k] = bi; }
    }
    __syncthreads();
    const int r = s_prow;
    if (r != k) {
      for (int jj = threadIdx.x; jj < NB; jj += blockDim.x) {
        const double tmp = M[k * LD + jj];
        M[k * LD + jj] = M[r * LD + jj];
        M[r * LD + jj] = tmp;
      }
    }
    __syncthreads();
    for (int ii = threadIdx.x; ii < NB; ii += blockDim.x) col[ii] = M[ii * LD + k];
    __syncthreads();
    const double pinv = 1.0 / col[k];
    for (int jj = threadIdx.x; jj < NB; jj += blockDim.x)
      M[k * LD + jj] = (jj == k ? 1.0 : M[k * LD + jj]) * pinv;
    __syncthreads();
    for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
      const int ii = idx / NB, jj = idx % NB;
      if (ii == k) continue;
      M[ii * LD + jj] = (jj == k ? 0.0 : M[ii * LD + jj]) - col[ii] * M[k * LD + jj];
    }
    __syncthreads();
  }
  for (int k = NB - 1; k >= 0; --k) {
    const int r = piv[k];
    if (r != k) {
      for (int ii = threadIdx.x; ii < NB; ii += blockDim.x) {
        const double tmp = M[ii * LD + k];
        M[ii * LD + k] = M[ii * LD + r];
        M[ii * LD + r] = tmp;
      }
    }
    __syncthreads();
  }
  // ---- store column-major: Minv[k*NB + i] = inverse(i, k) ----
  double* out = a.blocks + e * (long long)NB * NB;
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
    const int kk = idx / NB, ii = idx % NB;
    out[idx] = M[ii * LD + kk];
  }
}

// z = Minv r (optionally r scaled by *scale first and written back), optional
// sum of squares of z.  EPC elements per CTA, one thread per block row.
template <int NB>
__global__ void __launch_bounds__(256) k_apply(const double* __restrict__ Minv, double* r,
                                               const double* scale, double* __restrict__ z,
                                               long long ne, double* sumsq, Reduce red,
                                               const int* done, EpsArgs ea) {
  constexpr int EPC = 256 / NB;
  __shared__ double rs[EPC][NB];
  __shared__ double sh[32];
  if (done && *done) return;
  const int el = threadIdx.x / NB, i = threadIdx.x % NB;
  const double s = scale ? *scale : 1.0;
  double ss = 0.0;
  for (long long e0 = (long long)blockIdx.x * EPC; e0 < ne; e0 += (long long)gridDim.x * EPC) {
    const long long e = e0 + el;
    const bool act = el < EPC && e < ne;
    __syncthreads();
    if (act) {
      double v = r[e * NB + i];
      if (scale) {
        v *= s;
        r[e * NB + i] = v;
      }
      rs[el][i] = v;
    }
    __syncthreads();
    if (act) {
      const double* Me = Minv + e * (long long)NB * NB;
      double acc0 = 0.0, acc1 = 0.0;
#pragma unroll 8
      for (int k = 0; k < NB; k += 2) {
        acc0 = fma(Me[k * NB + i], rs[el][k], acc0);
        if (k + 1 < NB) acc1 = fma(Me[(k + 1) * NB + i], rs[el][k + 1], acc1);
      }
      const double zi = acc0 + acc1;
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
template <int NB>
__global__ void __launch_bounds__(256) k_solupdate(const double* __restrict__ Minv,
                                                   const double* __restrict__ V, long long ldv,
                                                   const double* y, const int* kp, double* x,
                                                   long long ne) {
  constexpr int EPC = 256 / NB;
  __shared__ double ts[EPC][NB];
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
      ts[el][i] = t;
    }
    __syncthreads();
    if (act) {
      const double* Me = Minv + e * (long long)NB * NB;
      double acc = 0.0;
      for (int kk = 0; kk < NB; ++kk) acc = fma(Me[kk * NB + i], ts[el][kk], acc);
      x[e * NB + i] += acc;
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

template <int P>
int factor_p(fr_ctx* ctx, const FactorArgs& a, cudaStream_t s) {
  using L = FactorLayout<P>;
  FRK_CUDA(ctx, cudaFuncSetAttribute(k_factor<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)L::BYTES));
  // work: read U (8 B/DOF), write ne nb^2 doubles; flops per element as counted
  const double fb = 8.0 * (double)ctx->ndof + 8.0 * (double)ctx->ne * L::NB * L::NB;
  const double ff = factor_flops_per_element(P) * (double)ctx->ne;
  { ProfScope ps_(ctx, FR_KF_FACTOR, s, fb, ff); k_factor<P><<<(unsigned)ctx->ne, L::THREADS, L::BYTES, s>>>(a); }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

template <int NB>
unsigned apply_grid(long long ne) {
  constexpr int EPC = 256 / NB;
  long long g = (ne + EPC - 1) / EPC;
  if (g > kRedBlocks) g = kRedBlocks;
  return (unsigned)(g < 1 ? 1 : g);
}

template <int NB>
int apply_nb(fr_ctx* ctx, double* r, const double* scale, double* z, double* sumsq,
             const int* done, cudaStream_t s, bool with_eps) {
  // work: ne nb^2 block entries, r in, z out (and r written back when scaled):
  // 2 nb flops per DOF.  Inside a GMRES cycle it is booked per finished iteration.
  const bool in_cycle = done != nullptr;
  const double nd = (double)ctx->ndof;
  const double wb = in_cycle ? 0.0 : 8.0 * (double)ctx->ne * NB * NB + 16.0 * nd + (scale ? 8.0 * nd : 0.0);
  const double wf = in_cycle ? 0.0 : 2.0 * NB * nd;
  { ProfScope ps_(ctx, FR_KF_APPLY, s, wb, wf); k_apply<NB><<<apply_grid<NB>(ctx->ne), (256 / NB) * NB, 0, s>>>(ctx->blocks, r, scale, z, ctx->ne,
                                                                  sumsq, ctx->red, done, eps_args(ctx, with_eps)); }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

template <int NB>
int solupdate_nb(fr_ctx* ctx, double* x, cudaStream_t s) {
  { ProfScope ps_(ctx, FR_KF_SOLUPDATE, s); k_solupdate<NB><<<apply_grid<NB>(ctx->ne), (256 / NB) * NB, 0, s>>>(
      ctx->blocks, ctx->V, ctx->ndof, ctx->gd.y, ctx->gd.k, x, ctx->ne); }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

unsigned vec_grid(long long n) {
  long long g = (n + kThreads - 1) / kThreads;
  if (g > kVecBlocks) g = kVecBlocks;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

int launch_block_factor(fr_ctx* ctx, const double* U, double shift, cudaStream_t s) {
  FactorArgs a;
  a.U = U; a.blocks = ctx->blocks; a.hx = ctx->hx; a.hy = ctx->hy;
  a.ne = ctx->ne; a.nx = ctx->nx; a.ny = ctx->ny;
  a.gam = ctx->opts.gamma; a.shift = shift; a.beps = ctx->opts.block_eps_rel;
  a.tab = ctx->tab;
  switch (ctx->p) {
    case 2: return factor_p<2>(ctx, a, s);
    case 3: return factor_p<3>(ctx, a, s);
    case 4: return factor_p<4>(ctx, a, s);
    default: return set_error(ctx, FR_ERR_UNSUPPORTED, "degree %d not compiled", ctx->p);
  }
}

int launch_block_apply(fr_ctx* ctx, double* r, const double* scale, double* z, double* sumsq,
                       const int* done, cudaStream_t s, bool with_eps) {
  if (!ctx->opts.precond) {
    { ProfScope ps_(ctx, FR_KF_APPLY, s); k_scale_copy<<<vec_grid(ctx->ndof), kThreads, 0, s>>>(r, scale, z, ctx->ndof, sumsq, ctx->red,
                                                          done, eps_args(ctx, with_eps)); }
    FRK_LAUNCHED(ctx);
    return FR_OK;
  }
  switch (ctx->nb) {
    case 36: return apply_nb<36>(ctx, r, scale, z, sumsq, done, s, with_eps);
    case 64: return apply_nb<64>(ctx, r, scale, z, sumsq, done, s, with_eps);
    case 100: return apply_nb<100>(ctx, r, scale, z, sumsq, done, s, with_eps);
    default: return set_error(ctx, FR_ERR_UNSUPPORTED, "block size %d not compiled", ctx->nb);
  }
}

int launch_solution_update(fr_ctx* ctx, double* x, cudaStream_t s) {
  if (!ctx->opts.precond) {
    { ProfScope ps_(ctx, FR_KF_SOLUPDATE, s); k_solupdate_plain<<<vec_grid(ctx->ndof), kThreads, 0, s>>>(ctx->V, ctx->ndof, ctx->gd.y,
                                                               ctx->gd.k, x, ctx->ndof); }
    FRK_LAUNCHED(ctx);
    return FR_OK;
  }
  switch (ctx->nb) {
    case 36: return solupdate_nb<36>(ctx, x, s);
    case 64: return solupdate_nb<64>(ctx, x, s);
    case 100: return solupdate_nb<100>(ctx, x, s);
    default: return set_error(ctx, FR_ERR_UNSUPPORTED, "block size %d not compiled", ctx->nb);
  }
}

}  // namespace frk
