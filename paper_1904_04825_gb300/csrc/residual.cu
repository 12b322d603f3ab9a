// FR/CPR residual R(U) and the finite-difference operator A z of Sec. 3 / 4.5.
//
// One thread per (element, solution point); EPB = 256 / Np elements per CTA.
// Per element, in shared memory: the (possibly perturbed) state, the
// transformed fluxes F = (hy/2) f, G = (hx/2) g at the solution points, and
// the common fluxes F^num on the 4 (p+1) face points.  Fluxes are kept in
// physical form (f, g, f_n); the metric factors |J| |grad xi| / |J| = 2/hx,
// 2/hy are applied once per output.  A face point's own
// trace comes from shared memory, the neighbour's from global memory (L2),
// both summed in the same order with the same coefficients, so the two
// elements sharing a face compute bit-identical common fluxes (discrete
// conservation holds to round-off).  The corrected divergence uses the
// folded derivative matrix Dt (the local-flux traces F^l(+-1) are absorbed
// into Dt, which removes their extrapolation from the flop count).
#include "device.cuh"

namespace frk {
namespace {

struct ResArgs {
  const double* U;
  const double* z;
  const double* R0;
  const double* b;
  double* out;
  const double* hx;
  const double* hy;
  const double* eps2;  // (eps, 1/eps) of the FD product
  const int* done;
  long long ne;
  int nx, ny;
  double gam;
  double shift;
  double eps_rel;
  double eps_fixed;
  Tables tab;
};

// sum_k c[k] * x[k*stride], fixed order, explicit FMAs
template <int N>
__device__ __forceinline__ double trace_sum(const double* __restrict__ x, int stride,
                                            const double* c) {
  double s = c[0] * x[0];
#pragma unroll
  for (int k = 1; k < N; ++k) s = fma(c[k], x[k * stride], s);
  return s;
}

// neighbour trace from global memory, optionally perturbed by eps * z
template <int N, bool PERTURB>
__device__ __forceinline__ double trace_global(const double* __restrict__ U,
                                               const double* __restrict__ z, long long off,
                                               int stride, const double* c, double eps) {
  if (!PERTURB) return trace_sum<N>(U + off, stride, c);
  double s = c[0] * fma(eps, z[off], U[off]);
#pragma unroll
  for (int k = 1; k < N; ++k) s = fma(c[k], fma(eps, z[off + k * stride], U[off + k * stride]), s);
  return s;
}

template <int P, int MODE>
__global__ void __launch_bounds__(256) k_residual(const ResArgs a) {
  constexpr int N = P + 1, NP = N * N, EPB = 256 / NP, NFP = 4 * N;
  constexpr bool PERTURB = MODE > 0;
  __shared__ double sq[EPB][4][NP];
  __shared__ double sF[EPB][4][NP];
  __shared__ double sG[EPB][4][NP];
  __shared__ double sFn[EPB][4][4][N];  // [face W,E,S,N][var][k]
  __shared__ double sDt[N][N], slm[N], slp[N], sdgL[N], sdgR[N];

  if (a.done && *a.done) return;
  if (threadIdx.x < N * N) sDt[threadIdx.x / N][threadIdx.x % N] = a.tab.Dt[threadIdx.x / N][threadIdx.x % N];
  if (threadIdx.x < N) {
    slm[threadIdx.x] = a.tab.lm[threadIdx.x];
    slp[threadIdx.x] = a.tab.lp[threadIdx.x];
    sdgL[threadIdx.x] = a.tab.dgL[threadIdx.x];
    sdgR[threadIdx.x] = a.tab.dgR[threadIdx.x];
  }

  const int el = threadIdx.x / NP, t = threadIdx.x % NP;
  const long long e = (long long)blockIdx.x * EPB + el;
  const bool active = e < a.ne;

  double eps = 0.0, ieps = 0.0;
  if (PERTURB) {
    eps = a.eps2[0];
    ieps = a.eps2[1];
  }
  int ix = 0, iy = 0;
  double hx = 1.0, hy = 1.0;
  if (active) {
    ix = (int)(e % a.nx);
    iy = (int)(e / a.nx);
    hx = a.hx[ix];
    hy = a.hy[iy];
    const long long base = e * 4 * NP + t;
    double q[4], f[4], g[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const long long o = base + v * NP;
      q[v] = PERTURB ? fma(eps, a.z[o], a.U[o]) : a.U[o];
      sq[el][v][t] = q[v];
    }
    euler_fluxes(q, a.gam, f, g);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      sF[el][v][t] = f[v];
      sG[el][v][t] = g[v];
    }
  }
  __syncthreads();

  if (active) {
    for (int fp = t; fp < NFP; fp += NP) {
      const int face = fp / N, k = fp % N;
      double qo[4], qn[4], fc[4];
      long long nbr;
      if (face == 0) nbr = (long long)((ix + a.nx - 1) % a.nx) + (long long)a.nx * iy;
      else if (face == 1) nbr = (long long)((ix + 1) % a.nx) + (long long)a.nx * iy;
      else if (face == 2) nbr = (long long)ix + (long long)a.nx * ((iy + a.ny - 1) % a.ny);
      else nbr = (long long)ix + (long long)a.nx * ((iy + 1) % a.ny);
      // own trace: faces W/E run along row k (stride 1), S/N along column k (stride N)
      const int off_own = face < 2 ? N * k : k;
      const int stride = face < 2 ? 1 : N;
      const double* c_own = (face == 0 || face == 2) ? slm : slp;   // own -1 or +1 end
      const double* c_nbr = (face == 0 || face == 2) ? slp : slm;   // neighbour's opposite end
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        qo[v] = trace_sum<N>(&sq[el][v][off_own], stride, c_own);
        qn[v] = trace_global<N, PERTURB>(a.U, a.z, nbr * 4 * NP + v * NP + off_own, stride, c_nbr,
                                          eps);
      }
      const int dir = face < 2 ? 0 : 1;
      if (face == 0 || face == 2) rusanov(qn, qo, dir, a.gam, fc);
      else rusanov(qo, qn, dir, a.gam, fc);
#pragma unroll
      for (int v = 0; v < 4; ++v) sFn[el][face][v][k] = fc[v];
    }
  }
  __syncthreads();

  if (!active) return;
  const int i = t % N, j = t / N;
  // with unscaled fluxes, -(1/|J|)(dF~/dxi + dG~/deta) = -(2/hx) df~ - (2/hy) dg~
  const double sx = 2.0 / hx, sy = 2.0 / hy;
  const long long base = e * 4 * NP + t;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    double dF = sdgL[i] * sFn[el][0][v][j];
    dF = fma(sdgR[i], sFn[el][1][v][j], dF);
#pragma unroll
    for (int k = 0; k < N; ++k) dF = fma(sDt[i][k], sF[el][v][k + N * j], dF);
    double dG = sdgL[j] * sFn[el][2][v][i];
    dG = fma(sdgR[j], sFn[el][3][v][i], dG);
#pragma unroll
    for (int k = 0; k < N; ++k) dG = fma(sDt[j][k], sG[el][v][i + N * k], dG);
    const double R = -fma(sx, dF, sy * dG);
    const long long o = base + v * NP;
    if (MODE == 0) {
      a.out[o] = R;
    } else {
      const double zo = a.z[o];
      const double Az = eps > 0.0 ? fma(-(R - a.R0[o]), ieps, a.shift * zo) : a.shift * zo;
      a.out[o] = MODE == 2 ? a.b[o] - Az : Az;
    }
  }
}

template <int P>
int launch_p(fr_ctx* ctx, int mode, const ResArgs& a, cudaStream_t s) {
  constexpr int NP = (P + 1) * (P + 1), EPB = 256 / NP;
  const long long grid = (ctx->ne + EPB - 1) / EPB;
  const dim3 blk(EPB * NP);
  // algorithmic work: R reads U and writes R (16 B/DOF); A z also reads z and
  // R0 (and b) and adds the perturbation and the difference quotient.  Inside
  // a GMRES cycle the work is booked per finished iteration instead.
  const double nd = (double)ctx->ndof, fl = residual_flops_per_element(P) * (double)ctx->ne;
  const bool in_cycle = a.done != nullptr;
  const double wb = in_cycle ? 0.0 : (mode == 0 ? 16.0 : (mode == 1 ? 32.0 : 40.0)) * nd;
  const double wf = in_cycle ? 0.0 : (mode == 0 ? fl : fl + 6.0 * nd);
  if (mode == 0) { ProfScope ps_(ctx, FR_KF_RESIDUAL, s, wb, wf); k_residual<P, 0><<<(unsigned)grid, blk, 0, s>>>(a); }
  else if (mode == 1) { ProfScope ps_(ctx, FR_KF_JV, s, wb, wf); k_residual<P, 1><<<(unsigned)grid, blk, 0, s>>>(a); }
  else { ProfScope ps_(ctx, FR_KF_JV, s, wb, wf); k_residual<P, 2><<<(unsigned)grid, blk, 0, s>>>(a); }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

}  // namespace

int launch_residual(fr_ctx* ctx, int mode, const double* U, const double* z, const double* R0,
                    const double* b, double* out, double shift, const double* eps2,
                    const int* done, cudaStream_t s) {
  ResArgs a;
  a.U = U; a.z = z; a.R0 = R0; a.b = b; a.out = out;
  a.hx = ctx->hx; a.hy = ctx->hy; a.eps2 = eps2; a.done = done;
  a.ne = ctx->ne; a.nx = ctx->nx; a.ny = ctx->ny;
  a.gam = ctx->opts.gamma; a.shift = shift;
  a.eps_rel = ctx->opts.eps_rel; a.eps_fixed = ctx->opts.eps_fixed;
  a.tab = ctx->tab;
  switch (ctx->p) {
    case 2: return launch_p<2>(ctx, mode, a, s);
    case 3: return launch_p<3>(ctx, mode, a, s);
    case 4: return launch_p<4>(ctx, mode, a, s);
    default: return set_error(ctx, FR_ERR_UNSUPPORTED, "degree %d not compiled", ctx->p);
  }
}

}  // namespace frk
