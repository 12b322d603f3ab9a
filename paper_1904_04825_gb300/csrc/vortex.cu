// Accuracy measure of the isentropic vortex study (Sec. 5.1): the exact
// solution of Eq. VP_Solution evaluated at every solution point and the error
// Error(s) = sqrt( int (s_exact - s_num)^2 dV / V ) by Gauss-Legendre
// quadrature, for s = rho, u, v, p, in one grid-stride pass over the state
// with a deterministic two-stage reduction.
#include <cmath>

#include "device.cuh"
#include "internal.cuh"

namespace frk {
namespace {

struct VortexArgs {
  const double* U;
  const double* xo;   // left edge of each element column
  const double* yo;   // bottom edge of each element row
  const double* hx;
  const double* hy;
  long long ne;
  int nx, n1, np;
  double xi[kMaxN], w[kMaxN];
  double gam;
  double xc, yc;      // centre at time t (before taking the periodic image)
  double lx, ly;      // periodic box
  double swirl;       // alpha / (2 pi)
  double dT0;         // -alpha^2 (gamma - 1) / (16 phi gamma pi^2)
  double phi;
  double rho_inf, u_inf, v_inf, t_inf;
};

// Work per point: the exact state (one exp, one pow) and the numerical
// primitives (one division); the four weighted squared differences.
__global__ void __launch_bounds__(256) k_vortex_error(const VortexArgs a, Reduce red, double* out) {
  __shared__ double sh[32];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const long long total = a.ne * a.np;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const long long e = g / a.np;
    const int t = (int)(g - e * a.np);
    const int i = t % a.n1, j = t / a.n1;
    const int ix = (int)(e % a.nx), iy = (int)(e / a.nx);
    const double hx = a.hx[ix], hy = a.hy[iy];
    const double x = a.xo[ix] + 0.5 * hx * (1.0 + a.xi[i]);
    const double y = a.yo[iy] + 0.5 * hy * (1.0 + a.xi[j]);
    double dx = x - a.xc, dy = y - a.yc;
    dx -= a.lx * floor(dx / a.lx + 0.5);
    dy -= a.ly * floor(dy / a.ly + 0.5);
    const double bump = exp(a.phi * (1.0 - (dx * dx + dy * dy)));
    const double ue = a.u_inf - a.swirl * dy * bump;
    const double ve = a.v_inf + a.swirl * dx * bump;
    const double Te = a.t_inf + a.dT0 * bump * bump;
    const double re = a.rho_inf * pow(Te / a.t_inf, 1.0 / (a.gam - 1.0));  // dS = 0
    const double pe = re * Te;                                             // R = 1
    const double* q = a.U + e * 4 * a.np + t;
    const double rho = q[0];
    const double ri = 1.0 / rho;
    const double u = q[a.np] * ri, v = q[2 * a.np] * ri;
    const double pr = (a.gam - 1.0) * (q[3 * a.np] - 0.5 * rho * (u * u + v * v));
    const double wt = a.w[i] * a.w[j] * (0.25 * hx * hy);
    const double d0 = re - rho, d1 = ue - u, d2 = ve - v, d3 = pe - pr;
    acc[0] = fma(wt * d0, d0, acc[0]);
    acc[1] = fma(wt * d1, d1, acc[1]);
    acc[2] = fma(wt * d2, d2, acc[2]);
    acc[3] = fma(wt * d3, d3, acc[3]);
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double bs = block_sum(acc[c], sh);
    if (threadIdx.x == 0) red.partials[(size_t)blockIdx.x * kMaxVec + c] = bs;
  }
  if (last_block(red.counter)) finish_sums(red, 4, out);
}

}  // namespace

int launch_vortex_error(fr_ctx* ctx, const double* U, const fr_vortex* vx, double t, double* out,
                        cudaStream_t s) {
  VortexArgs a{};
  a.U = U;
  a.xo = ctx->xo;
  a.yo = ctx->yo;
  a.hx = ctx->hx;
  a.hy = ctx->hy;
  a.ne = ctx->ne;
  a.nx = ctx->nx;
  a.n1 = ctx->n1;
  a.np = ctx->np;
  for (int i = 0; i < ctx->n1; ++i) {
    a.xi[i] = ctx->tab.xi[i];
    a.w[i] = ctx->tab.w[i];
  }
  const double g = ctx->opts.gamma;
  const double pi = 3.14159265358979323846;
  a.gam = g;
  a.xc = vx->x0 + vx->u_inf * t;
  a.yc = vx->y0 + vx->v_inf * t;
  a.lx = ctx->box[1] - ctx->box[0];
  a.ly = ctx->box[3] - ctx->box[2];
  a.swirl = vx->alpha / (2.0 * pi);
  a.dT0 = -vx->alpha * vx->alpha * (g - 1.0) / (16.0 * vx->phi * g * pi * pi);
  a.phi = vx->phi;
  a.rho_inf = vx->rho_inf;
  a.u_inf = vx->u_inf;
  a.v_inf = vx->v_inf;
  a.t_inf = (vx->u_inf * vx->u_inf + vx->v_inf * vx->v_inf) / (g * vx->mach * vx->mach);
  const long long total = ctx->ne * ctx->np;
  long long grid = (total + 255) / 256;
  if (grid > 4 * (long long)ctx->num_sms) grid = 4 * (long long)ctx->num_sms;
  if (grid > kRedBlocks) grid = kRedBlocks;
  {
    // 32 B read per point of the four conserved variables actually used
    ProfScope ps_(ctx, FR_KF_OTHER, s, 32.0 * (double)total, 0.0);
    k_vortex_error<<<(unsigned)grid, 256, 0, s>>>(a, ctx->red, out);
  }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

}  // namespace frk
