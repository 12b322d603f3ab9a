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
  double* lin_fg;  // mode 3 writes / mixed A z reads: F(U), G(U) [ne][8][NP]
  double* lin_fx;  // per element's west face point: q-, q+, f^num (4 each) [ne][N][12]
  double* lin_fy;  // per element's south face point, same layout
  int riemann;     // common flux: 0 Rusanov, 1 Roe
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

// Element tile handled by one CTA (TX x TY elements, one thread per point);
// two shapes per degree, picked at run time by the autotuner.
template <int P, int V> struct Tile;
template <> struct Tile<2, 0> { static constexpr int TX = 5, TY = 5; };
template <> struct Tile<2, 1> { static constexpr int TX = 7, TY = 4; };
template <> struct Tile<3, 0> { static constexpr int TX = 4, TY = 4; };
template <> struct Tile<3, 1> { static constexpr int TX = 8, TY = 2; };
template <> struct Tile<4, 0> { static constexpr int TX = 3, TY = 3; };
template <> struct Tile<4, 1> { static constexpr int TX = 5, TY = 2; };
template <> struct Tile<5, 0> { static constexpr int TX = 2, TY = 3; };
template <> struct Tile<5, 1> { static constexpr int TX = 3, TY = 2; };
template <> struct Tile<6, 0> { static constexpr int TX = 2, TY = 2; };
template <> struct Tile<6, 1> { static constexpr int TX = 5, TY = 1; };

template <int P, int MODE, int TV, int RM>
__device__ __forceinline__ void residual_body(const ResArgs& a, double* __restrict__ out, int bid) {
  constexpr int N = P + 1, NP = N * N;
  constexpr int TX = Tile<P, TV>::TX, TY = Tile<P, TV>::TY, NE = TX * TY;
  constexpr int NXF = (TX + 1) * TY * N;  // points on the tile's x-faces (normal +x)
  constexpr int NYF = (TY + 1) * TX * N;  // points on the tile's y-faces (normal +y)
  constexpr bool PERTURB = MODE == 1 || MODE == 2;  // MODE 3: R's fluxes at U into the caches
  __shared__ double sq[NE][4][NP];
  __shared__ double sF[NE][4][NP];
  __shared__ double sG[NE][4][NP];
  __shared__ double str[NE][4][4][N];       // own traces [face W,E,S,N][var][k]
  __shared__ double shx[2][TY][4][N];       // outside traces on the tile's west / east faces
  __shared__ double shy[2][TX][4][N];       // outside traces on the tile's south / north faces
  __shared__ double sfx[TY][TX + 1][4][N];  // common flux f_n on x-face xf of tile row ly
  __shared__ double sfy[TX][TY + 1][4][N];  // common flux g_n on y-face yf of tile column lx
  __shared__ double sDt[N][N], slm[N], slp[N], sdgL[N], sdgR[N];
  constexpr int NOWN = NE * 4 * N;           // own-trace work items
  constexpr int NHALO = 2 * (TX + TY) * N;   // outside-trace work items

  if (a.done && *a.done) return;
  if (threadIdx.x < N * N) sDt[threadIdx.x / N][threadIdx.x % N] = a.tab.Dt[threadIdx.x / N][threadIdx.x % N];
  if (threadIdx.x < N) {
    slm[threadIdx.x] = a.tab.lm[threadIdx.x];
    slp[threadIdx.x] = a.tab.lp[threadIdx.x];
    sdgL[threadIdx.x] = a.tab.dgL[threadIdx.x];
    sdgR[threadIdx.x] = a.tab.dgR[threadIdx.x];
  }

  const int tiles_x = (a.nx + TX - 1) / TX;
  const int ix0 = (int)(bid % tiles_x) * TX, iy0 = (int)(bid / tiles_x) * TY;
  const int ax = min(TX, a.nx - ix0), ay = min(TY, a.ny - iy0);  // active tile extent
  const int el = threadIdx.x / NP, t = threadIdx.x % NP;
  const int lx = el % TX, ly = el / TX;
  const bool active = el < NE && lx < ax && ly < ay;
  const long long e = (long long)(ix0 + lx) + (long long)a.nx * (iy0 + ly);

  double eps = 0.0, ieps = 0.0;
  if (PERTURB) {
    eps = a.eps2[0];
    ieps = a.eps2[1];
  }
  // ---- 1: state (perturbed for A z) and pointwise fluxes ----
  if (active) {
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
      if (MODE == 3) {
        a.lin_fg[(e * 8 + v) * NP + t] = f[v];
        a.lin_fg[(e * 8 + 4 + v) * NP + t] = g[v];
      }
    }
  }
  __syncthreads();
  // ---- 2a: own solution traces on the four faces of every tile element,
  //      then (separate work items, starting on a warp boundary when NOWN is
  //      a multiple of 32, so the FP64 work does not diverge) the outside
  //      neighbours' traces on the tile's boundary faces, from global memory ----
  for (int idx = threadIdx.x; idx < NOWN + NHALO; idx += blockDim.x) {
    if (idx < NOWN) {
      const int e2 = idx / (4 * N), face = (idx / N) % 4, k = idx % N;
      if ((e2 % TX) >= ax || (e2 / TX) >= ay) continue;
      const int off = face < 2 ? N * k : k;
      const int stride = face < 2 ? 1 : N;
      const double* c = (face == 0 || face == 2) ? slm : slp;
#pragma unroll
      for (int v = 0; v < 4; ++v) str[e2][face][v][k] = trace_sum<N>(&sq[e2][v][off], stride, c);
    } else {
      const int h = idx - NOWN, seg = h / N, k = h % N;
      long long nb;
      int off, stride;
      const double* c;
      double* dst;
      if (seg < 2 * TY) {  // west (side 0) / east (side 1) boundary of tile row fy
        const int side = seg / TY, fy = seg % TY;
        if (fy >= ay) continue;
        const int gx = side == 0 ? (ix0 + a.nx - 1) % a.nx : (ix0 + ax) % a.nx;
        nb = (long long)gx + (long long)a.nx * (iy0 + fy);
        off = N * k;
        stride = 1;
        c = side == 0 ? slp : slm;  // the west neighbour's east trace, the east one's west trace
        dst = &shx[side][fy][0][k];
      } else {             // south (side 0) / north (side 1) boundary of tile column fx
        const int s2 = seg - 2 * TY, side = s2 / TX, fx = s2 % TX;
        if (fx >= ax) continue;
        const int gy = side == 0 ? (iy0 + a.ny - 1) % a.ny : (iy0 + ay) % a.ny;
        nb = (long long)(ix0 + fx) + (long long)a.nx * gy;
        off = k;
        stride = N;
        c = side == 0 ? slp : slm;
        dst = &shy[side][fx][0][k];
      }
#pragma unroll
      for (int v = 0; v < 4; ++v)
        dst[v * N] = trace_global<N, PERTURB>(a.U, a.z, nb * 4 * NP + v * NP + off, stride, c, eps);
    }
  }
  __syncthreads();
  // ---- 2b: one Rusanov flux per face point, both traces from shared memory ----
  for (int idx = threadIdx.x; idx < NXF + NYF; idx += blockDim.x) {
    double qm[4], qp[4], fc[4];
    if (idx < NXF) {
      const int k = idx % N, rr = idx / N, xf = rr % (TX + 1), fy = rr / (TX + 1);
      if (fy >= ay || xf > ax) continue;
      const int gy = iy0 + fy;
      const double* pm = xf >= 1 ? &str[xf - 1 + TX * fy][1][0][k] : &shx[0][fy][0][k];
      const double* pp = xf < ax ? &str[xf + TX * fy][0][0][k] : &shx[1][fy][0][k];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        qm[v] = pm[v * N];
        qp[v] = pp[v * N];
      }
      riemann_flux(RM, qm, qp, 0, a.gam, fc);
#pragma unroll
      for (int v = 0; v < 4; ++v) sfx[fy][xf][v][k] = fc[v];
      if (MODE == 3 && xf < ax) {  // the west face of tile element xf
        double* c = a.lin_fx + (((long long)(ix0 + xf) + (long long)a.nx * gy) * N + k) * 12;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          c[v] = qm[v];
          c[4 + v] = qp[v];
          c[8 + v] = fc[v];
        }
      }
    } else {
      const int i2 = idx - NXF;
      const int k = i2 % N, rr = i2 / N, yf = rr % (TY + 1), fx = rr / (TY + 1);
      if (fx >= ax || yf > ay) continue;
      const int gx = ix0 + fx;
      const double* pm = yf >= 1 ? &str[fx + TX * (yf - 1)][3][0][k] : &shy[0][fx][0][k];
      const double* pp = yf < ay ? &str[fx + TX * yf][2][0][k] : &shy[1][fx][0][k];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        qm[v] = pm[v * N];
        qp[v] = pp[v * N];
      }
      riemann_flux(RM, qm, qp, 1, a.gam, fc);
#pragma unroll
      for (int v = 0; v < 4; ++v) sfy[fx][yf][v][k] = fc[v];
      if (MODE == 3 && yf < ay) {  // the south face of tile element yf
        double* c = a.lin_fy + ((long long)gx + (long long)a.nx * (iy0 + yf)) * N * 12 + k * 12;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          c[v] = qm[v];
          c[4 + v] = qp[v];
          c[8 + v] = fc[v];
        }
      }
    }
  }
  __syncthreads();

  // ---- 3: corrected divergence and the output ----
  if (MODE == 3 || !active) return;
  const double hx = a.hx[ix0 + lx], hy = a.hy[iy0 + ly];
  const int i = t % N, j = t / N;
  // with unscaled fluxes, -(1/|J|)(dF~/dxi + dG~/deta) = -(2/hx) df~ - (2/hy) dg~
  const double sx = 2.0 / hx, sy = 2.0 / hy;
  const long long base = e * 4 * NP + t;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    double dF = sdgL[i] * sfx[ly][lx][v][j];
    dF = fma(sdgR[i], sfx[ly][lx + 1][v][j], dF);
#pragma unroll
    for (int k = 0; k < N; ++k) dF = fma(sDt[i][k], sF[el][v][k + N * j], dF);
    double dG = sdgL[j] * sfy[lx][ly][v][i];
    dG = fma(sdgR[j], sfy[lx][ly + 1][v][i], dG);
#pragma unroll
    for (int k = 0; k < N; ++k) dG = fma(sDt[j][k], sG[el][v][i + N * k], dG);
    const double R = -fma(sx, dF, sy * dG);
    const long long o = base + v * NP;
    if (MODE == 0) {
      out[o] = R;
    } else {
      const double zo = a.z[o];
      const double Az = eps > 0.0 ? fma(-(R - a.R0[o]), ieps, a.shift * zo) : a.shift * zo;
      out[o] = MODE == 2 ? a.b[o] - Az : Az;
    }
  }
}

template <int P, int MODE, int TV, int RM>
__global__ void __launch_bounds__(256, 4) k_residual(const ResArgs a) {
  residual_body<P, MODE, TV, RM>(a, a.out, blockIdx.x);
}

// A z of Arnoldi iteration j of every instance (of one degree) in one grid:
// instance k owns the tiles [start[k], start[k+1]); its table entry holds
// the basis in `out`, and A z is written to V_{j+1}.
template <int P, int RM>
__global__ void __launch_bounds__(256, 4) kb_residual(const ResArgs* __restrict__ tab, const int* __restrict__ start,
                                                      int ninst, int j) {
  const int k = batch_instance(start, ninst, blockIdx.x);
  const ResArgs& a = tab[k];
  const long long ndof = a.ne * 4 * (P + 1) * (P + 1);
  residual_body<P, 1, 0, RM>(a, a.out + (size_t)(j + 1) * ndof, blockIdx.x - start[k]);
}

// A z with FP32 linear parts (jv_precision 1).  R(U+eps z) - R(U) is the
// corrected divergence of the flux differences dF = F(U+eps z) - F(U) at the
// points and df = f^num(U+eps z) - f^num(U) on the faces; the divergence and
// correction are linear, so they run in FP32 on dF, df.  The nonlinear parts
// stay FP64: the pointwise fluxes at U + eps z and their difference from the
// cached F(U), the face states q(U) + eps trace(z) (trace of z in FP32, the
// state itself in FP64) and the Rusanov fluxes at them, differenced against
// the cached f^num(U).  Same element tiles as k_residual; MODE 1: A z,
// MODE 2: b - A z.
template <int P, int MODE, int TV, int RM>
__global__ void __launch_bounds__(256) k_jv32(const ResArgs a) {
  constexpr int N = P + 1, NP = N * N;
  constexpr int TX = Tile<P, TV>::TX, TY = Tile<P, TV>::TY, NE = TX * TY;
  constexpr int NXF = (TX + 1) * TY * N;
  constexpr int NYF = (TY + 1) * TX * N;
  __shared__ float sdF[NE][4][NP], sdG[NE][4][NP], sz[NE][4][NP];
  __shared__ float strz[NE][4][4][N];         // own traces of z [face W,E,S,N][var][k]
  __shared__ float shzx[2][TY][4][N];         // outside traces of z on the tile's west / east faces
  __shared__ float shzy[2][TX][4][N];         // outside traces of z on the tile's south / north faces
  constexpr int NOWN = NE * 4 * N, NHALO = 2 * (TX + TY) * N;
  __shared__ float sfx[TY][TX + 1][4][N];     // df on x-faces
  __shared__ float sfy[TX][TY + 1][4][N];     // df on y-faces
  __shared__ float sDt[N][N], slm[N], slp[N], sdgL[N], sdgR[N];

  if (a.done && *a.done) return;
  if (threadIdx.x < N * N) sDt[threadIdx.x / N][threadIdx.x % N] = (float)a.tab.Dt[threadIdx.x / N][threadIdx.x % N];
  if (threadIdx.x < N) {
    slm[threadIdx.x] = (float)a.tab.lm[threadIdx.x];
    slp[threadIdx.x] = (float)a.tab.lp[threadIdx.x];
    sdgL[threadIdx.x] = (float)a.tab.dgL[threadIdx.x];
    sdgR[threadIdx.x] = (float)a.tab.dgR[threadIdx.x];
  }
  const int tiles_x = (a.nx + TX - 1) / TX;
  const int ix0 = (int)(blockIdx.x % tiles_x) * TX, iy0 = (int)(blockIdx.x / tiles_x) * TY;
  const int ax = min(TX, a.nx - ix0), ay = min(TY, a.ny - iy0);
  const int el = threadIdx.x / NP, t = threadIdx.x % NP;
  const int lx = el % TX, ly = el / TX;
  const bool active = el < NE && lx < ax && ly < ay;
  const long long e = (long long)(ix0 + lx) + (long long)a.nx * (iy0 + ly);
  const double eps = a.eps2[0], ieps = a.eps2[1];
  // ---- 1: perturbed state, point fluxes (FP64) and their differences ----
  if (active) {
    const long long base = e * 4 * NP + t;
    double q[4], f[4], g[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const long long o = base + v * NP;
      const double zv = a.z[o];
      q[v] = fma(eps, zv, a.U[o]);
      sz[el][v][t] = (float)zv;
    }
    euler_fluxes(q, a.gam, f, g);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      sdF[el][v][t] = (float)(f[v] - a.lin_fg[(e * 8 + v) * NP + t]);
      sdG[el][v][t] = (float)(g[v] - a.lin_fg[(e * 8 + 4 + v) * NP + t]);
    }
  }
  __syncthreads();
  // ---- 2a: own traces of z (FP32), then the outside neighbours' traces of z
  //      on the tile's boundary faces (separate work items, from global memory) ----
  for (int idx = threadIdx.x; idx < NOWN + NHALO; idx += blockDim.x) {
    if (idx < NOWN) {
      const int e2 = idx / (4 * N), face = (idx / N) % 4, k = idx % N;
      if ((e2 % TX) >= ax || (e2 / TX) >= ay) continue;
      const int off = face < 2 ? N * k : k;
      const int stride = face < 2 ? 1 : N;
      const float* c = (face == 0 || face == 2) ? slm : slp;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        float s2 = c[0] * sz[e2][v][off];
#pragma unroll
        for (int q = 1; q < N; ++q) s2 = fmaf(c[q], sz[e2][v][off + q * stride], s2);
        strz[e2][face][v][k] = s2;
      }
    } else {
      const int h = idx - NOWN, seg = h / N, k = h % N;
      long long nb;
      int off, stride;
      const double* c;
      float* dst;
      if (seg < 2 * TY) {
        const int side = seg / TY, fy = seg % TY;
        if (fy >= ay) continue;
        const int gx = side == 0 ? (ix0 + a.nx - 1) % a.nx : (ix0 + ax) % a.nx;
        nb = (long long)gx + (long long)a.nx * (iy0 + fy);
        off = N * k;
        stride = 1;
        c = side == 0 ? a.tab.lp : a.tab.lm;
        dst = &shzx[side][fy][0][k];
      } else {
        const int s2 = seg - 2 * TY, side = s2 / TX, fx = s2 % TX;
        if (fx >= ax) continue;
        const int gy = side == 0 ? (iy0 + a.ny - 1) % a.ny : (iy0 + ay) % a.ny;
        nb = (long long)(ix0 + fx) + (long long)a.nx * gy;
        off = k;
        stride = N;
        c = side == 0 ? a.tab.lp : a.tab.lm;
        dst = &shzy[side][fx][0][k];
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) dst[v * N] = (float)trace_sum<N>(a.z + nb * 4 * NP + v * NP + off, stride, c);
    }
  }
  __syncthreads();
  // ---- 2b: face states q(U) + eps trace(z), Rusanov (FP64), df ----
  for (int idx = threadIdx.x; idx < NXF + NYF; idx += blockDim.x) {
    double qm[4], qp[4], fc[4];
    float tzm[4], tzp[4];
    const double* cache;
    int dir;
    int sx0, sx1, sx2, sx3;  // destination (row/column, face index, -, k)
    if (idx < NXF) {
      const int k = idx % N, rr = idx / N, xf = rr % (TX + 1), fy = rr / (TX + 1);
      if (fy >= ay || xf > ax) continue;
      const int gy = iy0 + fy;
      const long long ep = (long long)((ix0 + xf) % a.nx) + (long long)a.nx * gy;  // element east of the face
      cache = a.lin_fx + (ep * N + k) * 12;
      const float* pm = xf >= 1 ? &strz[xf - 1 + TX * fy][1][0][k] : &shzx[0][fy][0][k];
      const float* pp = xf < ax ? &strz[xf + TX * fy][0][0][k] : &shzx[1][fy][0][k];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        tzm[v] = pm[v * N];
        tzp[v] = pp[v * N];
      }
      dir = 0; sx0 = fy; sx1 = xf; sx3 = k; sx2 = 0;
    } else {
      const int i2 = idx - NXF;
      const int k = i2 % N, rr = i2 / N, yf = rr % (TY + 1), fx = rr / (TY + 1);
      if (fx >= ax || yf > ay) continue;
      const int gx = ix0 + fx;
      const long long ep = (long long)gx + (long long)a.nx * ((iy0 + yf) % a.ny);  // element north of the face
      cache = a.lin_fy + (ep * N + k) * 12;
      const float* pm = yf >= 1 ? &strz[fx + TX * (yf - 1)][3][0][k] : &shzy[0][fx][0][k];
      const float* pp = yf < ay ? &strz[fx + TX * yf][2][0][k] : &shzy[1][fx][0][k];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        tzm[v] = pm[v * N];
        tzp[v] = pp[v * N];
      }
      dir = 1; sx0 = fx; sx1 = yf; sx3 = k; sx2 = 0;
    }
    (void)sx2;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      qm[v] = fma(eps, (double)tzm[v], cache[v]);
      qp[v] = fma(eps, (double)tzp[v], cache[4 + v]);
    }
    riemann_flux(RM, qm, qp, dir, a.gam, fc);
    if (dir == 0) {
#pragma unroll
      for (int v = 0; v < 4; ++v) sfx[sx0][sx1][v][sx3] = (float)(fc[v] - cache[8 + v]);
    } else {
#pragma unroll
      for (int v = 0; v < 4; ++v) sfy[sx0][sx1][v][sx3] = (float)(fc[v] - cache[8 + v]);
    }
  }
  __syncthreads();
  // ---- 3: corrected divergence of the differences (FP32), output (FP64) ----
  if (!active) return;
  const float sx = (float)(2.0 / a.hx[ix0 + lx]), sy = (float)(2.0 / a.hy[iy0 + ly]);
  const int i = t % N, j = t / N;
  const long long base = e * 4 * NP + t;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    float dF = sdgL[i] * sfx[ly][lx][v][j];
    dF = fmaf(sdgR[i], sfx[ly][lx + 1][v][j], dF);
#pragma unroll
    for (int k = 0; k < N; ++k) dF = fmaf(sDt[i][k], sdF[el][v][k + N * j], dF);
    float dG = sdgL[j] * sfy[lx][ly][v][i];
    dG = fmaf(sdgR[j], sfy[lx][ly + 1][v][i], dG);
#pragma unroll
    for (int k = 0; k < N; ++k) dG = fmaf(sDt[j][k], sdG[el][v][i + N * k], dG);
    const float dR = -fmaf(sx, dF, sy * dG);  // R(U + eps z) - R(U)
    const long long o = base + v * NP;
    const double zo = a.z[o];
    const double Az = eps > 0.0 ? fma(-(double)dR, ieps, a.shift * zo) : a.shift * zo;
    a.out[o] = MODE == 2 ? a.b[o] - Az : Az;
  }
}

template <int P, int TV, int RM>
int launch_pvr(fr_ctx* ctx, int mode, const ResArgs& a, cudaStream_t s) {
  constexpr int NP = (P + 1) * (P + 1), TX = Tile<P, TV>::TX, TY = Tile<P, TV>::TY;
  const long long grid = (long long)((ctx->nx + TX - 1) / TX) * ((ctx->ny + TY - 1) / TY);
  const dim3 blk(TX * TY * NP);
  // algorithmic work: R reads U and writes R (16 B/DOF); A z also reads z and
  // R0 (and b) and adds the perturbation and the difference quotient.  Inside
  // a GMRES cycle the work is booked per finished iteration instead.
  const double nd = (double)ctx->ndof, fl = residual_flops_per_element(P) * (double)ctx->ne;
  const bool in_cycle = a.done != nullptr;
  const double wb = in_cycle ? 0.0 : (mode == 0 ? 16.0 : (mode == 1 ? 32.0 : 40.0)) * nd;
  const double wf = in_cycle ? 0.0 : (mode == 0 ? fl : fl + 6.0 * nd);
  const bool mixed = ctx->opts.jv_precision == 1;
  if (mode == 0) { ProfScope ps_(ctx, FR_KF_RESIDUAL, s, wb, wf); k_residual<P, 0, TV, RM><<<(unsigned)grid, blk, 0, s>>>(a); }
  else if (mode == 3) { ProfScope ps_(ctx, FR_KF_OTHER, s); k_residual<P, 3, TV, RM><<<(unsigned)grid, blk, 0, s>>>(a); }
  else if (mode == 1 && mixed) { ProfScope ps_(ctx, FR_KF_JV, s, wb, wf); k_jv32<P, 1, TV, RM><<<(unsigned)grid, blk, 0, s>>>(a); }
  else if (mode == 1) { ProfScope ps_(ctx, FR_KF_JV, s, wb, wf); k_residual<P, 1, TV, RM><<<(unsigned)grid, blk, 0, s>>>(a); }
  else if (mixed) { ProfScope ps_(ctx, FR_KF_JV, s, wb, wf); k_jv32<P, 2, TV, RM><<<(unsigned)grid, blk, 0, s>>>(a); }
  else { ProfScope ps_(ctx, FR_KF_JV, s, wb, wf); k_residual<P, 2, TV, RM><<<(unsigned)grid, blk, 0, s>>>(a); }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

// the common flux is a template parameter so each flux gets its own register allocation
template <int P, int TV>
int launch_pv(fr_ctx* ctx, int mode, const ResArgs& a, cudaStream_t s) {
  return a.riemann == 1 ? launch_pvr<P, TV, 1>(ctx, mode, a, s) : launch_pvr<P, TV, 0>(ctx, mode, a, s);
}

template <int P>
int launch_p(fr_ctx* ctx, int mode, const ResArgs& a, cudaStream_t s) {
  return ctx->tile_variant == 1 ? launch_pv<P, 1>(ctx, mode, a, s) : launch_pv<P, 0>(ctx, mode, a, s);
}

}  // namespace

int launch_residual(fr_ctx* ctx, int mode, const double* U, const double* z, const double* R0,
                    const double* b, double* out, double shift, const double* eps2,
                    const int* done, cudaStream_t s) {
  if (ctx->dim3) return launch_f3_residual(ctx, mode, U, z, R0, b, out, shift, eps2, done, s);
  if (ctx->viscous) return launch_ns_residual(ctx, mode, U, z, R0, b, out, shift, eps2, done, s);
  ResArgs a;
  a.U = U; a.z = z; a.R0 = R0; a.b = b; a.out = out;
  a.hx = ctx->hx; a.hy = ctx->hy; a.eps2 = eps2; a.done = done;
  a.ne = ctx->ne; a.nx = ctx->nx; a.ny = ctx->ny;
  a.gam = ctx->opts.gamma; a.shift = shift;
  a.eps_rel = ctx->opts.eps_rel; a.eps_fixed = ctx->opts.eps_fixed;
  a.lin_fg = ctx->lin_fg; a.lin_fx = ctx->lin_fx; a.lin_fy = ctx->lin_fy;
  a.riemann = ctx->opts.riemann;
  a.tab = ctx->tab;
  switch (ctx->p) {
    case 2: return launch_p<2>(ctx, mode, a, s);
    case 3: return launch_p<3>(ctx, mode, a, s);
    case 4: return launch_p<4>(ctx, mode, a, s);
    case 5: return launch_p<5>(ctx, mode, a, s);
    case 6: return launch_p<6>(ctx, mode, a, s);
    default: return set_error(ctx, FR_ERR_UNSUPPORTED, "degree %d not compiled", ctx->p);
  }
}

size_t batch_residual_bytes() { return sizeof(ResArgs); }

// tiles of the residual launch (tile variant 0, the one the batched launch uses)
unsigned residual_grid_of(const fr_ctx* ctx) {
  int tx = 1, ty = 1;
  switch (ctx->p) {
    case 2: tx = Tile<2, 0>::TX; ty = Tile<2, 0>::TY; break;
    case 3: tx = Tile<3, 0>::TX; ty = Tile<3, 0>::TY; break;
    case 4: tx = Tile<4, 0>::TX; ty = Tile<4, 0>::TY; break;
    default: return 0;
  }
  return (unsigned)(((ctx->nx + tx - 1) / tx) * ((ctx->ny + ty - 1) / ty));
}

// table entry of the batched A z: A = shift I - dR/dU at U, z = the
// context's preconditioned vector, output base = the Krylov basis
int fill_batch_residual(fr_ctx* ctx, const double* U, const double* R0, double shift, void* out) {
  if (ctx->dim3 || ctx->viscous || ctx->opts.jv_precision != 0 || ctx->p < 2 || ctx->p > 4) return FR_ERR_UNSUPPORTED;
  ResArgs a{};
  a.U = U; a.z = ctx->z; a.R0 = R0; a.b = nullptr; a.out = ctx->V;
  a.hx = ctx->hx; a.hy = ctx->hy; a.eps2 = ctx->scal + S_EPS; a.done = ctx->gd.done;
  a.ne = ctx->ne; a.nx = ctx->nx; a.ny = ctx->ny;
  a.gam = ctx->opts.gamma; a.shift = shift;
  a.eps_rel = ctx->opts.eps_rel; a.eps_fixed = ctx->opts.eps_fixed;
  a.lin_fg = ctx->lin_fg; a.lin_fx = ctx->lin_fx; a.lin_fy = ctx->lin_fy;
  a.riemann = ctx->opts.riemann;
  a.tab = ctx->tab;
  *reinterpret_cast<ResArgs*>(out) = a;
  return FR_OK;
}

int launch_batch_residual(int p, int riemann, const void* tab, const int* start, int ninst, int nblocks, int j,
                          cudaStream_t s) {
  const ResArgs* t = reinterpret_cast<const ResArgs*>(tab);
  count_launch();
  switch (p) {
    case 2: riemann ? kb_residual<2, 1><<<nblocks, Tile<2, 0>::TX * Tile<2, 0>::TY * 9, 0, s>>>(t, start, ninst, j)
                    : kb_residual<2, 0><<<nblocks, Tile<2, 0>::TX * Tile<2, 0>::TY * 9, 0, s>>>(t, start, ninst, j); break;
    case 3: riemann ? kb_residual<3, 1><<<nblocks, Tile<3, 0>::TX * Tile<3, 0>::TY * 16, 0, s>>>(t, start, ninst, j)
                    : kb_residual<3, 0><<<nblocks, Tile<3, 0>::TX * Tile<3, 0>::TY * 16, 0, s>>>(t, start, ninst, j); break;
    case 4: riemann ? kb_residual<4, 1><<<nblocks, Tile<4, 0>::TX * Tile<4, 0>::TY * 25, 0, s>>>(t, start, ninst, j)
                    : kb_residual<4, 0><<<nblocks, Tile<4, 0>::TX * Tile<4, 0>::TY * 25, 0, s>>>(t, start, ninst, j); break;
    default: return FR_ERR_UNSUPPORTED;
  }
  return cudaGetLastError() == cudaSuccess ? FR_OK : FR_ERR_CUDA;
}

int launch_linearize(fr_ctx* ctx, const double* U, cudaStream_t s) {
  if (ctx->dim3) return launch_f3_linearize(ctx, U, s);
  if (ctx->opts.jv_precision != 1 || ctx->viscous) return FR_OK;
  return launch_residual(ctx, 3, U, nullptr, nullptr, nullptr, nullptr, 0.0, nullptr, nullptr, s);
}

}  // namespace frk
