// Viscous (Navier-Stokes) FR residual with BR2 common gradients, Sec. 2-3
// (Eqs. com_q, com_grad_q and the BR2 lifting with g'(+-1) = +-(P+1)(P+2)/2).
//
// R(U), A z and b - A z take three kernels:
//  k_ns_trace: per element, the (possibly perturbed) state and its own
//    polynomial gradient traced to the 4 (p+1) face points -> trace buffer.
//  k_ns_face:  per west / south face point (and north wall), the common
//    solution, BR2 common gradient and common total flux (Rusanov inviscid
//    minus viscous) from the two traces -> face buffer, each face once.
//  k_ns_cell:  per element, the FR-corrected gradient and total flux at the
//    solution points, the corrected divergence with the four faces' common
//    fluxes, the body-force source and the output.  Both elements of a face
//    read the same stored flux, so conservation holds to round-off.
// Element-Jacobi columns use k_ns_res (its mode 3) after a trace pass of the
// unperturbed state: slot = (element, column c), own state perturbed in DOF
// c by eps_c = beps (1 + |q_c|), own traces recomputed, neighbour traces
// frozen; it forms the element's four face fluxes itself and stages column c
// of shift*I - J_ee for the inversion kernel.
// Walls (isothermal, no slip) at the y ends: boundary state
// (rho_int, 0, 0, rho_int R T_w / (gamma - 1)), common gradient = own
// gradient + own lifting, inviscid wall flux g(q_b).  Gas constant R = 1.
#include "device.cuh"

namespace frk {
namespace {

struct NsArgs {
  const double* U;
  const double* z;
  const double* R0;
  const double* b;
  double* out;
  double* tb;          // traces [ne][4 faces][N][4 vars][3] = (q, q_x, q_y)
  double* fb;          // common data per element's W, S (and top-wall N) face [ne][3][N][8] = (q_com, f_n)
  const double* hx;
  const double* hy;
  const double* eps2;
  const int* done;
  long long ne;
  int nx, ny, wall_y;
  double gam, mu, kappa, gx, t_wall;
  double shift, beps;
  Tables tab;
};

template <int P> struct NsSlots;
template <> struct NsSlots<2> { static constexpr int E = 14; };
template <> struct NsSlots<3> { static constexpr int E = 8; };
template <> struct NsSlots<4> { static constexpr int E = 5; };

template <int N>
__device__ __forceinline__ double tsum(const double* x, int stride, const double* c) {
  double s = c[0] * x[0];
#pragma unroll
  for (int k = 1; k < N; ++k) s = fma(c[k], x[k * stride], s);
  return s;
}

// viscous fluxes (f_vis, g_vis) from the state and its gradients, R = 1
__device__ __forceinline__ void visc_flux(const double q[4], const double qx[4], const double qy[4],
                                          double gam, double mu, double kappa, double fv[4],
                                          double gv[4]) {
  const double rinv = 1.0 / q[0];
  const double u = q[1] * rinv, v = q[2] * rinv, e = q[3] * rinv;
  const double ux = (qx[1] - u * qx[0]) * rinv, vx = (qx[2] - v * qx[0]) * rinv;
  const double uy = (qy[1] - u * qy[0]) * rinv, vy = (qy[2] - v * qy[0]) * rinv;
  const double Tx = (gam - 1.0) * ((qx[3] - e * qx[0]) * rinv - (u * ux + v * vx));
  const double Ty = (gam - 1.0) * ((qy[3] - e * qy[0]) * rinv - (u * uy + v * vy));
  const double div = ux + vy;
  const double txx = mu * (2.0 * ux - (2.0 / 3.0) * div);
  const double tyy = mu * (2.0 * vy - (2.0 / 3.0) * div);
  const double txy = mu * (uy + vx);
  fv[0] = 0.0; fv[1] = txx; fv[2] = txy; fv[3] = u * txx + v * txy + kappa * Tx;
  gv[0] = 0.0; gv[1] = txy; gv[2] = tyy; gv[3] = u * txy + v * tyy + kappa * Ty;
}

// Shared per-element work: state into sq, reference-space derivatives into
// dxi / deta, traces (q, q_x, q_y) of face point (face, k) into t[v][3].
template <int N>
__device__ __forceinline__ void face_trace(const double* sq, const double* dxi, const double* deta,
                                           int face, int k, double sx, double sy, const double* lm,
                                           const double* lp, double t[4][3]) {
  constexpr int NP = N * N;
  const int off = face < 2 ? N * k : k;
  const int stride = face < 2 ? 1 : N;
  const double* c = (face == 0 || face == 2) ? lm : lp;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    t[v][0] = tsum<N>(sq + v * NP + off, stride, c);
    t[v][1] = sx * tsum<N>(dxi + v * NP + off, stride, c);
    t[v][2] = sy * tsum<N>(deta + v * NP + off, stride, c);
  }
}

template <int P, bool PERTURB>
__global__ void __launch_bounds__(256) k_ns_trace(const NsArgs a) {
  constexpr int N = P + 1, NP = N * N, E = NsSlots<P>::E;
  __shared__ double sq[E][4 * NP], dxi[E][4 * NP], deta[E][4 * NP];
  __shared__ double sD[N][N], slm[N], slp[N];
  if (threadIdx.x < N * N) sD[threadIdx.x / N][threadIdx.x % N] = a.tab.D[threadIdx.x / N][threadIdx.x % N];
  if (threadIdx.x < N) {
    slm[threadIdx.x] = a.tab.lm[threadIdx.x];
    slp[threadIdx.x] = a.tab.lp[threadIdx.x];
  }
  if (a.done && *a.done) return;
  const int el = threadIdx.x / NP, t = threadIdx.x % NP;
  const long long e = (long long)blockIdx.x * E + el;
  const bool active = el < E && e < a.ne;
  const double eps = PERTURB ? a.eps2[0] : 0.0;
  if (active) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const long long o = e * 4 * NP + v * NP + t;
      sq[el][v * NP + t] = PERTURB ? fma(eps, a.z[o], a.U[o]) : a.U[o];
    }
  }
  __syncthreads();
  if (active) {
    const int i = t % N, j = t / N;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      double d1 = 0.0, d2 = 0.0;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        d1 = fma(sD[i][k], sq[el][v * NP + k + N * j], d1);
        d2 = fma(sD[j][k], sq[el][v * NP + i + N * k], d2);
      }
      dxi[el][v * NP + t] = d1;
      deta[el][v * NP + t] = d2;
    }
  }
  __syncthreads();
  if (!active) return;
  const int ix = (int)(e % a.nx), iy = (int)(e / a.nx);
  const double sx = 2.0 / a.hx[ix], sy = 2.0 / a.hy[iy];
  for (int fp = t; fp < 4 * N; fp += NP) {
    const int face = fp / N, k = fp % N;
    double tr[4][3];
    face_trace<N>(sq[el], dxi[el], deta[el], face, k, sx, sy, slm, slp, tr);
    double* dst = a.tb + (((e * 4 + face) * N + k) * 4) * 3;
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int c = 0; c < 3; ++c) dst[v * 3 + c] = tr[v][c];
  }
}

// common total flux across a face from the left (-) and right (+) data;
// dir 0: x-face (normal +x), 1: y-face (normal +y); hm, hp: element sizes
// normal to the face; cbr2 = (P+1)(P+2)/2.
__device__ __forceinline__ void common_flux(const double m[4][3], const double pp[4][3], int dir,
                                            double hm, double hp, double cbr2, const NsArgs& a,
                                            double qc[4], double fn[4]) {
  double qm[4], qp[4], gxc[4], gyc[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    qm[v] = m[v][0];
    qp[v] = pp[v][0];
    qc[v] = 0.5 * (qm[v] + qp[v]);
    const double rm = (2.0 / hm) * cbr2 * (qc[v] - qm[v]);   // lifting of the (-) element
    const double rp = -(2.0 / hp) * cbr2 * (qc[v] - qp[v]);  // lifting of the (+) element
    if (dir == 0) {
      gxc[v] = 0.5 * ((m[v][1] + rm) + (pp[v][1] + rp));
      gyc[v] = 0.5 * (m[v][2] + pp[v][2]);
    } else {
      gxc[v] = 0.5 * (m[v][1] + pp[v][1]);
      gyc[v] = 0.5 * ((m[v][2] + rm) + (pp[v][2] + rp));
    }
  }
  double fi[4], fv[4], gv[4];
  rusanov(qm, qp, dir, a.gam, fi);
  visc_flux(qc, gxc, gyc, a.gam, a.mu, a.kappa, fv, gv);
#pragma unroll
  for (int v = 0; v < 4; ++v) fn[v] = fi[v] - (dir == 0 ? fv[v] : gv[v]);
}

// wall face: own data o (the element is (+) on the south wall, (-) on the north wall)
__device__ __forceinline__ void wall_flux(const double o[4][3], bool south, double h, double cbr2,
                                          const NsArgs& a, double qc[4], double fn[4]) {
  double qo[4], gxc[4], gyc[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) qo[v] = o[v][0];
  qc[0] = qo[0];
  qc[1] = 0.0;
  qc[2] = 0.0;
  qc[3] = qo[0] * a.t_wall / (a.gam - 1.0);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const double r = (south ? -1.0 : 1.0) * (2.0 / h) * cbr2 * (qc[v] - qo[v]);
    gxc[v] = o[v][1];
    gyc[v] = o[v][2] + r;
  }
  double f[4], g[4], fv[4], gv[4];
  euler_fluxes(qc, a.gam, f, g);
  visc_flux(qc, gxc, gyc, a.gam, a.mu, a.kappa, fv, gv);
#pragma unroll
  for (int v = 0; v < 4; ++v) fn[v] = g[v] - gv[v];
}

template <int P, int MODE>
__global__ void __launch_bounds__(256) k_ns_res(const NsArgs a) {
  constexpr int N = P + 1, NP = N * N, E = NsSlots<P>::E, NB = 4 * NP;
  constexpr bool PERTURB = MODE == 1 || MODE == 2;
  constexpr double cbr2 = (P + 1) * (P + 2) / 2.0;
  __shared__ double sq[E][4 * NP], dxi[E][4 * NP], deta[E][4 * NP];  // dxi/deta reused for F, G
  __shared__ double tr[E][4][N][4][3];   // own face traces
  __shared__ double cq[E][4][N][4];      // common solution on the own faces
  __shared__ double fnum[E][4][N][4];    // common total normal flux on the own faces
  __shared__ double sD[N][N], sDt[N][N], slm[N], slp[N], sdgL[N], sdgR[N];
  if (a.done && *a.done) return;
  if (threadIdx.x < N * N) {
    sD[threadIdx.x / N][threadIdx.x % N] = a.tab.D[threadIdx.x / N][threadIdx.x % N];
    sDt[threadIdx.x / N][threadIdx.x % N] = a.tab.Dt[threadIdx.x / N][threadIdx.x % N];
  }
  if (threadIdx.x < N) {
    slm[threadIdx.x] = a.tab.lm[threadIdx.x];
    slp[threadIdx.x] = a.tab.lp[threadIdx.x];
    sdgL[threadIdx.x] = a.tab.dgL[threadIdx.x];
    sdgR[threadIdx.x] = a.tab.dgR[threadIdx.x];
  }
  const int el = threadIdx.x / NP, t = threadIdx.x % NP;
  const long long slot = (long long)blockIdx.x * E + el;
  const long long nslots = MODE == 3 ? a.ne * NB : a.ne;
  const bool active = el < E && slot < nslots;
  const long long e = MODE == 3 ? slot / NB : slot;
  const int col = MODE == 3 ? (int)(slot % NB) : 0;
  double eps = 0.0, ieps = 0.0;
  if (PERTURB) {
    eps = a.eps2[0];
    ieps = a.eps2[1];
  }
  int ix = 0, iy = 0;
  double hx = 1.0, hy = 1.0;
  double ceps = 0.0;
  if (active) {
    ix = (int)(e % a.nx);
    iy = (int)(e / a.nx);
    hx = a.hx[ix];
    hy = a.hy[iy];
    if (MODE == 3) ceps = a.beps * (1.0 + fabs(a.U[e * NB + col]));
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const long long o = e * 4 * NP + v * NP + t;
      double qv = PERTURB ? fma(eps, a.z[o], a.U[o]) : a.U[o];
      if (MODE == 3 && v * NP + t == col) qv += ceps;
      sq[el][v * NP + t] = qv;
    }
  }
  __syncthreads();
  const int i = t % N, j = t / N;
  if (active) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      double d1 = 0.0, d2 = 0.0;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        d1 = fma(sD[i][k], sq[el][v * NP + k + N * j], d1);
        d2 = fma(sD[j][k], sq[el][v * NP + i + N * k], d2);
      }
      dxi[el][v * NP + t] = d1;
      deta[el][v * NP + t] = d2;
    }
  }
  __syncthreads();
  const double sx = 2.0 / hx, sy = 2.0 / hy;
  if (active) {
    for (int fp = t; fp < 4 * N; fp += NP) {
      const int face = fp / N, k = fp % N;
      double o[4][3];
      face_trace<N>(sq[el], dxi[el], deta[el], face, k, sx, sy, slm, slp, o);
#pragma unroll
      for (int v = 0; v < 4; ++v)
#pragma unroll
        for (int c = 0; c < 3; ++c) tr[el][face][k][v][c] = o[v][c];
    }
  }
  __syncthreads();
  // common solution, BR2 common gradient and common total flux per own face point
  if (active) {
    for (int fp = t; fp < 4 * N; fp += NP) {
      const int face = fp / N, k = fp % N;
      double o[4][3], nb[4][3], qc[4], fn[4];
#pragma unroll
      for (int v = 0; v < 4; ++v)
#pragma unroll
        for (int c = 0; c < 3; ++c) o[v][c] = tr[el][face][k][v][c];
      const bool wall = a.wall_y && ((face == 2 && iy == 0) || (face == 3 && iy == a.ny - 1));
      if (wall) {
        wall_flux(o, face == 2, hy, cbr2, a, qc, fn);
      } else {
        long long nbe;
        int nface;
        double hn;
        if (face == 0) { const int jx = (ix + a.nx - 1) % a.nx; nbe = jx + (long long)a.nx * iy; nface = 1; hn = a.hx[jx]; }
        else if (face == 1) { const int jx = (ix + 1) % a.nx; nbe = jx + (long long)a.nx * iy; nface = 0; hn = a.hx[jx]; }
        else if (face == 2) { const int jy = (iy + a.ny - 1) % a.ny; nbe = ix + (long long)a.nx * jy; nface = 3; hn = a.hy[jy]; }
        else { const int jy = (iy + 1) % a.ny; nbe = ix + (long long)a.nx * jy; nface = 2; hn = a.hy[jy]; }
        const double* src = a.tb + (((nbe * 4 + nface) * N + k) * 4) * 3;
#pragma unroll
        for (int v = 0; v < 4; ++v)
#pragma unroll
          for (int c = 0; c < 3; ++c) nb[v][c] = src[v * 3 + c];
        const int dir = face < 2 ? 0 : 1;
        const double hown = dir == 0 ? hx : hy;
        if (face == 0 || face == 2) common_flux(nb, o, dir, hn, hown, cbr2, a, qc, fn);
        else common_flux(o, nb, dir, hown, hn, cbr2, a, qc, fn);
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        cq[el][face][k][v] = qc[v];
        fnum[el][face][k][v] = fn[v];
      }
    }
  }
  __syncthreads();
  // corrected gradient and total flux at the own point (overwrites dxi / deta)
  if (active) {
    double q[4], gxv[4], gyv[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      q[v] = sq[el][v * NP + t];
      double dx = dxi[el][v * NP + t];
      dx = fma(cq[el][0][j][v] - tr[el][0][j][v][0], sdgL[i], dx);
      dx = fma(cq[el][1][j][v] - tr[el][1][j][v][0], sdgR[i], dx);
      double dy = deta[el][v * NP + t];
      dy = fma(cq[el][2][i][v] - tr[el][2][i][v][0], sdgL[j], dy);
      dy = fma(cq[el][3][i][v] - tr[el][3][i][v][0], sdgR[j], dy);
      gxv[v] = sx * dx;
      gyv[v] = sy * dy;
    }
    double f[4], g[4], fv[4], gv[4];
    euler_fluxes(q, a.gam, f, g);
    visc_flux(q, gxv, gyv, a.gam, a.mu, a.kappa, fv, gv);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      dxi[el][v * NP + t] = f[v] - fv[v];
      deta[el][v * NP + t] = g[v] - gv[v];
    }
  }
  __syncthreads();
  if (!active) return;
  const long long base = e * 4 * NP + t;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    double dF = sdgL[i] * fnum[el][0][j][v];
    dF = fma(sdgR[i], fnum[el][1][j][v], dF);
#pragma unroll
    for (int k = 0; k < N; ++k) dF = fma(sDt[i][k], dxi[el][v * NP + k + N * j], dF);
    double dG = sdgL[j] * fnum[el][2][i][v];
    dG = fma(sdgR[j], fnum[el][3][i][v], dG);
#pragma unroll
    for (int k = 0; k < N; ++k) dG = fma(sDt[j][k], deta[el][v * NP + i + N * k], dG);
    double R = -fma(sx, dF, sy * dG);
    if (v == 1) R = fma(sq[el][t], a.gx, R);
    if (v == 3) R = fma(sq[el][NP + t], a.gx, R);
    const long long o = base + v * NP;
    if (MODE == 0) {
      a.out[o] = R;
    } else if (MODE == 3) {
      // column col of M = shift I - J_ee, staged column-major [col][row]
      const int row = v * NP + t;
      const double m = (row == col ? a.shift : 0.0) - (R - a.R0[o]) / ceps;
      a.out[(e * NB + col) * NB + row] = m;
    } else {
      const double zo = a.z[o];
      const double Az = eps > 0.0 ? fma(-(R - a.R0[o]), ieps, a.shift * zo) : a.shift * zo;
      a.out[o] = MODE == 2 ? a.b[o] - Az : Az;
    }
  }
}

// Modes 0-2 in two passes so every face's common data is formed once:
// k_ns_face: one thread per (element, face W or S, point): q_com and the
//   common total flux from the two traces in the trace buffer (or the wall
//   state), into the face buffer; top-row elements also form their north
//   wall face.
// k_ns_cell: per element the FR-corrected gradient with q_com of its four
//   faces, the point fluxes, the corrected divergence with the common fluxes
//   of its four faces (W, S own; E, N the neighbours' W, S), body force and
//   the output.  Both elements of a face read the same stored flux, so
//   conservation holds to round-off.
template <int P>
__global__ void __launch_bounds__(256) k_ns_face(const NsArgs a) {
  constexpr int N = P + 1;
  constexpr double cbr2 = (P + 1) * (P + 2) / 2.0;
  if (a.done && *a.done) return;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = a.ne * 3 * N;
  if (tid >= total) return;
  const int k = (int)(tid % N);
  const int slot = (int)((tid / N) % 3);  // 0: west face, 1: south face, 2: north wall
  const long long e = tid / (3 * N);
  const int ix = (int)(e % a.nx), iy = (int)(e / a.nx);
  if (slot == 2 && !(a.wall_y && iy == a.ny - 1)) return;
  const double hx = a.hx[ix], hy = a.hy[iy];
  double o[4][3], nb[4][3], qc[4], fn[4];
  const int oface = slot == 0 ? 0 : (slot == 1 ? 2 : 3);
  const double* src = a.tb + (((e * 4 + oface) * N + k) * 4) * 3;
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int c = 0; c < 3; ++c) o[v][c] = src[v * 3 + c];
  if (slot == 2) {
    wall_flux(o, false, hy, cbr2, a, qc, fn);
  } else if (slot == 1 && a.wall_y && iy == 0) {
    wall_flux(o, true, hy, cbr2, a, qc, fn);
  } else {
    long long nbe;
    double hn;
    int nface;
    if (slot == 0) { const int jx = (ix + a.nx - 1) % a.nx; nbe = jx + (long long)a.nx * iy; nface = 1; hn = a.hx[jx]; }
    else { const int jy = (iy + a.ny - 1) % a.ny; nbe = ix + (long long)a.nx * jy; nface = 3; hn = a.hy[jy]; }
    const double* ns = a.tb + (((nbe * 4 + nface) * N + k) * 4) * 3;
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int c = 0; c < 3; ++c) nb[v][c] = ns[v * 3 + c];
    common_flux(nb, o, slot == 0 ? 0 : 1, hn, slot == 0 ? hx : hy, cbr2, a, qc, fn);
  }
  double* dst = a.fb + ((e * 3 + slot) * N + k) * 8;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    dst[v] = qc[v];
    dst[4 + v] = fn[v];
  }
}

template <int P, int MODE>
__global__ void __launch_bounds__(256) k_ns_cell(const NsArgs a) {
  constexpr int N = P + 1, NP = N * N, E = NsSlots<P>::E;
  constexpr bool PERTURB = MODE == 1 || MODE == 2;
  __shared__ double sq[E][4 * NP], dxi[E][4 * NP], deta[E][4 * NP];
  __shared__ double cq[E][4][N][4];    // q_com on the own faces [W,E,S,N]
  __shared__ double tq[E][4][N][4];    // own face traces of q
  __shared__ double fnum[E][4][N][4];  // common total flux on the own faces
  __shared__ double sD[N][N], sDt[N][N], sdgL[N], sdgR[N];
  if (a.done && *a.done) return;
  if (threadIdx.x < N * N) {
    sD[threadIdx.x / N][threadIdx.x % N] = a.tab.D[threadIdx.x / N][threadIdx.x % N];
    sDt[threadIdx.x / N][threadIdx.x % N] = a.tab.Dt[threadIdx.x / N][threadIdx.x % N];
  }
  if (threadIdx.x < N) {
    sdgL[threadIdx.x] = a.tab.dgL[threadIdx.x];
    sdgR[threadIdx.x] = a.tab.dgR[threadIdx.x];
  }
  const int el = threadIdx.x / NP, t = threadIdx.x % NP;
  const long long e = (long long)blockIdx.x * E + el;
  const bool active = el < E && e < a.ne;
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
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const long long o = e * 4 * NP + v * NP + t;
      sq[el][v * NP + t] = PERTURB ? fma(eps, a.z[o], a.U[o]) : a.U[o];
    }
    // own traces of q and the common data of the four faces
    for (int fp = t; fp < 4 * N; fp += NP) {
      const int face = fp / N, k = fp % N;
      const double* tr = a.tb + (((e * 4 + face) * N + k) * 4) * 3;
      long long fe;
      int fs;
      if (face == 0) { fe = e; fs = 0; }
      else if (face == 2) { fe = e; fs = 1; }
      else if (face == 1) { fe = (long long)((ix + 1) % a.nx) + (long long)a.nx * iy; fs = 0; }
      else if (a.wall_y && iy == a.ny - 1) { fe = e; fs = 2; }
      else { fe = (long long)ix + (long long)a.nx * ((iy + 1) % a.ny); fs = 1; }
      const double* fd = a.fb + ((fe * 3 + fs) * N + k) * 8;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        tq[el][face][k][v] = tr[v * 3];
        cq[el][face][k][v] = fd[v];
        fnum[el][face][k][v] = fd[4 + v];
      }
    }
  }
  __syncthreads();
  const int i = t % N, j = t / N;
  if (active) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      double d1 = 0.0, d2 = 0.0;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        d1 = fma(sD[i][k], sq[el][v * NP + k + N * j], d1);
        d2 = fma(sD[j][k], sq[el][v * NP + i + N * k], d2);
      }
      dxi[el][v * NP + t] = d1;
      deta[el][v * NP + t] = d2;
    }
  }
  __syncthreads();
  const double sx = 2.0 / hx, sy = 2.0 / hy;
  // corrected gradient and total flux at the own point (overwrites dxi / deta)
  if (active) {
    double q[4], gxv[4], gyv[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      q[v] = sq[el][v * NP + t];
      double dx = dxi[el][v * NP + t];
      dx = fma(cq[el][0][j][v] - tq[el][0][j][v], sdgL[i], dx);
      dx = fma(cq[el][1][j][v] - tq[el][1][j][v], sdgR[i], dx);
      double dy = deta[el][v * NP + t];
      dy = fma(cq[el][2][i][v] - tq[el][2][i][v], sdgL[j], dy);
      dy = fma(cq[el][3][i][v] - tq[el][3][i][v], sdgR[j], dy);
      gxv[v] = sx * dx;
      gyv[v] = sy * dy;
    }
    double f[4], g[4], fv[4], gv[4];
    euler_fluxes(q, a.gam, f, g);
    visc_flux(q, gxv, gyv, a.gam, a.mu, a.kappa, fv, gv);
    // each thread reads and overwrites only its own point
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      dxi[el][v * NP + t] = f[v] - fv[v];
      deta[el][v * NP + t] = g[v] - gv[v];
    }
  }
  __syncthreads();
  if (!active) return;
  const long long base = e * 4 * NP + t;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    double dF = sdgL[i] * fnum[el][0][j][v];
    dF = fma(sdgR[i], fnum[el][1][j][v], dF);
#pragma unroll
    for (int k = 0; k < N; ++k) dF = fma(sDt[i][k], dxi[el][v * NP + k + N * j], dF);
    double dG = sdgL[j] * fnum[el][2][i][v];
    dG = fma(sdgR[j], fnum[el][3][i][v], dG);
#pragma unroll
    for (int k = 0; k < N; ++k) dG = fma(sDt[j][k], deta[el][v * NP + i + N * k], dG);
    double R = -fma(sx, dF, sy * dG);
    if (v == 1) R = fma(sq[el][t], a.gx, R);
    if (v == 3) R = fma(sq[el][NP + t], a.gx, R);
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

NsArgs make_args(fr_ctx* ctx) {
  NsArgs a{};
  a.tb = ctx->tb;
  a.fb = ctx->fb;
  a.hx = ctx->hx;
  a.hy = ctx->hy;
  a.ne = ctx->ne;
  a.nx = ctx->nx;
  a.ny = ctx->ny;
  a.wall_y = ctx->wall_y;
  a.gam = ctx->opts.gamma;
  a.mu = ctx->opts.mu;
  const double cp = ctx->opts.gamma / (ctx->opts.gamma - 1.0);  // R = 1
  a.kappa = ctx->opts.mu * cp / ctx->opts.prandtl;
  a.gx = ctx->opts.body_force_x;
  a.t_wall = ctx->opts.wall_temperature;
  a.beps = ctx->opts.block_eps_rel;
  a.tab = ctx->tab;
  return a;
}

template <int P>
int ns_launch(fr_ctx* ctx, int mode, const NsArgs& a, bool perturb_trace, cudaStream_t s, double wb,
              double wf) {
  constexpr int NP = (P + 1) * (P + 1), E = NsSlots<P>::E, NB = 4 * NP;
  const unsigned gt = (unsigned)((ctx->ne + E - 1) / E);
  const int fam = mode == 3 ? FR_KF_FACTOR : (mode == 0 ? FR_KF_RESIDUAL : FR_KF_JV);
  {
    ProfScope ps_(ctx, fam, s, wb, wf);  // one timed record for the trace + residual pair
    if (perturb_trace) k_ns_trace<P, true><<<gt, E * NP, 0, s>>>(a);
    else k_ns_trace<P, false><<<gt, E * NP, 0, s>>>(a);
    FRK_LAUNCHED(ctx);
    count_launch();  // the scope counted the trace kernel
    if (mode == 3) {
      k_ns_res<P, 3><<<(unsigned)((ctx->ne * NB + E - 1) / E), E * NP, 0, s>>>(a);
    } else {
      const long long nf = ctx->ne * 3 * (P + 1);
      k_ns_face<P><<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(a);
      FRK_LAUNCHED(ctx);
      count_launch();
      if (mode == 0) k_ns_cell<P, 0><<<gt, E * NP, 0, s>>>(a);
      else if (mode == 1) k_ns_cell<P, 1><<<gt, E * NP, 0, s>>>(a);
      else k_ns_cell<P, 2><<<gt, E * NP, 0, s>>>(a);
    }
  }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

int dispatch(fr_ctx* ctx, int mode, const NsArgs& a, bool perturb_trace, cudaStream_t s, double wb,
             double wf) {
  switch (ctx->p) {
    case 2: return ns_launch<2>(ctx, mode, a, perturb_trace, s, wb, wf);
    case 3: return ns_launch<3>(ctx, mode, a, perturb_trace, s, wb, wf);
    case 4: return ns_launch<4>(ctx, mode, a, perturb_trace, s, wb, wf);
    default: return set_error(ctx, FR_ERR_UNSUPPORTED, "degree %d not compiled", ctx->p);
  }
}

}  // namespace

int launch_ns_residual(fr_ctx* ctx, int mode, const double* U, const double* z, const double* R0,
                       const double* b, double* out, double shift, const double* eps2,
                       const int* done, cudaStream_t s) {
  NsArgs a = make_args(ctx);
  a.U = U;
  a.z = z;
  a.R0 = R0;
  a.b = b;
  a.out = out;
  a.eps2 = eps2;
  a.done = done;
  a.shift = shift;
  // inside a GMRES cycle both kernels return at once once the cycle is done
  const double nd = (double)ctx->ndof;
  const bool in_cycle = done != nullptr;
  const double wb = in_cycle ? 0.0 : (mode == 0 ? 16.0 : (mode == 1 ? 32.0 : 40.0)) * nd;
  const double wf = in_cycle ? 0.0 : ns_residual_flops_per_element(ctx->p) * (double)ctx->ne + (mode == 0 ? 0.0 : 6.0 * nd);
  return dispatch(ctx, mode, a, mode != 0, s, wb, wf);
}

int launch_ns_factor(fr_ctx* ctx, const double* U, double shift, cudaStream_t s) {
  // R0 of the element-local residuals = R(U) with the same (unperturbed) traces
  NsArgs a = make_args(ctx);
  a.U = U;
  a.z = nullptr;
  a.out = ctx->rloc;
  a.shift = 0.0;
  FRK_TRY(dispatch(ctx, 0, a, false, s, 0.0, 0.0));
  a.R0 = ctx->rloc;
  a.out = ctx->mst;
  a.shift = shift;
  FRK_TRY(dispatch(ctx, 3, a, false, s, 0.0, 0.0));
  return launch_block_invert(ctx, ctx->mst, 0.0, s);
}

}  // namespace frk
