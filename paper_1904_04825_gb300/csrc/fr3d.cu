// 3D Navier-Stokes FR residual on periodic axis-aligned hexahedra (Sec. 2-3
// in three reference directions, BR2 common gradients, Eqs. com_q and
// com_grad_q, g'(+-1) = +-(P+1)(P+2)/2) and the kinetic-energy dissipation
// rate of the Taylor-Green study (Sec. 5).  mu = 0 gives the Euler residual.
//
// Layout: U[ne][5][Np], Np = N^3 (N = p+1), point i + N j + N^2 k (i along x),
// element ix + nx (iy + ny iz).  Face 2d is the low face of direction d
// (d = 0 x, 1 y, 2 z), face 2d+1 the high face; face point f = a + N b over
// the two other directions in increasing order.
//
// R(U), A z and b - A z take three kernels, like the 2D viscous path:
//  k3_trace: per element, the (possibly perturbed) state and its own
//    polynomial gradient traced to the 6 N^2 face points -> trace buffer
//    [ne][6][N^2][5][4] = (q, q_x, q_y, q_z).
//  k3_face:  per low face point of every element (each face once), the
//    common solution, BR2 common gradient and common total normal flux
//    (Rusanov inviscid minus viscous) from the two traces -> face buffer
//    [ne][3][N^2][10] = (q_com, f_n).
//  k3_cell:  per element, the FR-corrected gradient, the total fluxes along
//    x, y, z at the solution points and their corrected divergence with the
//    six faces' common fluxes (low faces its own, high faces the neighbours'
//    low faces), then the output of the mode.  Both elements of a face read
//    the same stored flux, so conservation holds to round-off.
// Element-Jacobi columns (k3_cell mode 3, degrees 1 to 3): slot = (element,
// column c), own state perturbed in DOF c by eps_c = beps (1 + |q_c|), own
// traces recomputed in the kernel, neighbour traces frozen (trace buffer of
// the unperturbed state); the slot forms its six faces' common data itself
// and stages column c of shift I - J_ee for the inversion kernel.  Degree 3
// (320 x 320 blocks, 800 KB each in FP64) stages and inverts the elements in
// chunks, so the FP64 staging holds one chunk.
#include "device.cuh"

namespace frk {
namespace {

struct F3Args {
  const double* U;
  const double* z;
  const double* R0;
  const double* b;
  double* out;
  double* tb;          // traces [ne][6][N^2][5][4]
  double* fb;          // low-face common data [ne][3][N^2][10]
  const double* hx;
  const double* hy;
  const double* hz;
  const double* eps2;
  const int* done;
  long long ne;
  long long e0, nchunk;  // mode 3: the elements e0 .. e0 + nchunk - 1, columns staged from out[0]
  float* r0f;            // mode 3 in FP32: element-local R(U) of the chunk, [nchunk][NB]
  const float* tbf;      // mode 3 in FP32: the trace buffer in FP32
  // A z with FP32 linear parts (jv_precision 1): caches at the linearisation
  // point U and the FP32 buffers of the product
  double* ltb;           // traces of U [ne][6][N^2][20]
  double* lfb;           // low-face common data of U [ne][3][N^2][10]
  double* lg;            // corrected gradient of U at the points [ne][3][5][Np]
  double* lf;            // total fluxes at U at the points [ne][3][5][Np]
  float* tbz;            // traces of z and of its gradient [ne][6][N^2][20]
  float* fbz;            // per unit eps: q_com differences and f_n differences [ne][3][N^2][10]
  double* lgc;           // BR2 common gradient of U at the low-face points [ne][3][N^2][15]
  int write_gc;          // cache pass: k3_face writes lgc
  int r0_pass;           // mode 3 in FP32: 1 = write r0f (one unperturbed slot per element)
  int nx, ny, nz;
  double gam, mu, kappa, shift, beps;
  Tables tab;
};

// elements per CTA, one thread per solution point
template <int P> struct F3Slots;
template <> struct F3Slots<1> { static constexpr int E = 16; };
template <> struct F3Slots<2> { static constexpr int E = 8; };
template <> struct F3Slots<3> { static constexpr int E = 4; };
template <> struct F3Slots<4> { static constexpr int E = 2; };

// values (of type T) of dynamic shared memory per element of k3_cell: state,
// three derivative / flux arrays, q_com - q_face and f_n on the 6 N^2 face points
template <int P, typename T = double> struct CellLayout {
  static constexpr int N = P + 1, N2 = N * N, NP = N2 * N;
  static constexpr int PER = 20 * NP + 60 * N2;
  static constexpr size_t BYTES = (size_t)F3Slots<P>::E * PER * sizeof(T);
};

// The pointwise and face functions below take the arithmetic type T: double
// for R(U) and A z, float for the FP32 element-Jacobi columns.
template <int N, typename T>
__device__ __forceinline__ T tsum3(const T* x, int stride, const T* c) {
  T s = c[0] * x[0];
#pragma unroll
  for (int l = 1; l < N; ++l) s = fma(c[l], x[l * stride], s);
  return s;
}

// first point and stride of the line through face point f normal to direction d
template <int N>
__device__ __forceinline__ void line_of(int d, int f, int* off, int* stride) {
  constexpr int N2 = N * N;
  if (d == 0) { *off = N * (f % N) + N2 * (f / N); *stride = 1; }
  else if (d == 1) { *off = (f % N) + N2 * (f / N); *stride = N; }
  else { *off = f; *stride = N2; }
}

// inviscid flux along direction d and |v_d| + c (selects instead of indexing
// by d, so the arrays stay in registers when d is not a constant)
template <typename T>
__device__ __forceinline__ T flux3(const T q[5], int d, T gam, T f[5]) {
  const T ri = T(1) / q[0];
  const T md = d == 0 ? q[1] : (d == 1 ? q[2] : q[3]);
  const T vd = md * ri;
  const T p = (gam - T(1)) * (q[4] - T(0.5) * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) * ri);
  f[0] = md;
  f[1] = fma(q[1], vd, d == 0 ? p : T(0));
  f[2] = fma(q[2], vd, d == 1 ? p : T(0));
  f[3] = fma(q[3], vd, d == 2 ? p : T(0));
  f[4] = vd * (q[4] + p);
  return fabs(vd) + sqrt(gam * p * ri);
}

template <typename T>
__device__ __forceinline__ void rusanov3(const T qm[5], const T qp[5], int d, T gam, T fn[5]) {
  T fm[5], fp[5];
  const T lm = flux3(qm, d, gam, fm);
  const T lp = flux3(qp, d, gam, fp);
  const T lam = fmax(lm, lp);
#pragma unroll
  for (int v = 0; v < 5; ++v) fn[v] = T(0.5) * (fm[v] + fp[v]) - T(0.5) * lam * (qp[v] - qm[v]);
}

// viscous fluxes along the directions d with mask bit d set, from q and the
// gradients g[c][v] (c: direction); R = 1
template <typename T>
__device__ __forceinline__ void visc3(const T q[5], const T g[3][5], T gam, T mu, T kappa, int mask, T fv[3][5]) {
  const T ri = T(1) / q[0];
  const T vel[3] = {q[1] * ri, q[2] * ri, q[3] * ri};
  const T e = q[4] * ri;
  T dv[3][3];  // dv[c][m] = d v_m / d x_c
  T dT[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int m = 0; m < 3; ++m) dv[c][m] = (g[c][1 + m] - vel[m] * g[c][0]) * ri;
    dT[c] = (gam - T(1)) * ((g[c][4] - e * g[c][0]) * ri - (vel[0] * dv[c][0] + vel[1] * dv[c][1] + vel[2] * dv[c][2]));
  }
  const T div = dv[0][0] + dv[1][1] + dv[2][2];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (!(mask & (1 << d))) continue;
    T tau[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) tau[m] = mu * (dv[d][m] + dv[m][d]);
    tau[d] -= T(2.0 / 3.0) * mu * div;
    fv[d][0] = T(0);
    fv[d][1] = tau[0];
    fv[d][2] = tau[1];
    fv[d][3] = tau[2];
    fv[d][4] = vel[0] * tau[0] + vel[1] * tau[1] + vel[2] * tau[2] + kappa * dT[d];
  }
}

// common solution and total normal flux on a face normal to d from the (-)
// and (+) traces m, pp ([v][q, q_x, q_y, q_z]); hm, hp: the two elements'
// sizes along d; cbr2 = (P+1)(P+2)/2
template <typename T>
__device__ __forceinline__ void common3(const T m[5][4], const T pp[5][4], int d, T hm, T hp, T cbr2,
                                        const F3Args& a, T qc[5], T fn[5], T (*gout)[5] = nullptr) {
  T qm[5], qp[5], g[3][5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    qm[v] = m[v][0];
    qp[v] = pp[v][0];
    qc[v] = T(0.5) * (qm[v] + qp[v]);
#pragma unroll
    for (int c = 0; c < 3; ++c) g[c][v] = T(0.5) * (m[v][1 + c] + pp[v][1 + c]);
    const T rm = (T(2) / hm) * cbr2 * (qc[v] - qm[v]);   // lifting of the (-) element
    const T rp = -(T(2) / hp) * cbr2 * (qc[v] - qp[v]);  // lifting of the (+) element
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c == d) g[c][v] = T(0.5) * ((m[v][1 + c] + rm) + (pp[v][1 + c] + rp));
  }
  T fi[5], fv[3][5];
  rusanov3(qm, qp, d, (T)a.gam, fi);
  visc3(qc, g, (T)a.gam, (T)a.mu, (T)a.kappa, 1 << d, fv);
#pragma unroll
  for (int v = 0; v < 5; ++v) fn[v] = fi[v] - (d == 0 ? fv[0][v] : (d == 1 ? fv[1][v] : fv[2][v]));
  if (gout) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int v = 0; v < 5; ++v) gout[c][v] = g[c][v];
  }
}

__device__ __forceinline__ void coords(long long e, const F3Args& a, int* ix, int* iy, int* iz) {
  *ix = (int)(e % a.nx);
  const long long r = e / a.nx;
  *iy = (int)(r % a.ny);
  *iz = (int)(r / a.ny);
}

__device__ __forceinline__ long long elem(int ix, int iy, int iz, const F3Args& a) {
  return (long long)ix + (long long)a.nx * ((long long)iy + (long long)a.ny * iz);
}

// neighbour of (ix, iy, iz) across face `face` (periodic) and its size along the face normal
__device__ __forceinline__ long long neighbour(int ix, int iy, int iz, int face, const F3Args& a, double* h) {
  const int d = face >> 1, s = (face & 1) ? 1 : -1;
  if (d == 0) { ix = (ix + a.nx + s) % a.nx; *h = a.hx[ix]; }
  else if (d == 1) { iy = (iy + a.ny + s) % a.ny; *h = a.hy[iy]; }
  else { iz = (iz + a.nz + s) % a.nz; *h = a.hz[iz]; }
  return elem(ix, iy, iz, a);
}

// reference derivatives of the 5 variables at point t of one element
template <int N, typename T>
__device__ __forceinline__ void ref_derivs(const T* sq, const T (*sD)[N], int t, T* d0, T* d1, T* d2) {
  constexpr int N2 = N * N, NP = N2 * N;
  const int i = t % N, j = (t / N) % N, k = t / N2;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const T* x = sq + v * NP;
    T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll
    for (int l = 0; l < N; ++l) {
      a0 = fma(sD[i][l], x[l + N * j + N2 * k], a0);
      a1 = fma(sD[j][l], x[i + N * l + N2 * k], a1);
      a2 = fma(sD[k][l], x[i + N * j + N2 * l], a2);
    }
    d0[v * NP + t] = a0;
    d1[v * NP + t] = a1;
    d2[v * NP + t] = a2;
  }
}

// full trace (q and physical gradient) of face point (face, f)
template <int N, typename T>
__device__ __forceinline__ void own_trace(const T* sq, const T* d0, const T* d1, const T* d2, int face, int f,
                                          const T s[3], const T* lm, const T* lp, T o[5][4]) {
  constexpr int NP = N * N * N;
  int off, stride;
  line_of<N>(face >> 1, f, &off, &stride);
  const T* c = (face & 1) ? lp : lm;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    o[v][0] = tsum3<N>(sq + v * NP + off, stride, c);
    o[v][1] = s[0] * tsum3<N>(d0 + v * NP + off, stride, c);
    o[v][2] = s[1] * tsum3<N>(d1 + v * NP + off, stride, c);
    o[v][3] = s[2] * tsum3<N>(d2 + v * NP + off, stride, c);
  }
}

template <int P, bool PERTURB>
__global__ void __launch_bounds__(256) k3_trace(const F3Args a) {
  constexpr int N = P + 1, N2 = N * N, NP = N2 * N, E = F3Slots<P>::E;
  __shared__ double sq[E][5 * NP], dd[3][E][5 * NP];
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
    for (int v = 0; v < 5; ++v) {
      const long long o = e * 5 * NP + v * NP + t;
      sq[el][v * NP + t] = PERTURB ? fma(eps, a.z[o], a.U[o]) : a.U[o];
    }
  }
  __syncthreads();
  if (active) ref_derivs<N>(sq[el], sD, t, dd[0][el], dd[1][el], dd[2][el]);
  __syncthreads();
  if (!active) return;
  int ix, iy, iz;
  coords(e, a, &ix, &iy, &iz);
  const double s[3] = {2.0 / a.hx[ix], 2.0 / a.hy[iy], 2.0 / a.hz[iz]};
  for (int fp = t; fp < 6 * N2; fp += NP) {
    const int face = fp / N2, f = fp % N2;
    double o[5][4];
    own_trace<N>(sq[el], dd[0][el], dd[1][el], dd[2][el], face, f, s, slm, slp, o);
    double* dst = a.tb + ((e * 6 + face) * N2 + f) * 20;
#pragma unroll
    for (int v = 0; v < 5; ++v)
#pragma unroll
      for (int c = 0; c < 4; ++c) dst[v * 4 + c] = o[v][c];
  }
}

// one thread per (element, direction d, point of its low face d)
template <int P>
__global__ void __launch_bounds__(256) k3_face(const F3Args a) {
  constexpr int N = P + 1, N2 = N * N;
  constexpr double cbr2 = (P + 1) * (P + 2) / 2.0;
  if (a.done && *a.done) return;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= a.ne * 3 * N2) return;
  const int f = (int)(tid % N2);
  const int d = (int)((tid / N2) % 3);
  const long long e = tid / (3 * N2);
  int ix, iy, iz;
  coords(e, a, &ix, &iy, &iz);
  double hm;
  const long long nbe = neighbour(ix, iy, iz, 2 * d, a, &hm);
  const double hp = d == 0 ? a.hx[ix] : (d == 1 ? a.hy[iy] : a.hz[iz]);
  const double* own = a.tb + ((e * 6 + 2 * d) * N2 + f) * 20;
  const double* nb = a.tb + ((nbe * 6 + 2 * d + 1) * N2 + f) * 20;
  double m[5][4], pp[5][4], qc[5], fn[5];
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      m[v][c] = nb[v * 4 + c];
      pp[v][c] = own[v * 4 + c];
    }
  double gc[3][5];
  common3(m, pp, d, hm, hp, cbr2, a, qc, fn, a.write_gc ? gc : nullptr);
  double* dst = a.fb + ((e * 3 + d) * N2 + f) * 10;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    dst[v] = qc[v];
    dst[5 + v] = fn[v];
  }
  if (a.write_gc) {  // cache pass of the FP32-linear-parts A z: the common gradient at U
    double* g = a.lgc + ((e * 3 + d) * N2 + f) * 15;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int v = 0; v < 5; ++v) g[c * 5 + v] = gc[c][v];
  }
}

// MODE 0: out = R(U); 1: out = A z; 2: out = b - A z (state U + eps z, face
// data from the face buffer); 3: element-Jacobi column (see the file header);
// 4: the caches of the FP32-linear-parts A z at U (corrected gradient and
// total fluxes at the points to a.lg, a.lf; face data from the face buffer).
// T: arithmetic type, double except for FP32 element-Jacobi columns (MODE 3,
// T = float): then a first pass (a.r0_pass) writes the element-local R(U) of
// each element of the chunk in FP32 to a.r0f, and the columns pass divides
// R(U + eps_c e_c) - r0f by the step actually taken in FP32.
template <int P, int MODE, typename T = double>
__global__ void __launch_bounds__(256) k3_cell(const F3Args a) {
  using L = CellLayout<P, T>;
  constexpr int N = P + 1, N2 = N * N, NP = N2 * N, E = F3Slots<P>::E, NB = 5 * NP;
  constexpr bool PERTURB = MODE == 1 || MODE == 2;
  constexpr bool JAC = MODE == 3;
  constexpr bool J32 = JAC && sizeof(T) == 4;
  static_assert(sizeof(T) == 8 || JAC, "R(U) and A z run in FP64");
  constexpr T cbr2 = T((P + 1) * (P + 2) / 2.0);
  extern __shared__ __align__(16) unsigned char smem3_raw[];
  T* smem3 = reinterpret_cast<T*>(smem3_raw);
  __shared__ T sD[N][N], sDt[N][N], slm[N], slp[N], sdgL[N], sdgR[N];
  __shared__ float sceps[E];  // FP32 columns: the step each slot took
  if (a.done && *a.done) return;
  if (threadIdx.x < N * N) {
    sD[threadIdx.x / N][threadIdx.x % N] = (T)a.tab.D[threadIdx.x / N][threadIdx.x % N];
    sDt[threadIdx.x / N][threadIdx.x % N] = (T)a.tab.Dt[threadIdx.x / N][threadIdx.x % N];
  }
  if (threadIdx.x < N) {
    slm[threadIdx.x] = (T)a.tab.lm[threadIdx.x];
    slp[threadIdx.x] = (T)a.tab.lp[threadIdx.x];
    sdgL[threadIdx.x] = (T)a.tab.dgL[threadIdx.x];
    sdgR[threadIdx.x] = (T)a.tab.dgR[threadIdx.x];
  }
  const int el = threadIdx.x / NP, t = threadIdx.x % NP;
  T* base = smem3 + (size_t)(el < E ? el : 0) * L::PER;
  T* sq = base;                 // [5][NP]
  T* d0 = sq + 5 * NP;          // derivatives, then fluxes, along x / y / z
  T* d1 = d0 + 5 * NP;
  T* d2 = d1 + 5 * NP;
  T* dq = d2 + 5 * NP;          // [6][N2][5] q_com - q_face
  T* fn = dq + 30 * N2;         // [6][N2][5] common total normal flux
  const bool r0_pass = J32 && a.r0_pass;
  const long long slot = (long long)blockIdx.x * E + el;
  const long long nslots = JAC ? (r0_pass ? a.nchunk : a.nchunk * NB) : a.ne;
  const bool active = el < E && slot < nslots;
  const long long e = JAC ? a.e0 + (r0_pass ? slot : slot / NB) : slot;
  const int col = JAC && !r0_pass ? (int)(slot % NB) : -1;
  double eps = 0.0, ieps = 0.0;
  if (PERTURB) {
    eps = a.eps2[0];
    ieps = a.eps2[1];
  }
  int ix = 0, iy = 0, iz = 0;
  T s[3] = {T(1), T(1), T(1)}, hown[3] = {T(1), T(1), T(1)};
  double ceps = 0.0;  // FD step of the column (FP32: the step taken after rounding)
  if (active) {
    coords(e, a, &ix, &iy, &iz);
    hown[0] = (T)a.hx[ix];
    hown[1] = (T)a.hy[iy];
    hown[2] = (T)a.hz[iz];
#pragma unroll
    for (int c = 0; c < 3; ++c) s[c] = T(2) / hown[c];
    if (JAC && !J32 && col >= 0) {
      const double uc = a.U[e * NB + col];
      ceps = a.beps * (1.0 + fabs(uc));
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const long long o = e * NB + v * NP + t;
      double qv = PERTURB ? fma(eps, a.z[o], a.U[o]) : a.U[o];
      if (JAC && !J32 && v * NP + t == col) qv += ceps;
      T tq = (T)qv;
      if (J32 && v * NP + t == col) {
        // the step in FP32 (no FP64 arithmetic in this kernel: on GB300 one
        // FP64 operation costs as much issue as 64 FP32 ones)
        const float c32 = (float)a.beps * (1.f + fabsf((float)tq));
        const float pq = (float)tq + c32;
        sceps[el] = pq - (float)tq;
        tq = pq;
      }
      sq[v * NP + t] = tq;
    }
  }
  __syncthreads();
  const float ceps32 = J32 && active && col >= 0 ? sceps[el] : 1.f;
  if (active) ref_derivs<N>(sq, sD, t, d0, d1, d2);
  __syncthreads();
  // face data of the six faces
  if (active) {
    for (int fp = t; fp < 6 * N2; fp += NP) {
      const int face = fp / N2, f = fp % N2, d = face >> 1;
      T qface[5], qc[5], fnum[5];
      if (JAC) {
        T o[5][4], nbt[5][4];
        own_trace<N>(sq, d0, d1, d2, face, f, s, slm, slp, o);
        double hn;
        const long long nbe = neighbour(ix, iy, iz, face, a, &hn);
        const long long so = ((nbe * 6 + (face ^ 1)) * N2 + f) * 20;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          qface[v] = o[v][0];
#pragma unroll
          for (int c = 0; c < 4; ++c) nbt[v][c] = J32 ? (T)a.tbf[so + v * 4 + c] : (T)a.tb[so + v * 4 + c];
        }
        if (face & 1) common3(o, nbt, d, hown[d], (T)hn, cbr2, a, qc, fnum);
        else common3(nbt, o, d, (T)hn, hown[d], cbr2, a, qc, fnum);
      } else {
        int off, stride;
        line_of<N>(d, f, &off, &stride);
        const T* c = (face & 1) ? slp : slm;
#pragma unroll
        for (int v = 0; v < 5; ++v) qface[v] = tsum3<N>(sq + v * NP + off, stride, c);
        long long fe = e;
        if (face & 1) {
          double hn;
          fe = neighbour(ix, iy, iz, face, a, &hn);
        }
        const double* src = a.fb + ((fe * 3 + d) * N2 + f) * 10;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          qc[v] = (T)src[v];
          fnum[v] = (T)src[5 + v];
        }
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        dq[(face * N2 + f) * 5 + v] = qc[v] - qface[v];
        fn[(face * N2 + f) * 5 + v] = fnum[v];
      }
    }
  }
  __syncthreads();
  const int i = t % N, j = (t / N) % N, k = t / N2;
  const int f0 = j + N * k, f1 = i + N * k, f2 = i + N * j;  // this point's face points per direction
  // corrected gradient and total fluxes at the own point (overwrite d0..d2)
  if (active) {
    T q[5], g[3][5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      q[v] = sq[v * NP + t];
      T x = d0[v * NP + t];
      x = fma(dq[(0 * N2 + f0) * 5 + v], sdgL[i], x);
      x = fma(dq[(1 * N2 + f0) * 5 + v], sdgR[i], x);
      T y = d1[v * NP + t];
      y = fma(dq[(2 * N2 + f1) * 5 + v], sdgL[j], y);
      y = fma(dq[(3 * N2 + f1) * 5 + v], sdgR[j], y);
      T zz = d2[v * NP + t];
      zz = fma(dq[(4 * N2 + f2) * 5 + v], sdgL[k], zz);
      zz = fma(dq[(5 * N2 + f2) * 5 + v], sdgR[k], zz);
      g[0][v] = s[0] * x;
      g[1][v] = s[1] * y;
      g[2][v] = s[2] * zz;
    }
    T fv[3][5];
    visc3(q, g, (T)a.gam, (T)a.mu, (T)a.kappa, 7, fv);
    T* dst[3] = {d0, d1, d2};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      T fi[5];
      (void)flux3(q, d, (T)a.gam, fi);
      // each thread reads and overwrites only its own point
#pragma unroll
      for (int v = 0; v < 5; ++v) dst[d][v * NP + t] = fi[v] - fv[d][v];
    }
    if (MODE == 4) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const long long o = ((e * 3 + c) * 5 + v) * NP + t;
          a.lg[o] = (double)g[c][v];
          a.lf[o] = (double)dst[c][v * NP + t];
        }
    }
  }
  if (MODE == 4) return;
  __syncthreads();
  if (!active) return;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const T* F = d0 + v * NP;
    const T* G = d1 + v * NP;
    const T* H = d2 + v * NP;
    T dF = sdgL[i] * fn[(0 * N2 + f0) * 5 + v];
    dF = fma(sdgR[i], fn[(1 * N2 + f0) * 5 + v], dF);
    T dG = sdgL[j] * fn[(2 * N2 + f1) * 5 + v];
    dG = fma(sdgR[j], fn[(3 * N2 + f1) * 5 + v], dG);
    T dH = sdgL[k] * fn[(4 * N2 + f2) * 5 + v];
    dH = fma(sdgR[k], fn[(5 * N2 + f2) * 5 + v], dH);
#pragma unroll
    for (int l = 0; l < N; ++l) {
      dF = fma(sDt[i][l], F[l + N * j + N2 * k], dF);
      dG = fma(sDt[j][l], G[i + N * l + N2 * k], dG);
      dH = fma(sDt[k][l], H[i + N * j + N2 * l], dH);
    }
    const T R = -fma(s[0], dF, fma(s[1], dG, s[2] * dH));
    const long long o = e * NB + v * NP + t;
    if (MODE == 0) {
      a.out[o] = (double)R;
    } else if (MODE == 3) {
      // column col of M = shift I - J_ee, staged column-major [col][row]
      const int row = v * NP + t;
      double* dst = a.out + ((e - a.e0) * NB + col) * NB + row;
      if (r0_pass) {
        a.r0f[(e - a.e0) * NB + row] = (float)R;
      } else if (J32) {  // the difference quotient and the column in FP32
        const float dq32 = ((float)R - a.r0f[(e - a.e0) * NB + row]) / ceps32;
        *dst = (double)((row == col ? (float)a.shift : 0.f) - dq32);
      } else {
        *dst = (row == col ? a.shift : 0.0) - ((double)R - a.R0[o]) / ceps;
      }
    } else {
      const double zo = a.z[o];
      const double Az = eps > 0.0 ? fma(-((double)R - a.R0[o]), ieps, a.shift * zo) : a.shift * zo;
      a.out[o] = MODE == 2 ? a.b[o] - Az : Az;
    }
  }
}

// ---- A z with FP32 linear parts (jv_precision 1) ----
// R(U + eps z) - R(U) splits into linear maps (reference derivatives, traces,
// BR2 liftings, the FR correction of the gradient, the corrected divergence)
// and the nonlinear pointwise and common fluxes.  The linear maps act on z
// in FP32; the fluxes are evaluated in FP64 at U + eps z from the cached
// state, traces and corrected gradient at U plus eps times their FP32
// counterparts of z, and differenced in FP64 against the fluxes cached at U;
// the differences, divided by eps, go through the corrected divergence in
// FP32.  Mode 1: out = shift z - (R(U + eps z) - R(U)) / eps; mode 2: b - that.

// traces of z and of its physical gradient at the 6 N^2 face points, FP32
template <int P>
__global__ void __launch_bounds__(256) k3z_trace(const F3Args a) {
  constexpr int N = P + 1, N2 = N * N, NP = N2 * N, E = F3Slots<P>::E;
  __shared__ float sq[E][5 * NP], dd[3][E][5 * NP];
  __shared__ float sD[N][N], slm[N], slp[N];
  if (threadIdx.x < N * N) sD[threadIdx.x / N][threadIdx.x % N] = (float)a.tab.D[threadIdx.x / N][threadIdx.x % N];
  if (threadIdx.x < N) {
    slm[threadIdx.x] = (float)a.tab.lm[threadIdx.x];
    slp[threadIdx.x] = (float)a.tab.lp[threadIdx.x];
  }
  if (a.done && *a.done) return;
  const int el = threadIdx.x / NP, t = threadIdx.x % NP;
  const long long e = (long long)blockIdx.x * E + el;
  const bool active = el < E && e < a.ne;
  if (active) {
#pragma unroll
    for (int v = 0; v < 5; ++v) sq[el][v * NP + t] = (float)a.z[e * 5 * NP + v * NP + t];
  }
  __syncthreads();
  if (active) ref_derivs<N>(sq[el], sD, t, dd[0][el], dd[1][el], dd[2][el]);
  __syncthreads();
  if (!active) return;
  int ix, iy, iz;
  coords(e, a, &ix, &iy, &iz);
  // 2 / h in FP32 (an FP64 division costs this FP32 kernel more than all its FP32 work)
  const float s[3] = {2.f / (float)a.hx[ix], 2.f / (float)a.hy[iy], 2.f / (float)a.hz[iz]};
  for (int fp = t; fp < 6 * N2; fp += NP) {
    const int face = fp / N2, f = fp % N2;
    float o[5][4];
    own_trace<N>(sq[el], dd[0][el], dd[1][el], dd[2][el], face, f, s, slm, slp, o);
    float* dst = a.tbz + ((e * 6 + face) * N2 + f) * 20;
#pragma unroll
    for (int v = 0; v < 5; ++v)
#pragma unroll
      for (int c = 0; c < 4; ++c) dst[v * 4 + c] = o[v][c];
  }
}

// per low face point: the common data at U + eps z in FP64 from the cached
// traces at U and eps times the FP32 traces of z; per unit eps, the change
// of q_com (linear: the mean of the two traces of z) and of the common total
// normal flux (FP64 difference against the cache) to a.fbz
template <int P>
__global__ void __launch_bounds__(256) k3z_face(const F3Args a) {
  constexpr int N = P + 1, N2 = N * N;
  constexpr double cbr2 = (P + 1) * (P + 2) / 2.0;
  if (a.done && *a.done) return;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= a.ne * 3 * N2) return;
  const int f = (int)(tid % N2);
  const int d = (int)((tid / N2) % 3);
  const long long e = tid / (3 * N2);
  const double eps = a.eps2[0];
  const double ieps = eps > 0.0 ? a.eps2[1] : 0.0;
  int ix, iy, iz;
  coords(e, a, &ix, &iy, &iz);
  double hm;
  const long long nbe = neighbour(ix, iy, iz, 2 * d, a, &hm);
  const double hp = d == 0 ? a.hx[ix] : (d == 1 ? a.hy[iy] : a.hz[iz]);
  const long long om = ((nbe * 6 + 2 * d + 1) * N2 + f) * 20;  // (-) side: the neighbour's high face
  const long long op = ((e * 6 + 2 * d) * N2 + f) * 20;        // (+) side: this element's low face
  const long long fo = (e * 3 + d) * N2 + f;
  // the linear part in FP32: q_com and the BR2 common gradient of z (the
  // same average and liftings as common3)
  const float cb = (float)cbr2;
  float qcz[5], gz[3][5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const float zm = a.tbz[om + v * 4], zp = a.tbz[op + v * 4];
    qcz[v] = 0.5f * (zm + zp);
#pragma unroll
    for (int c = 0; c < 3; ++c) gz[c][v] = 0.5f * (a.tbz[om + v * 4 + 1 + c] + a.tbz[op + v * 4 + 1 + c]);
    const float rm = (2.f / (float)hm) * cb * (qcz[v] - zm);
    const float rp = -(2.f / (float)hp) * cb * (qcz[v] - zp);
#pragma unroll
    for (int c = 0; c < 3; ++c)  // selected, not indexed by d, so gz stays in registers
      if (c == d) gz[c][v] = 0.5f * ((a.tbz[om + v * 4 + 1 + c] + rm) + (a.tbz[op + v * 4 + 1 + c] + rp));
  }
  // the fluxes at U + eps z in FP64: face states for the Rusanov flux, q_com
  // and the common gradient for the viscous flux, each = cache + eps * FP32 part
  const double* f0 = a.lfb + fo * 10;
  const double* g0 = a.lgc + fo * 15;
  double qm[5], qp[5], qc[5], g[3][5], fi[5], fv[3][5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    qm[v] = fma(eps, (double)a.tbz[om + v * 4], a.ltb[om + v * 4]);
    qp[v] = fma(eps, (double)a.tbz[op + v * 4], a.ltb[op + v * 4]);
    qc[v] = fma(eps, (double)qcz[v], f0[v]);
#pragma unroll
    for (int c = 0; c < 3; ++c) g[c][v] = fma(eps, (double)gz[c][v], g0[c * 5 + v]);
  }
  rusanov3(qm, qp, d, a.gam, fi);
  visc3(qc, g, a.gam, a.mu, a.kappa, 1 << d, fv);
  float* dst = a.fbz + fo * 10;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const double fnv = fi[v] - (d == 0 ? fv[0][v] : (d == 1 ? fv[1][v] : fv[2][v]));
    dst[v] = qcz[v];
    dst[5 + v] = (float)((fnv - f0[5 + v]) * ieps);
  }
}

// per element: FP32 derivatives and corrected gradient of z; at each point
// the fluxes at U + eps z in FP64 (state U + eps z, gradient = cached
// corrected gradient + eps times that of z) minus the cached fluxes, per
// unit eps, then the corrected divergence in FP32
template <int P, int MODE>
__global__ void __launch_bounds__(256) k3z_cell(const F3Args a) {
  using L = CellLayout<P, float>;
  constexpr int N = P + 1, N2 = N * N, NP = N2 * N, E = F3Slots<P>::E, NB = 5 * NP;
  static_assert(MODE == 1 || MODE == 2, "A z or b - A z");
  extern __shared__ __align__(16) unsigned char smemz_raw[];
  float* smemz = reinterpret_cast<float*>(smemz_raw);
  __shared__ float sD[N][N], sDt[N][N], slm[N], slp[N], sdgL[N], sdgR[N];
  if (a.done && *a.done) return;
  if (threadIdx.x < N * N) {
    sD[threadIdx.x / N][threadIdx.x % N] = (float)a.tab.D[threadIdx.x / N][threadIdx.x % N];
    sDt[threadIdx.x / N][threadIdx.x % N] = (float)a.tab.Dt[threadIdx.x / N][threadIdx.x % N];
  }
  if (threadIdx.x < N) {
    slm[threadIdx.x] = (float)a.tab.lm[threadIdx.x];
    slp[threadIdx.x] = (float)a.tab.lp[threadIdx.x];
    sdgL[threadIdx.x] = (float)a.tab.dgL[threadIdx.x];
    sdgR[threadIdx.x] = (float)a.tab.dgR[threadIdx.x];
  }
  const int el = threadIdx.x / NP, t = threadIdx.x % NP;
  float* base = smemz + (size_t)(el < E ? el : 0) * L::PER;
  float* sz = base;              // [5][NP] z
  float* d0 = sz + 5 * NP;       // derivatives of z, then flux differences per unit eps
  float* d1 = d0 + 5 * NP;
  float* d2 = d1 + 5 * NP;
  float* dq = d2 + 5 * NP;       // [6][N2][5] q_com(z) - q_face(z)
  float* fn = dq + 30 * N2;      // [6][N2][5] common flux differences per unit eps
  const long long e = (long long)blockIdx.x * E + el;
  const bool active = el < E && e < a.ne;
  const double eps = a.eps2[0];
  const double ieps = eps > 0.0 ? a.eps2[1] : 0.0;
  int ix = 0, iy = 0, iz = 0;
  float s[3] = {1.f, 1.f, 1.f};
  if (active) {
    coords(e, a, &ix, &iy, &iz);
    s[0] = 2.f / (float)a.hx[ix];
    s[1] = 2.f / (float)a.hy[iy];
    s[2] = 2.f / (float)a.hz[iz];
#pragma unroll
    for (int v = 0; v < 5; ++v) sz[v * NP + t] = (float)a.z[e * NB + v * NP + t];
  }
  __syncthreads();
  if (active) ref_derivs<N>(sz, sD, t, d0, d1, d2);
  __syncthreads();
  if (active) {
    for (int fp = t; fp < 6 * N2; fp += NP) {
      const int face = fp / N2, f = fp % N2, d = face >> 1;
      int off, stride;
      line_of<N>(d, f, &off, &stride);
      const float* c = (face & 1) ? slp : slm;
      long long fe = e;
      if (face & 1) {
        double hn;
        fe = neighbour(ix, iy, iz, face, a, &hn);
      }
      const float* src = a.fbz + ((fe * 3 + d) * N2 + f) * 10;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        dq[(face * N2 + f) * 5 + v] = src[v] - tsum3<N>(sz + v * NP + off, stride, c);
        fn[(face * N2 + f) * 5 + v] = src[5 + v];
      }
    }
  }
  __syncthreads();
  const int i = t % N, j = (t / N) % N, k = t / N2;
  const int f0 = j + N * k, f1 = i + N * k, f2 = i + N * j;
  if (active) {
    double q[5], g[3][5];
    const long long cb = e * 15 * NP + t;  // caches [e][3][5][NP]
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const long long o = e * NB + v * NP + t;
      q[v] = fma(eps, a.z[o], a.U[o]);
      float x = d0[v * NP + t];
      x = fmaf(dq[(0 * N2 + f0) * 5 + v], sdgL[i], x);
      x = fmaf(dq[(1 * N2 + f0) * 5 + v], sdgR[i], x);
      float y = d1[v * NP + t];
      y = fmaf(dq[(2 * N2 + f1) * 5 + v], sdgL[j], y);
      y = fmaf(dq[(3 * N2 + f1) * 5 + v], sdgR[j], y);
      float zz = d2[v * NP + t];
      zz = fmaf(dq[(4 * N2 + f2) * 5 + v], sdgL[k], zz);
      zz = fmaf(dq[(5 * N2 + f2) * 5 + v], sdgR[k], zz);
      g[0][v] = fma(eps, (double)(s[0] * x), a.lg[cb + (0 * 5 + v) * NP]);
      g[1][v] = fma(eps, (double)(s[1] * y), a.lg[cb + (1 * 5 + v) * NP]);
      g[2][v] = fma(eps, (double)(s[2] * zz), a.lg[cb + (2 * 5 + v) * NP]);
    }
    double fv[3][5];
    visc3(q, g, a.gam, a.mu, a.kappa, 7, fv);
    float* dst[3] = {d0, d1, d2};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double fi[5];
      (void)flux3(q, d, a.gam, fi);
      // each thread reads and overwrites only its own point
#pragma unroll
      for (int v = 0; v < 5; ++v)
        dst[d][v * NP + t] = (float)(((fi[v] - fv[d][v]) - a.lf[cb + (d * 5 + v) * NP]) * ieps);
    }
  }
  __syncthreads();
  if (!active) return;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const float* F = d0 + v * NP;
    const float* G = d1 + v * NP;
    const float* H = d2 + v * NP;
    float dF = sdgL[i] * fn[(0 * N2 + f0) * 5 + v];
    dF = fmaf(sdgR[i], fn[(1 * N2 + f0) * 5 + v], dF);
    float dG = sdgL[j] * fn[(2 * N2 + f1) * 5 + v];
    dG = fmaf(sdgR[j], fn[(3 * N2 + f1) * 5 + v], dG);
    float dH = sdgL[k] * fn[(4 * N2 + f2) * 5 + v];
    dH = fmaf(sdgR[k], fn[(5 * N2 + f2) * 5 + v], dH);
#pragma unroll
    for (int l = 0; l < N; ++l) {
      dF = fmaf(sDt[i][l], F[l + N * j + N2 * k], dF);
      dG = fmaf(sDt[j][l], G[i + N * l + N2 * k], dG);
      dH = fmaf(sDt[k][l], H[i + N * j + N2 * l], dH);
    }
    const float dR = -fmaf(s[0], dF, fmaf(s[1], dG, s[2] * dH));  // (R(U + eps z) - R(U)) / eps
    const long long o = e * NB + v * NP + t;
    const double Az = fma(a.shift, a.z[o], -(double)dR);
    a.out[o] = MODE == 2 ? a.b[o] - Az : Az;
  }
}

// Quadrature sums of S^d : S^d, p div v and rho |v|^2 / 2 (weights w_i w_j w_k
// |J_e|) for the dissipation rate; the velocity of each element is
// differentiated as its degree-p interpolant.  Grid-stride over element
// groups, deterministic two-stage reduction into out[0..2].
template <int P>
__global__ void __launch_bounds__(256) k3_dissipation(const F3Args a, Reduce red, double* out) {
  constexpr int N = P + 1, N2 = N * N, NP = N2 * N, E = F3Slots<P>::E;
  __shared__ double vel[E][3][NP];
  __shared__ double sD[N][N], sw[N], sh[32];
  if (threadIdx.x < N * N) sD[threadIdx.x / N][threadIdx.x % N] = a.tab.D[threadIdx.x / N][threadIdx.x % N];
  if (threadIdx.x < N) sw[threadIdx.x] = a.tab.w[threadIdx.x];
  const int el = threadIdx.x / NP, t = threadIdx.x % NP;
  const int i = t % N, j = (t / N) % N, k = t / N2;
  double acc[3] = {0.0, 0.0, 0.0};
  for (long long e0 = (long long)blockIdx.x * E; e0 < a.ne; e0 += (long long)gridDim.x * E) {
    const long long e = e0 + el;
    const bool active = el < E && e < a.ne;
    double q[5];
    __syncthreads();
    if (active) {
#pragma unroll
      for (int v = 0; v < 5; ++v) q[v] = a.U[e * 5 * NP + v * NP + t];
      const double ri = 1.0 / q[0];
      vel[el][0][t] = q[1] * ri;
      vel[el][1][t] = q[2] * ri;
      vel[el][2][t] = q[3] * ri;
    }
    __syncthreads();
    if (active) {
      int ix, iy, iz;
      coords(e, a, &ix, &iy, &iz);
      const double hx = a.hx[ix], hy = a.hy[iy], hz = a.hz[iz];
      const double s[3] = {2.0 / hx, 2.0 / hy, 2.0 / hz};
      double G[3][3];  // G[m][c] = d v_m / d x_c
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const double* x = vel[el][m];
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
#pragma unroll
        for (int l = 0; l < N; ++l) {
          a0 = fma(sD[i][l], x[l + N * j + N2 * k], a0);
          a1 = fma(sD[j][l], x[i + N * l + N2 * k], a1);
          a2 = fma(sD[k][l], x[i + N * j + N2 * l], a2);
        }
        G[m][0] = s[0] * a0;
        G[m][1] = s[1] * a1;
        G[m][2] = s[2] * a2;
      }
      const double div = G[0][0] + G[1][1] + G[2][2];
      double ss = 0.0;
#pragma unroll
      for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double Sd = 0.5 * (G[m][c] + G[c][m]) - (m == c ? div / 3.0 : 0.0);
          ss = fma(Sd, Sd, ss);
        }
      const double u = vel[el][0][t], v = vel[el][1][t], w = vel[el][2][t];
      const double ke2 = q[0] * (u * u + v * v + w * w);
      const double pr = (a.gam - 1.0) * (q[4] - 0.5 * ke2);
      const double wt = sw[i] * sw[j] * sw[k] * (0.125 * hx * hy * hz);
      acc[0] = fma(wt, ss, acc[0]);
      acc[1] = fma(wt, pr * div, acc[1]);
      acc[2] = fma(wt, 0.5 * ke2, acc[2]);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double bs = block_sum(acc[c], sh);
    if (threadIdx.x == 0) red.partials[(size_t)blockIdx.x * kMaxVec + c] = bs;
  }
  if (last_block(red.counter)) finish_sums(red, 3, out);
}

F3Args make_args3(fr_ctx* ctx) {
  F3Args a{};
  a.tb = ctx->tb;
  a.fb = ctx->fb;
  a.hx = ctx->hx;
  a.hy = ctx->hy;
  a.hz = ctx->hz;
  a.ne = ctx->ne;
  a.e0 = 0;
  a.nchunk = ctx->ne;
  a.r0f = nullptr;
  a.tbf = nullptr;
  a.r0_pass = 0;
  a.ltb = ctx->lin3_tb;
  a.lfb = ctx->lin3_fb;
  a.lg = ctx->lin3_g;
  a.lf = ctx->lin3_f;
  a.tbz = ctx->lin3_tbz;
  a.fbz = ctx->lin3_fbz;
  a.lgc = ctx->lin3_gc;
  a.write_gc = 0;
  a.nx = ctx->nx;
  a.ny = ctx->ny;
  a.nz = ctx->nz;
  a.gam = ctx->opts.gamma;
  a.mu = ctx->opts.mu;
  const double cp = ctx->opts.gamma / (ctx->opts.gamma - 1.0);  // R = 1
  a.kappa = ctx->opts.mu > 0.0 ? ctx->opts.mu * cp / ctx->opts.prandtl : 0.0;
  a.beps = ctx->opts.block_eps_rel;
  a.tab = ctx->tab;
  return a;
}

template <int P>
int f3_launch(fr_ctx* ctx, int mode, const F3Args& a, bool perturb_trace, cudaStream_t s, double wb,
              double wf) {
  using L = CellLayout<P>;
  constexpr int NP = L::NP, N2 = L::N2, E = F3Slots<P>::E, NB = 5 * NP;
  static bool attr = false;  // dynamic shared memory above 48 KB, set once per process
  if (!attr) {
    FRK_CUDA(ctx, cudaFuncSetAttribute(k3_cell<P, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES));
    FRK_CUDA(ctx, cudaFuncSetAttribute(k3_cell<P, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES));
    FRK_CUDA(ctx, cudaFuncSetAttribute(k3_cell<P, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES));
    FRK_CUDA(ctx, cudaFuncSetAttribute(k3_cell<P, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES));
    attr = true;
  }
  const unsigned gt = (unsigned)((ctx->ne + E - 1) / E);
  const int fam = mode == 3 ? FR_KF_FACTOR : (mode == 0 ? FR_KF_RESIDUAL : FR_KF_JV);
  if ((mode == 1 || mode == 2) && ctx->opts.jv_precision == 1) {
    // A z with FP32 linear parts: FP32 traces of z, face differences, cell
    using LZ = CellLayout<P, float>;
    static bool attrz = false;
    if (!attrz) {
      FRK_CUDA(ctx, cudaFuncSetAttribute(k3z_cell<P, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LZ::BYTES));
      FRK_CUDA(ctx, cudaFuncSetAttribute(k3z_cell<P, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LZ::BYTES));
      attrz = true;
    }
    if (!a.ltb || !a.tbz || !a.lgc) return set_error(ctx, FR_ERR_UNSUPPORTED, "jv_precision = 1 needs its caches (set at creation)");
    ProfScope ps_(ctx, fam, s, wb, wf);  // one timed record for the three kernels
    k3z_trace<P><<<gt, E * NP, 0, s>>>(a);
    FRK_LAUNCHED(ctx);
    count_launch();
    const long long nf = ctx->ne * 3 * N2;
    k3z_face<P><<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(a);
    FRK_LAUNCHED(ctx);
    count_launch();
    if (mode == 1) k3z_cell<P, 1><<<gt, E * NP, LZ::BYTES, s>>>(a);
    else k3z_cell<P, 2><<<gt, E * NP, LZ::BYTES, s>>>(a);
    FRK_LAUNCHED(ctx);
    return FR_OK;
  }
  {
    ProfScope ps_(ctx, fam, s, wb, wf);  // one timed record for the three kernels
    if (perturb_trace) k3_trace<P, true><<<gt, E * NP, 0, s>>>(a);
    else k3_trace<P, false><<<gt, E * NP, 0, s>>>(a);
    FRK_LAUNCHED(ctx);
    count_launch();  // the scope counted the trace kernel
    if (mode == 3) {
      const long long g3 = (a.nchunk * NB + E - 1) / E;
      k3_cell<P, 3><<<(unsigned)g3, E * NP, L::BYTES, s>>>(a);
    } else {
      const long long nf = ctx->ne * 3 * N2;
      k3_face<P><<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(a);
      FRK_LAUNCHED(ctx);
      count_launch();
      if (mode == 0) k3_cell<P, 0><<<gt, E * NP, L::BYTES, s>>>(a);
      else if (mode == 1) k3_cell<P, 1><<<gt, E * NP, L::BYTES, s>>>(a);
      else k3_cell<P, 2><<<gt, E * NP, L::BYTES, s>>>(a);
    }
  }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

int f3_dispatch(fr_ctx* ctx, int mode, const F3Args& a, bool perturb_trace, cudaStream_t s, double wb,
                double wf) {
  switch (ctx->p) {
    case 1: return f3_launch<1>(ctx, mode, a, perturb_trace, s, wb, wf);
    case 2: return f3_launch<2>(ctx, mode, a, perturb_trace, s, wb, wf);
    case 3: return f3_launch<3>(ctx, mode, a, perturb_trace, s, wb, wf);
    case 4: return f3_launch<4>(ctx, mode, a, perturb_trace, s, wb, wf);
    default: return set_error(ctx, FR_ERR_UNSUPPORTED, "3D degree %d not compiled", ctx->p);
  }
}

template <int P>
int dissipation_launch(fr_ctx* ctx, const double* U, double* out, cudaStream_t s) {
  constexpr int NP = (P + 1) * (P + 1) * (P + 1), E = F3Slots<P>::E;
  F3Args a = make_args3(ctx);
  a.U = U;
  long long g = (ctx->ne + E - 1) / E;
  if (g > kRedBlocks) g = kRedBlocks;
  const int threads = (E * NP + 31) / 32 * 32;  // whole warps (the reductions shuffle)
  { ProfScope ps_(ctx, FR_KF_OTHER, s); k3_dissipation<P><<<(unsigned)g, threads, 0, s>>>(a, ctx->red, out); }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

}  // namespace

// Navier-Stokes residual per element in 3D, counted like the 2D one (a fused
// multiply-add = 2) from the method's steps, each once: the reference
// derivatives of the 5 variables along 3 directions (30 Np N); the face
// traces of (q, grad q) (6 N^2 faces points x 20 values x 2N); per face point,
// with each face shared by two elements (3 N^2 per element), averages and
// BR2 liftings (60), Rusanov (90), the viscous flux (90) and the total (5);
// per point the corrected gradient (75), the inviscid fluxes (45), the
// viscous fluxes (120), their difference (15), the corrected divergence
// (30 (N+2)) and the scaling (5).
double ns3d_residual_flops_per_element(int p) {
  const double N = p + 1, N2 = N * N, Np = N2 * N;
  return 30 * Np * N + 240 * N2 * N + 3 * N2 * (60 + 90 + 90 + 5) +
         Np * (75 + 45 + 120 + 15 + 30 * (N + 2) + 5);
}

int launch_f3_residual(fr_ctx* ctx, int mode, const double* U, const double* z, const double* R0,
                       const double* b, double* out, double shift, const double* eps2,
                       const int* done, cudaStream_t s) {
  F3Args a = make_args3(ctx);
  a.U = U;
  a.z = z;
  a.R0 = R0;
  a.b = b;
  a.out = out;
  a.eps2 = eps2;
  a.done = done;
  a.shift = shift;
  // inside a GMRES cycle all kernels return at once once the cycle is done
  const double nd = (double)ctx->ndof;
  const bool in_cycle = done != nullptr;
  const double wb = in_cycle ? 0.0 : (mode == 0 ? 16.0 : (mode == 1 ? 32.0 : 40.0)) * nd;
  const double wf = in_cycle ? 0.0 : ns3d_residual_flops_per_element(ctx->p) * (double)ctx->ne + (mode == 0 ? 0.0 : 6.0 * nd);
  return f3_dispatch(ctx, mode, a, mode != 0, s, wb, wf);
}

namespace {
__global__ void k_to_f32(const double* __restrict__ x, float* __restrict__ y, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

// element-Jacobi columns of the elements a.e0 .. a.e0 + a.nchunk - 1 in the
// arithmetic T; the trace buffer already holds the unperturbed traces
template <int P, typename T>
int f3_columns(fr_ctx* ctx, F3Args a, cudaStream_t s) {
  using L = CellLayout<P, T>;
  constexpr int NP = L::NP, E = F3Slots<P>::E, NB = 5 * NP;
  FRK_CUDA(ctx, cudaFuncSetAttribute(k3_cell<P, 3, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES));
  // one element residual per column: the own six faces' common data, counted
  // like the residual with every face of the element
  const double per = ns3d_residual_flops_per_element(P) + 3.0 * L::N2 * 245.0;
  if (sizeof(T) == 4) {
    // FP32: the element-local R(U) of each element by the same arithmetic first
    a.r0f = ctx->r0f;
    a.r0_pass = 1;
    { ProfScope ps_(ctx, FR_KF_FACTOR, s, 0.0, per * (double)a.nchunk);
      k3_cell<P, 3, T><<<(unsigned)((a.nchunk + E - 1) / E), E * NP, L::BYTES, s>>>(a); }
    FRK_LAUNCHED(ctx);
    a.r0_pass = 0;
  }
  { ProfScope ps_(ctx, FR_KF_FACTOR, s, 0.0, per * NB * (double)a.nchunk);
    k3_cell<P, 3, T><<<(unsigned)((a.nchunk * NB + E - 1) / E), E * NP, L::BYTES, s>>>(a); }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

template <int P>
int f3_columns_p(fr_ctx* ctx, const F3Args& a, cudaStream_t s) {
  return ctx->opts.block_columns == 1 ? f3_columns<P, float>(ctx, a, s) : f3_columns<P, double>(ctx, a, s);
}
}  // namespace

namespace {
// the caches of the FP32-linear-parts A z at U: traces and face data of U in
// their own buffers, then the corrected gradient and total fluxes at the points
template <int P>
int f3_linearize(fr_ctx* ctx, const double* U, cudaStream_t s) {
  using L = CellLayout<P>;
  constexpr int NP = L::NP, N2 = L::N2, E = F3Slots<P>::E;
  F3Args a = make_args3(ctx);
  a.U = U;
  a.tb = ctx->lin3_tb;
  a.fb = ctx->lin3_fb;
  a.write_gc = 1;
  FRK_CUDA(ctx, cudaFuncSetAttribute(k3_cell<P, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES));
  const unsigned gt = (unsigned)((ctx->ne + E - 1) / E);
  {
    ProfScope ps_(ctx, FR_KF_OTHER, s);
    k3_trace<P, false><<<gt, E * NP, 0, s>>>(a);
    FRK_LAUNCHED(ctx);
    count_launch();
    const long long nf = ctx->ne * 3 * N2;
    k3_face<P><<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(a);
    FRK_LAUNCHED(ctx);
    count_launch();
    k3_cell<P, 4><<<gt, E * NP, L::BYTES, s>>>(a);
  }
  FRK_LAUNCHED(ctx);
  return FR_OK;
}
}  // namespace

int launch_f3_linearize(fr_ctx* ctx, const double* U, cudaStream_t s) {
  if (ctx->opts.jv_precision != 1) return FR_OK;
  switch (ctx->p) {
    case 1: return f3_linearize<1>(ctx, U, s);
    case 2: return f3_linearize<2>(ctx, U, s);
    case 3: return f3_linearize<3>(ctx, U, s);
    case 4: return f3_linearize<4>(ctx, U, s);
    default: return set_error(ctx, FR_ERR_UNSUPPORTED, "3D degree %d not compiled", ctx->p);
  }
}

int launch_f3_factor(fr_ctx* ctx, const double* U, double shift, cudaStream_t s) {
  if (ctx->p > 3 || !ctx->mst || ctx->blk_chunk < 1)
    return set_error(ctx, FR_ERR_UNSUPPORTED, "3D element blocks are built for degrees 1 to 3");
  // R0 of the element-local residuals = R(U); it leaves the unperturbed
  // traces in the trace buffer, which the columns read as the frozen
  // neighbour traces
  F3Args a = make_args3(ctx);
  a.U = U;
  a.out = ctx->rloc;
  FRK_TRY(f3_dispatch(ctx, 0, a, false, s, 0.0, 0.0));
  a.R0 = ctx->rloc;
  a.out = ctx->mst;
  a.shift = shift;
  if (ctx->opts.block_columns == 1) {
    if (!ctx->r0f || !ctx->tbf)
      return set_error(ctx, FR_ERR_UNSUPPORTED, "FP32 block columns need block_columns = 1 at creation");
    a.beps = fmax(ctx->opts.block_eps_rel, 1.0 / 4096.0);  // ~ sqrt of FP32's unit roundoff
    // the frozen neighbour traces, once in FP32
    const long long nt = ctx->ne * 6 * (long long)(ctx->n1 * ctx->n1) * 20;
    { ProfScope ps_(ctx, FR_KF_FACTOR, s, 12.0 * (double)nt, 0.0);
      k_to_f32<<<(unsigned)(nt / 256 < 4096 ? (nt + 255) / 256 : 4096), 256, 0, s>>>(ctx->tb, ctx->tbf, nt); }
    FRK_LAUNCHED(ctx);
    a.tbf = ctx->tbf;
  }
  for (long long e0 = 0; e0 < ctx->ne; e0 += ctx->blk_chunk) {
    a.e0 = e0;
    a.nchunk = ctx->ne - e0 < ctx->blk_chunk ? ctx->ne - e0 : ctx->blk_chunk;
    switch (ctx->p) {
      case 1: FRK_TRY(f3_columns_p<1>(ctx, a, s)); break;
      case 2: FRK_TRY(f3_columns_p<2>(ctx, a, s)); break;
      default: FRK_TRY(f3_columns_p<3>(ctx, a, s)); break;
    }
    FRK_TRY(launch_block_invert_range(ctx, ctx->mst, 0.0, e0, a.nchunk, s));
  }
  return FR_OK;
}

int launch_f3_dissipation(fr_ctx* ctx, const double* U, double* out, cudaStream_t s) {
  switch (ctx->p) {
    case 1: return dissipation_launch<1>(ctx, U, out, s);
    case 2: return dissipation_launch<2>(ctx, U, out, s);
    case 3: return dissipation_launch<3>(ctx, U, out, s);
    case 4: return dissipation_launch<4>(ctx, U, out, s);
    default: return set_error(ctx, FR_ERR_UNSUPPORTED, "3D degree %d not compiled", ctx->p);
  }
}

}  // namespace frk
