// Device helpers: Euler fluxes, Rusanov flux, deterministic reductions.
#pragma once

#include "internal.cuh"

namespace frk {

// Inviscid fluxes f (x) and g (y) of the 2D Euler equations (Sec. 2).
__device__ __forceinline__ void euler_fluxes(const double q[4], double gam, double f[4],
                                             double g[4]) {
  const double rinv = 1.0 / q[0];
  const double u = q[1] * rinv, v = q[2] * rinv;
  const double p = (gam - 1.0) * (q[3] - 0.5 * (q[1] * u + q[2] * v));
  f[0] = q[1];
  f[1] = fma(q[1], u, p);
  f[2] = q[2] * u;
  f[3] = u * (q[3] + p);
  g[0] = q[2];
  g[1] = q[1] * v;
  g[2] = fma(q[2], v, p);
  g[3] = v * (q[3] + p);
}

// Normal flux along +x (dir 0) or +y (dir 1), plus |u_n| + c.
__device__ __forceinline__ double normal_flux(const double q[4], int dir, double gam, double f[4]) {
  const double rinv = 1.0 / q[0];
  const double u = q[1] * rinv, v = q[2] * rinv;
  const double p = (gam - 1.0) * (q[3] - 0.5 * (q[1] * u + q[2] * v));
  const double un = dir == 0 ? u : v;
  f[0] = q[1 + dir];
  f[1] = q[1] * un + (dir == 0 ? p : 0.0);
  f[2] = q[2] * un + (dir == 1 ? p : 0.0);
  f[3] = un * (q[3] + p);
  return fabs(un) + sqrt(gam * p * rinv);
}

// Rusanov common flux f_n = (f(qm)+f(qp))/2 - lam/2 (qp - qm),
// lam = max(|u_n|+c) over both sides; qm is the side the +x/+y normal leaves.
__device__ __forceinline__ void rusanov(const double qm[4], const double qp[4], int dir, double gam,
                                        double out[4]) {
  double fm[4], fp[4];
  const double am = normal_flux(qm, dir, gam, fm);
  const double ap = normal_flux(qp, dir, gam, fp);
  const double lam = fmax(am, ap);
#pragma unroll
  for (int v = 0; v < 4; ++v) out[v] = 0.5 * (fm[v] + fp[v]) - 0.5 * lam * (qp[v] - qm[v]);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum in a fixed order; result valid in thread 0. `sh` holds 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) s += sh[i];
  }
  return s;
}

// Called by every thread of every block after thread 0 wrote its partials.
// Returns true in the last of the nblk blocks of the reduction to arrive
// (nblk < 0: the whole grid).
__device__ __forceinline__ bool last_block(unsigned* counter, int nblk = -1) {
  __shared__ bool am_last;
  const unsigned nb = nblk < 0 ? gridDim.x : (unsigned)nblk;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(counter, 1u);
    am_last = (t == nb - 1);
  }
  __syncthreads();
  return am_last;
}

// In the last block: out[i] = sum over blocks b (fixed order) of partials[b][i],
// i < nvec, over the nblk blocks of the reduction (nblk < 0: the whole grid).
// Each warp sums one value with its lanes striding over the blocks through
// four independent accumulators.  Resets the counter.
__device__ __forceinline__ void finish_sums(const Reduce& red, int nvec, double* out, int nblk = -1) {
  __threadfence();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int G = nblk < 0 ? (int)gridDim.x : nblk;
  for (int i = wid; i < nvec; i += nw) {
    const double* p = red.partials + i;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int b = lane;
    for (; b + 96 < G; b += 128) {
      s0 += __ldcg(p + (size_t)b * kMaxVec);
      s1 += __ldcg(p + (size_t)(b + 32) * kMaxVec);
      s2 += __ldcg(p + (size_t)(b + 64) * kMaxVec);
      s3 += __ldcg(p + (size_t)(b + 96) * kMaxVec);
    }
    for (; b < G; b += 32) s0 += __ldcg(p + (size_t)b * kMaxVec);
    double s = warp_sum((s0 + s1) + (s2 + s3));
    if (lane == 0) out[i] = s;
  }
  if (threadIdx.x == 0) *red.counter = 0u;
}

// Batched launches: the CTAs of all instances in one grid; instance k owns
// blocks [start[k], start[k+1]).  Returns k for block b (binary search).
__device__ __forceinline__ int batch_instance(const int* __restrict__ start, int ninst, int b) {
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// eps and 1/eps of the FD product from the finished ||z||^2 (one thread).
__device__ __forceinline__ void write_eps(const EpsArgs& ea, double nz2) {
  if (!ea.out) return;
  double eps = 0.0;
  if (nz2 > 0.0) eps = ea.eps_fixed > 0.0 ? ea.eps_fixed : ea.eps_rel * (1.0 + sqrt(*ea.nU2)) / sqrt(nz2);
  ea.out[0] = eps;
  ea.out[1] = eps > 0.0 ? 1.0 / eps : 0.0;
}

// Roe's approximate Riemann flux (no entropy fix) along +x (dir 0) or +y
// (dir 1): the mean of the two fluxes minus half the sum over the four waves
// |lambda_k| alpha_k r_k of the flux Jacobian at the Roe average
// (sqrt(rho)-weighted velocity and total enthalpy; waves u_n - a, entropy
// and shear at u_n, u_n + a).
__device__ __forceinline__ void roe(const double qm[4], const double qp[4], int dir, double gam,
                                    double out[4]) {
  double fm[4], fp[4];
  (void)normal_flux(qm, dir, gam, fm);
  (void)normal_flux(qp, dir, gam, fp);
  const double rim = 1.0 / qm[0], rip = 1.0 / qp[0];
  const double um = qm[1] * rim, vm = qm[2] * rim, up = qp[1] * rip, vp = qp[2] * rip;
  const double pm = (gam - 1.0) * (qm[3] - 0.5 * (qm[1] * um + qm[2] * vm));
  const double pp = (gam - 1.0) * (qp[3] - 0.5 * (qp[1] * up + qp[2] * vp));
  const double Hm = (qm[3] + pm) * rim, Hp = (qp[3] + pp) * rip;
  const double sm = sqrt(qm[0]), sp = sqrt(qp[0]);
  const double w = 1.0 / (sm + sp);
  const double u = (sm * um + sp * up) * w, v = (sm * vm + sp * vp) * w, H = (sm * Hm + sp * Hp) * w;
  const double rho = sm * sp;
  const double a2 = (gam - 1.0) * (H - 0.5 * (u * u + v * v));
  const double a = sqrt(a2), ia2 = 1.0 / a2;
  const double un = dir == 0 ? u : v;
  const double dun = dir == 0 ? up - um : vp - vm;
  const double dut = dir == 0 ? vp - vm : up - um;
  const double dr = qp[0] - qm[0], dp = pp - pm;
  const double al1 = 0.5 * (dp - rho * a * dun) * ia2;
  const double al2 = dr - dp * ia2;
  const double al3 = rho * dut;
  const double al4 = 0.5 * (dp + rho * a * dun) * ia2;
  const double l1 = fabs(un - a) * al1, l2 = fabs(un) * al2, l3 = fabs(un) * al3, l4 = fabs(un + a) * al4;
  const double k2 = 0.5 * (u * u + v * v);
  double d[4];
  d[0] = l1 + l2 + l4;
  if (dir == 0) {
    d[1] = l1 * (u - a) + l2 * u + l4 * (u + a);
    d[2] = (l1 + l2 + l4) * v + l3;
    d[3] = l1 * (H - u * a) + l2 * k2 + l3 * v + l4 * (H + u * a);
  } else {
    d[1] = (l1 + l2 + l4) * u + l3;
    d[2] = l1 * (v - a) + l2 * v + l4 * (v + a);
    d[3] = l1 * (H - v * a) + l2 * k2 + l3 * u + l4 * (H + v * a);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) out[k] = 0.5 * (fm[k] + fp[k]) - 0.5 * d[k];
}

// the common inviscid flux selected by fr_opts.riemann (0 Rusanov, 1 Roe)
__device__ __forceinline__ void riemann_flux(int kind, const double qm[4], const double qp[4], int dir,
                                             double gam, double out[4]) {
  if (kind == 1) roe(qm, qp, dir, gam, out);
  else rusanov(qm, qp, dir, gam, out);
}

// ---- asynchronous bulk copies (TMA engine) with mbarrier completion ----
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// makes initialised barriers visible to the async proxy
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// one arrival that also expects `bytes` of transactions in the current phase
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of parity `parity` to complete; gives up after `limit`
// polls (each poll may suspend the thread for a short system-defined time).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned limit) {
  for (unsigned it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// global -> shared bulk copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned), completing as transactions on `bar`
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
constexpr unsigned kWaitPolls = 1u << 22;  // bounded waits: far above any copy's latency

}  // namespace frk
