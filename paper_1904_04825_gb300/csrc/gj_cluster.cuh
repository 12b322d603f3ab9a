// Gauss-Jordan inversion of element blocks too large for one SM's shared
// memory (the element-Jacobi preconditioner of Sec. 4.5 for 3D degree 3:
// 5 (p+1)^3 = 320 rows, 400 KB in FP32), split over a cluster of two CTAs.
//
// CTA r of the cluster holds columns [r NB/2, (r+1) NB/2) of the FP32 matrix
// in its shared memory (row stride NB/2 + 1).  The pivots are taken in
// panels of BW = 16 columns; the CTA that holds a panel factorises it:
//  * for each column c of the panel, the pivot row is the unused row of
//    largest |M[r][c]| (rows stay in place, pr[c] = r is recorded), and the
//    elimination is applied to the panel's columns (all rows); during the
//    panel each thread holds one row of it in registers, so a pivot costs
//    a warp-shuffle arg-max, two barriers and a broadcast of the pivot row;
//  * U = (panel columns after the panel) - (unit vectors of the pivot rows),
//    NB x BW, is written into the shared memory of both CTAs (distributed
//    shared memory), with the panel's pivot rows;
//  * after a cluster barrier every CTA applies the panel to its other
//    columns: x <- x + U x_P, x_P the pivot rows' entries of x before the
//    panel (a rank-BW update on the CUDA cores, FP32);
//  * a second cluster barrier lets the next panel's holder overwrite U.
// The result is the inverse with permuted rows and columns:
// inverse(a, b) = M[pr[a]][c] with pr[c] = b.
#pragma once

#include <cooperative_groups.h>

#include "device.cuh"

namespace frk {
namespace gjcl {

constexpr int CL = 2;         // CTAs per cluster
constexpr int BW = 16;        // panel width
constexpr int THREADS = 320;  // 10 warps

template <int NB>
struct Shape {
  static_assert(NB % (CL * 32) == 0, "each CTA's columns are whole warps of lanes");
  static constexpr int CW = NB / CL;         // columns per CTA
  static constexpr int LDM = CW + 1;         // row stride of M (conflict-free column reads)
  static constexpr int QN = CW / 32;         // columns per lane in the update
  static constexpr int RPW = NB / (THREADS / 32);  // rows per warp in the update
  static_assert(NB % (THREADS / 32) == 0, "rows split evenly over the warps");
  // bytes: M, U, pr (int), rows (int), srow (16-byte aligned), per-warp
  // pivot candidates (value, row), used (byte)
  static constexpr size_t OFF_U = (size_t)NB * LDM * 4;
  static constexpr size_t OFF_PR = OFF_U + (size_t)NB * BW * 4;
  static constexpr size_t OFF_ROWS = OFF_PR + (size_t)NB * 4;
  static constexpr size_t OFF_SROW = (OFF_ROWS + BW * 4 + 15) / 16 * 16;
  static constexpr size_t OFF_REDV = OFF_SROW + BW * 4;
  static constexpr size_t OFF_REDI = OFF_REDV + 32 * 4;
  static constexpr size_t OFF_USED = OFF_REDI + 32 * 4;
  static constexpr size_t BYTES = (OFF_USED + NB + 15) / 16 * 16;
  static_assert(NB == THREADS, "the panel factorisation keeps one row per thread");
};

// Invert element blocks b = 0 .. (gridDim.x / CL) - 1 of the FP64 staging
// mst (column-major per element: mst[b][c][row]) into blocks + (e0 + b) NB^2
// (column-major: Minv[k NB + i] = inverse(i, k)), adding dshift to the
// diagonal first.  Launched with THREADS threads and Shape<NB>::BYTES of
// dynamic shared memory per CTA, clusters of CL CTAs along x.
template <int NB, typename S, typename Store>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(THREADS)
    k_invert_cluster(const double* __restrict__ mst, S* __restrict__ blocks, long long e0, double dshift) {
  namespace cg = cooperative_groups;
  using Sh = Shape<NB>;
  constexpr int CW = Sh::CW, LDM = Sh::LDM, QN = Sh::QN, RPW = Sh::RPW;
  extern __shared__ __align__(16) unsigned char smem_cl[];
  float* M = reinterpret_cast<float*>(smem_cl);
  float* U = reinterpret_cast<float*>(smem_cl + Sh::OFF_U);
  int* pr = reinterpret_cast<int*>(smem_cl + Sh::OFF_PR);
  int* rows = reinterpret_cast<int*>(smem_cl + Sh::OFF_ROWS);
  float* srow = reinterpret_cast<float*>(smem_cl + Sh::OFF_SROW);
  float* red_v = reinterpret_cast<float*>(smem_cl + Sh::OFF_REDV);
  int* red_i = reinterpret_cast<int*>(smem_cl + Sh::OFF_REDI);
  unsigned char* used = smem_cl + Sh::OFF_USED;
  constexpr int NWARP = THREADS / 32;

  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long b = blockIdx.x / CL;
  const int col0 = rank * CW;
  const double* src = mst + b * (long long)NB * NB;
  for (int idx = tid; idx < CW * NB; idx += THREADS) {
    const int lc = idx / NB, i = idx - lc * NB;
    const double v = src[(long long)(col0 + lc) * NB + i];
    M[i * LDM + lc] = (float)(i == col0 + lc ? v + dshift : v);
  }
  for (int i = tid; i < NB; i += THREADS) used[i] = 0;
  float* peerU = cluster.map_shared_rank(U, rank ^ 1);
  int* peerRows = cluster.map_shared_rank(rows, rank ^ 1);
  cluster.sync();  // both CTAs' shared memory is set up before any remote write

  for (int c0 = 0; c0 < NB; c0 += BW) {
    const int owner = c0 / CW;
    const int lc0 = c0 - col0;
    if (rank == owner) {
      // ---- panel factorisation on the local columns lc0 .. lc0 + BW: thread
      // i keeps row i of the panel in registers ----
      const int i = tid;
      float pv[BW];
#pragma unroll
      for (int t = 0; t < BW; ++t) pv[t] = M[i * LDM + lc0 + t];
      bool usd = used[i] != 0;
#pragma unroll
      for (int k = 0; k < BW; ++k) {
        // pivot: the unused row of largest |M[r][c]| (NaN ranks above
        // everything), the lowest row among equals
        float best = usd ? -1.f : fabsf(pv[k]);
        if (best != best) best = __int_as_float(0x7f800000);
        int bi = usd ? NB : i;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float ob = __shfl_down_sync(0xffffffffu, best, o);
          const int oi = __shfl_down_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) {
          red_v[warp] = best;
          red_i[warp] = bi;
        }
        __syncthreads();
        best = red_v[0];
        bi = red_i[0];
#pragma unroll
        for (int w = 1; w < NWARP; ++w) {
          const float ob = red_v[w];
          const int oi = red_i[w];
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        const float c = pv[k];  // this row's entry in the pivot column
        if (i == bi) {
          const float ip = 1.f / c;
#pragma unroll
          for (int t = 0; t < BW; ++t) srow[t] = (t == k ? 1.f : pv[t]) * ip;
          rows[k] = bi;
          usd = true;
          used[i] = 1;
        }
        __syncthreads();
        const float4* s4 = reinterpret_cast<const float4*>(srow);
        float sr[BW];
#pragma unroll
        for (int t4 = 0; t4 < BW / 4; ++t4) {
          const float4 v = s4[t4];
          sr[4 * t4] = v.x;
          sr[4 * t4 + 1] = v.y;
          sr[4 * t4 + 2] = v.z;
          sr[4 * t4 + 3] = v.w;
        }
#pragma unroll
        for (int t = 0; t < BW; ++t) pv[t] = i == bi ? sr[t] : (t == k ? 0.f : pv[t]) - c * sr[t];
      }
      // ---- the panel back into M; U = panel - unit vectors of the pivot
      // rows, to both CTAs ----
      float4* u4 = reinterpret_cast<float4*>(U + i * BW);
      float4* p4 = reinterpret_cast<float4*>(peerU + i * BW);
#pragma unroll
      for (int t4 = 0; t4 < BW / 4; ++t4) {
        float u[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int t = 4 * t4 + q;
          M[i * LDM + lc0 + t] = pv[t];
          u[q] = pv[t] - (i == rows[t] ? 1.f : 0.f);
        }
        const float4 v = make_float4(u[0], u[1], u[2], u[3]);
        u4[t4] = v;
        p4[t4] = v;
      }
      if (tid < BW) peerRows[tid] = rows[tid];
    }
    cluster.sync();  // U and the pivot rows are visible in both CTAs
    if (tid < BW) {
      pr[c0 + tid] = rows[tid];
      used[rows[tid]] = 1;
    }
    // x_P for this lane's columns, read before any row changes
    float x[BW][QN];
    bool keep[QN];
#pragma unroll
    for (int q = 0; q < QN; ++q) {
      const int j = lane + 32 * q;
      keep[q] = !(rank == owner && j >= lc0 && j < lc0 + BW);
#pragma unroll
      for (int k = 0; k < BW; ++k) x[k][q] = M[rows[k] * LDM + j];
    }
    __syncthreads();
    // ---- M[:, j] += U x_P[:, j] for this CTA's columns outside the panel ----
    for (int i = warp * RPW; i < (warp + 1) * RPW; ++i) {
      const float4* ui = reinterpret_cast<const float4*>(U + i * BW);
      float u[BW];
#pragma unroll
      for (int k4 = 0; k4 < BW / 4; ++k4) {
        const float4 v = ui[k4];
        u[4 * k4] = v.x;
        u[4 * k4 + 1] = v.y;
        u[4 * k4 + 2] = v.z;
        u[4 * k4 + 3] = v.w;
      }
#pragma unroll
      for (int q = 0; q < QN; ++q) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < BW; ++k) acc = fmaf(u[k], x[k][q], acc);
        if (keep[q]) M[i * LDM + lane + 32 * q] += acc;
      }
    }
    cluster.sync();  // every CTA is done with U before the next panel overwrites it
  }
  // ---- store: inverse(ii, kk) = M[pr[ii]][c] for this CTA's columns c, kk = pr[c] ----
  S* out = blocks + (e0 + b) * (long long)NB * NB;
  for (int idx = tid; idx < CW * NB; idx += THREADS) {
    const int lc = idx / NB, ii = idx - lc * NB;
    out[(long long)pr[col0 + lc] * NB + ii] = Store::to(M[pr[ii] * LDM + lc]);
  }
}

}  // namespace gjcl
}  // namespace frk
