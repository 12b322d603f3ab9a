// C ABI entry points: context lifetime, argument checks, and the thin
// wrappers around the kernels of residual.cu, blocks.cu and krylov.cu.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <new>

#include "device.cuh"
#include "internal.cuh"

namespace frk {

int set_error(fr_ctx* ctx, int code, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

namespace {

void free_ctx(fr_ctx* c) {
  if (!c) return;
  cudaFree(c->hx);
  cudaFree(c->hy);
  cudaFree(c->hz);
  cudaFree(c->xo);
  cudaFree(c->yo);
  cudaFree(c->diss);
  cudaFree(c->blocks);
  cudaFree(c->tb);
  cudaFree(c->fb);
  cudaFree(c->mst);
  cudaFree(c->lin_fg);
  cudaFree(c->lin_fx);
  cudaFree(c->lin_fy);
  cudaFree(c->rloc);
  cudaFree(c->r0f);
  cudaFree(c->tbf);
  cudaFree(c->lin3_tb);
  cudaFree(c->lin3_fb);
  cudaFree(c->lin3_g);
  cudaFree(c->lin3_f);
  cudaFree(c->lin3_tbz);
  cudaFree(c->lin3_fbz);
  cudaFree(c->lin3_gc);
  cudaFree(c->gfeat);
  for (double* p : c->bhist) cudaFree(p);
  cudaFree(c->gout);
  cudaFree(c->V);
  cudaFree(c->z);
  for (double* b : c->buf) cudaFree(b);
  cudaFree(c->scal);
  cudaFree(c->red.partials);
  cudaFree(c->red.counter);
  cudaFree(c->gd.H);
  cudaFree(c->gd.cs);
  cudaFree(c->gd.sn);
  cudaFree(c->gd.g);
  cudaFree(c->gd.y);
  cudaFree(c->gd.h1);
  cudaFree(c->gd.h2);
  cudaFree(c->gd.invh);
  cudaFree(c->gd.done);
  cudaFree(c->kerr);
  cudaFree(c->gd.rflag);
  cudaFree(c->gd.k);
  cudaFree(c->gd.res);
  cudaFree(c->gd.target);
  for (cudaEvent_t e : c->chunk_ev)
    if (e) cudaEventDestroy(e);
  for (int f = 0; f < FR_KF_COUNT; ++f) {
    if (!c->prof.ev[f]) continue;
    for (int i = 0; i < 2 * Prof::kPairs; ++i) cudaEventDestroy(c->prof.ev[f][i]);
    delete[] c->prof.ev[f];
  }
  cudaFreeHost(c->h_stat);
  cudaFreeHost(c->h_scal);
  delete c;
}

template <typename T>
int dalloc(fr_ctx* c, T** p, size_t count) {
  FRK_CUDA(c, cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T)));
  FRK_CUDA(c, cudaMemset(*p, 0, count * sizeof(T)));
  return FR_OK;
}

int create(const fr_mesh_desc* mesh, int p, const fr_opts* o, fr_ctx* c) {
  c->opts = *o;
  c->p = p;
  c->n1 = p + 1;
  c->np = c->n1 * c->n1;
  c->nb = 4 * c->np;
  c->nx = mesh->nx;
  c->ny = mesh->ny;
  c->ne = (long long)mesh->nx * mesh->ny;
  c->ndof = c->ne * c->nb;
  c->blk_chunk = c->ne;
  FRK_CUDA(c, cudaGetDevice(&c->device));
  build_tables(p, &c->tab);
  double* hx = new double[mesh->nx];
  double* hy = new double[mesh->ny];
  for (int i = 0; i < mesh->nx; ++i) hx[i] = mesh->x_edges[i + 1] - mesh->x_edges[i];
  for (int i = 0; i < mesh->ny; ++i) hy[i] = mesh->y_edges[i + 1] - mesh->y_edges[i];
  int rc = dalloc(c, &c->hx, mesh->nx);
  if (rc == FR_OK) rc = dalloc(c, &c->hy, mesh->ny);
  if (rc == FR_OK && cudaMemcpy(c->hx, hx, mesh->nx * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    rc = set_error(c, FR_ERR_CUDA, "copying the mesh failed");
  if (rc == FR_OK && cudaMemcpy(c->hy, hy, mesh->ny * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    rc = set_error(c, FR_ERR_CUDA, "copying the mesh failed");
  delete[] hx;
  delete[] hy;
  FRK_TRY(rc);
  c->box[0] = mesh->x_edges[0];
  c->box[1] = mesh->x_edges[mesh->nx];
  c->box[2] = mesh->y_edges[0];
  c->box[3] = mesh->y_edges[mesh->ny];
  c->volume = (c->box[1] - c->box[0]) * (c->box[3] - c->box[2]);
  FRK_TRY(dalloc(c, &c->xo, mesh->nx));
  FRK_TRY(dalloc(c, &c->yo, mesh->ny));
  FRK_CUDA(c, cudaMemcpy(c->xo, mesh->x_edges, mesh->nx * sizeof(double), cudaMemcpyHostToDevice));
  FRK_CUDA(c, cudaMemcpy(c->yo, mesh->y_edges, mesh->ny * sizeof(double), cudaMemcpyHostToDevice));
  FRK_TRY(dalloc(c, &c->diss, 4));
  const size_t n = (size_t)c->ndof;
  const int m = o->m_max;
  FRK_TRY(dalloc(c, &c->blocks, (size_t)c->ne * c->nb * c->nb));
  c->wall_y = mesh->wall_y ? 1 : 0;
  c->viscous = (o->mu > 0.0 || c->wall_y) ? 1 : 0;
  if (c->viscous) {
    FRK_TRY(dalloc(c, &c->tb, (size_t)c->ne * 4 * c->n1 * 4 * 3));
    FRK_TRY(dalloc(c, &c->fb, (size_t)c->ne * 3 * c->n1 * 8));
    FRK_TRY(dalloc(c, &c->rloc, n));
  }
  FRK_TRY(dalloc(c, &c->mst, (size_t)c->ne * c->nb * c->nb));
  if (o->jv_precision == 1) {  // linearisation caches of the mixed-precision A z
    FRK_TRY(dalloc(c, &c->lin_fg, (size_t)c->ne * 8 * c->np));
    FRK_TRY(dalloc(c, &c->lin_fx, (size_t)c->ne * c->n1 * 12));
    FRK_TRY(dalloc(c, &c->lin_fy, (size_t)c->ne * c->n1 * 12));
  }
  FRK_TRY(dalloc(c, &c->V, (size_t)(m + 1) * n));
  FRK_TRY(dalloc(c, &c->z, n));
  for (double*& b : c->buf) FRK_TRY(dalloc(c, &b, n));
  FRK_TRY(dalloc(c, &c->scal, S_COUNT));
  FRK_TRY(dalloc(c, &c->red.partials, (size_t)kRedBlocks * kMaxVec));
  FRK_TRY(dalloc(c, &c->red.counter, 1));
  c->gd.ldh = m + 1;
  FRK_TRY(dalloc(c, &c->gd.H, (size_t)(m + 1) * m));
  FRK_TRY(dalloc(c, &c->gd.cs, m));
  FRK_TRY(dalloc(c, &c->gd.sn, m));
  FRK_TRY(dalloc(c, &c->gd.g, m + 1));
  FRK_TRY(dalloc(c, &c->gd.y, m));
  FRK_TRY(dalloc(c, &c->gd.h1, kMaxVec));
  FRK_TRY(dalloc(c, &c->gd.h2, kMaxVec));
  FRK_TRY(dalloc(c, &c->gd.invh, m + 1));
  FRK_TRY(dalloc(c, &c->gd.done, 1));
  FRK_TRY(dalloc(c, &c->gd.rflag, m));
  FRK_TRY(dalloc(c, &c->gd.k, 1));
  FRK_TRY(dalloc(c, &c->gd.res, 1));
  FRK_TRY(dalloc(c, &c->gd.target, 1));
  FRK_TRY(dalloc(c, &c->kerr, 1));
  FRK_CUDA(c, cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  FRK_CUDA(c, cudaMallocHost(reinterpret_cast<void**>(&c->h_stat), (4 + kMaxVec) * sizeof(int)));
  FRK_CUDA(c, cudaMallocHost(reinterpret_cast<void**>(&c->h_scal), 8 * sizeof(double)));
  for (cudaEvent_t& e : c->chunk_ev) FRK_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  FRK_CUDA(c, cudaDeviceSynchronize());
  return FR_OK;
}

// 3D context: periodic hexahedra, 5 variables, (p+1)^3 points per element.
// Element blocks and their staging exist only with the preconditioner on
// (p <= 3).  Degree 3 (320-row blocks): the blocks are stored in the block
// precision (FP32 or BF16) and the FP64 staging holds kStageChunk3
// elements at a time (3.4 GB).
int create3d(const fr_mesh3d_desc* mesh, int p, const fr_opts* o, fr_ctx* c) {
  c->opts = *o;
  c->dim3 = 1;
  c->viscous = o->mu > 0.0 ? 1 : 0;
  c->p = p;
  c->n1 = p + 1;
  c->np = c->n1 * c->n1 * c->n1;
  c->nb = 5 * c->np;
  c->nx = mesh->nx;
  c->ny = mesh->ny;
  c->nz = mesh->nz;
  c->ne = (long long)mesh->nx * mesh->ny * mesh->nz;
  c->ndof = c->ne * c->nb;
  c->volume = (mesh->x_edges[mesh->nx] - mesh->x_edges[0]) * (mesh->y_edges[mesh->ny] - mesh->y_edges[0]) *
              (mesh->z_edges[mesh->nz] - mesh->z_edges[0]);
  FRK_CUDA(c, cudaGetDevice(&c->device));
  build_tables(p, &c->tab);
  const double* edges[3] = {mesh->x_edges, mesh->y_edges, mesh->z_edges};
  const int counts[3] = {mesh->nx, mesh->ny, mesh->nz};
  double** dst[3] = {&c->hx, &c->hy, &c->hz};
  for (int d = 0; d < 3; ++d) {
    double* h = new double[counts[d]];
    for (int i = 0; i < counts[d]; ++i) h[i] = edges[d][i + 1] - edges[d][i];
    int rc = dalloc(c, dst[d], counts[d]);
    if (rc == FR_OK && cudaMemcpy(*dst[d], h, counts[d] * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
      rc = set_error(c, FR_ERR_CUDA, "copying the mesh failed");
    delete[] h;
    FRK_TRY(rc);
  }
  const size_t n = (size_t)c->ndof;
  const int m = o->m_max;
  const size_t n2 = (size_t)c->n1 * c->n1;
  FRK_TRY(dalloc(c, &c->tb, (size_t)c->ne * 6 * n2 * 20));
  FRK_TRY(dalloc(c, &c->fb, (size_t)c->ne * 3 * n2 * 10));
  if (o->jv_precision == 1) {  // caches of the A z with FP32 linear parts
    FRK_TRY(dalloc(c, &c->lin3_tb, (size_t)c->ne * 6 * n2 * 20));
    FRK_TRY(dalloc(c, &c->lin3_fb, (size_t)c->ne * 3 * n2 * 10));
    FRK_TRY(dalloc(c, &c->lin3_g, (size_t)c->ndof * 3));
    FRK_TRY(dalloc(c, &c->lin3_f, (size_t)c->ndof * 3));
    FRK_TRY(dalloc(c, &c->lin3_tbz, (size_t)c->ne * 6 * n2 * 20));
    FRK_TRY(dalloc(c, &c->lin3_fbz, (size_t)c->ne * 3 * n2 * 10));
    FRK_TRY(dalloc(c, &c->lin3_gc, (size_t)c->ne * 3 * n2 * 15));
  }
  if (o->precond) {
    const size_t nb2 = (size_t)c->nb * c->nb;
    if (p <= 2) {
      c->blk_chunk = c->ne;
      FRK_TRY(dalloc(c, &c->blocks, (size_t)c->ne * nb2));
    } else {
      c->blk_chunk = c->ne < kStageChunk3 ? c->ne : kStageChunk3;
      const size_t sbytes = o->block_precision == 1 ? 4 : 2;
      FRK_TRY(dalloc(c, &c->blocks, ((size_t)c->ne * nb2 * sbytes + 7) / 8));
    }
    FRK_TRY(dalloc(c, &c->mst, (size_t)c->blk_chunk * nb2));
    FRK_TRY(dalloc(c, &c->rloc, n));
    if (o->block_columns == 1) {
      FRK_TRY(dalloc(c, &c->r0f, (size_t)c->blk_chunk * c->nb));
      FRK_TRY(dalloc(c, &c->tbf, (size_t)c->ne * 6 * n2 * 20));
    }
  }
  FRK_TRY(dalloc(c, &c->diss, 4));
  FRK_TRY(dalloc(c, &c->V, (size_t)(m + 1) * n));
  FRK_TRY(dalloc(c, &c->z, n));
  for (double*& b : c->buf) FRK_TRY(dalloc(c, &b, n));
  FRK_TRY(dalloc(c, &c->scal, S_COUNT));
  FRK_TRY(dalloc(c, &c->red.partials, (size_t)kRedBlocks * kMaxVec));
  FRK_TRY(dalloc(c, &c->red.counter, 1));
  c->gd.ldh = m + 1;
  FRK_TRY(dalloc(c, &c->gd.H, (size_t)(m + 1) * m));
  FRK_TRY(dalloc(c, &c->gd.cs, m));
  FRK_TRY(dalloc(c, &c->gd.sn, m));
  FRK_TRY(dalloc(c, &c->gd.g, m + 1));
  FRK_TRY(dalloc(c, &c->gd.y, m));
  FRK_TRY(dalloc(c, &c->gd.h1, kMaxVec));
  FRK_TRY(dalloc(c, &c->gd.h2, kMaxVec));
  FRK_TRY(dalloc(c, &c->gd.invh, m + 1));
  FRK_TRY(dalloc(c, &c->gd.done, 1));
  FRK_TRY(dalloc(c, &c->gd.rflag, m));
  FRK_TRY(dalloc(c, &c->gd.k, 1));
  FRK_TRY(dalloc(c, &c->gd.res, 1));
  FRK_TRY(dalloc(c, &c->gd.target, 1));
  FRK_TRY(dalloc(c, &c->kerr, 1));
  FRK_CUDA(c, cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  FRK_CUDA(c, cudaMallocHost(reinterpret_cast<void**>(&c->h_stat), (4 + kMaxVec) * sizeof(int)));
  FRK_CUDA(c, cudaMallocHost(reinterpret_cast<void**>(&c->h_scal), 8 * sizeof(double)));
  for (cudaEvent_t& e : c->chunk_ev) FRK_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  FRK_CUDA(c, cudaDeviceSynchronize());
  return FR_OK;
}

std::atomic<long long> g_launches{0};

int check_vec(fr_ctx* ctx, const void* p, const char* name) {
  if (!p) return set_error(ctx, FR_ERR_INVALID_ARG, "%s is NULL", name);
  return FR_OK;
}

char g_static_err[512] = "invalid context";

// harvest the recorded event pairs of one family into ms / n
void prof_harvest(fr_ctx* c, int f) {
  Prof& P = c->prof;
  for (int i = 0; i < P.used[f]; ++i) {
    float t = 0.f;
    if (cudaEventSynchronize(P.ev[f][2 * i + 1]) == cudaSuccess &&
        cudaEventElapsedTime(&t, P.ev[f][2 * i], P.ev[f][2 * i + 1]) == cudaSuccess) {
      P.ms[f] += t;
      P.n[f] += 1;
    }
  }
  P.used[f] = 0;
}

}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_static_error(const char* msg) {
  std::strncpy(g_static_err, msg, sizeof(g_static_err) - 1);
  g_static_err[sizeof(g_static_err) - 1] = 0;
}

void prof_begin(fr_ctx* c, int f, cudaStream_t s) {
  count_launch();
  Prof& P = c->prof;
  if (!(P.mask & (1u << f))) return;
  if (P.used[f] == Prof::kPairs) prof_harvest(c, f);
  cudaEventRecord(P.ev[f][2 * P.used[f]], s);
}

void prof_work(fr_ctx* c, int f, double bytes, double flops) {
  Prof& P = c->prof;
  if (!(P.mask & (1u << f))) return;
  P.bytes[f] += bytes;
  P.flops[f] += flops;
}

// FR residual, per element (N = p+1, Np = N^2), counted from the method's
// steps: pointwise fluxes 22 flops per point; face traces of the solution
// 4 faces x N points x 4 variables x N multiply-adds; one Rusanov flux per
// face point with each face shared by two elements (2N per element, 70 flops
// each); corrected divergence along x and y, 4 variables x Np points x
// (N + 2) multiply-adds each; the final scaling, 4 Np.
double residual_flops_per_element(int p) {
  const double N = p + 1, Np = N * N;
  return 22 * Np + 2 * 16 * N * N + 70 * 2 * N + 2 * 2 * 4 * Np * (N + 2) + 4 * Np;
}

// Navier-Stokes (BR2) residual per element, counted like the Euler one
// (a fused multiply-add = 2) from the method's steps, each once: the state
// and its reference derivatives (8Np + 16 Np N), the face traces of
// (q, q_x, q_y) (96 N^2 + 32 N); per face point, with each face shared by
// two elements (2N per element), averages and BR2 liftings (48), Rusanov
// (70), the viscous flux (50) and the total (4); per point the corrected
// gradient (56), the inviscid and viscous fluxes and their difference (80),
// the corrected divergence (16 (N+2) + 4) and the body force (4).
double ns_residual_flops_per_element(int p) {
  const double N = p + 1, Np = N * N;
  return 8 * Np + 16 * Np * N + 96 * N * N + 32 * N + 2 * N * (48 + 70 + 50 + 4) +
         Np * (56 + 80 + 16 * (N + 2) + 4 + 4);
}

double jv_flops_per_element(const fr_ctx* ctx) {
  if (ctx->dim3) return ns3d_residual_flops_per_element(ctx->p);
  return ctx->viscous ? ns_residual_flops_per_element(ctx->p) : residual_flops_per_element(ctx->p);
}

// Element block: nb = 4 Np columns, each a local FD column (one pointwise
// flux, four Rusanov fluxes, 2N x 4 entries of 3 multiply-adds) plus
// Gauss-Jordan inversion, 2 nb^3.
double factor_flops_per_element(int p) {
  const double N = p + 1, Np = N * N, nb = 4 * Np;
  return nb * (22 + 4 * 70 + 2 * N * 4 * 6) + 2 * nb * nb * nb;
}

void prof_end(fr_ctx* c, int f, cudaStream_t s) {
  Prof& P = c->prof;
  if (!(P.mask & (1u << f))) return;
  cudaEventRecord(P.ev[f][2 * P.used[f] + 1], s);
  P.used[f] += 1;
}

}  // namespace frk

using namespace frk;

extern "C" void fr_default_opts(fr_opts* o) {
  if (!o) return;
  o->gamma = 1.4;
  o->m_max = 30;
  o->eps_rel = 1e-7;
  o->eps_fixed = 0.0;
  o->block_eps_rel = 1e-7;
  o->precond = 1;
  o->gmres_m = 30;
  o->gmres_max_restarts = 20;
  o->tol_lin = 1e-8;
  o->reorth_eta = 1.0 / 64.0;
  o->block_precision = 0;
  o->mu = 0.0;
  o->prandtl = 0.72;
  o->body_force_x = 0.0;
  o->wall_temperature = 1.0;
  o->precond_refresh = 0;
  o->guess = 0;
  o->jv_precision = 0;
  o->riemann = 0;
  o->block_columns = 0;
}

extern "C" void fr_default_ptc_opts(fr_ptc_opts* o) {
  if (!o) return;
  o->tol_nl = 1e-6;
  o->tol_lin = 1e-1;
  o->dtau_init = 0.0;
  o->dtau_max = 1e20;
  o->max_iters = 200;
  o->max_rejections = 30;
  o->reject_above = 0.1;
}

extern "C" int fr_ctx_create(const fr_mesh_desc* mesh, int p, const fr_opts* opts, fr_ctx** out) {
  if (!out) return FR_ERR_INVALID_ARG;
  *out = nullptr;
  if (!mesh || !mesh->x_edges || !mesh->y_edges || mesh->nx < 2 || mesh->ny < 2)
    return FR_ERR_INVALID_ARG;
  if (p < 2 || p > 6) return FR_ERR_UNSUPPORTED;
  fr_opts o;
  fr_default_opts(&o);
  if (opts) o = *opts;
  if (o.m_max < 1 || o.m_max > kMaxVec - 1 || o.gmres_m < 1 || o.gmres_m > o.m_max ||
      o.gmres_max_restarts < 0 || !(o.gamma > 1.0) || !(o.eps_rel > 0.0) || !(o.block_eps_rel > 0.0) ||
      !(o.reorth_eta >= 0.0 && o.reorth_eta <= 1.0) || o.block_precision < 0 || o.block_precision > 2 ||
      !(o.mu >= 0.0) || (o.mu > 0.0 && !(o.prandtl > 0.0)) ||
      (mesh->wall_y && !(o.wall_temperature > 0.0)) || o.precond_refresh < 0 || o.precond_refresh > 2 ||
      o.guess < 0 || o.guess > 2 || o.jv_precision < 0 || o.jv_precision > 1 || o.riemann < 0 || o.riemann > 1)
    return FR_ERR_INVALID_ARG;
  if (o.riemann == 1 && (o.mu > 0.0 || mesh->wall_y)) return FR_ERR_UNSUPPORTED;  // Euler residual only
  if (o.block_columns < 0 || o.block_columns > 1) return FR_ERR_INVALID_ARG;
  if (o.block_columns == 1) return FR_ERR_UNSUPPORTED;  // FP32 columns: 3D contexts only
  if (o.jv_precision == 1 && (o.mu > 0.0 || mesh->wall_y)) return FR_ERR_UNSUPPORTED;  // Euler residual only
  // degrees 5 and 6: Euler residual only; p = 6 FP64 blocks (196 x 196) exceed shared memory
  if (p > 4 && (o.mu > 0.0 || mesh->wall_y)) return FR_ERR_UNSUPPORTED;
  if (p == 6 && o.precond && o.block_precision == 0) return FR_ERR_UNSUPPORTED;
  for (int i = 0; i < mesh->nx; ++i)
    if (!(mesh->x_edges[i + 1] > mesh->x_edges[i])) return FR_ERR_INVALID_ARG;
  for (int i = 0; i < mesh->ny; ++i)
    if (!(mesh->y_edges[i + 1] > mesh->y_edges[i])) return FR_ERR_INVALID_ARG;
  fr_ctx* c = new (std::nothrow) fr_ctx();
  if (!c) return FR_ERR_CUDA;
  const int rc = create(mesh, p, &o, c);
  if (rc != FR_OK) {
    free_ctx(c);
    return rc;
  }
  *out = c;
  return FR_OK;
}

extern "C" int fr_ctx_create_3d(const fr_mesh3d_desc* mesh, int p, const fr_opts* opts, fr_ctx** out) {
  if (!out) return FR_ERR_INVALID_ARG;
  *out = nullptr;
  if (!mesh || !mesh->x_edges || !mesh->y_edges || !mesh->z_edges || mesh->nx < 2 || mesh->ny < 2 ||
      mesh->nz < 2)
    return FR_ERR_INVALID_ARG;
  if (p < 1 || p > 4) return FR_ERR_UNSUPPORTED;
  fr_opts o;
  fr_default_opts(&o);
  if (opts) o = *opts;
  if (o.m_max < 1 || o.m_max > kMaxVec - 1 || o.gmres_m < 1 || o.gmres_m > o.m_max ||
      o.gmres_max_restarts < 0 || !(o.gamma > 1.0) || !(o.eps_rel > 0.0) || !(o.block_eps_rel > 0.0) ||
      !(o.reorth_eta >= 0.0 && o.reorth_eta <= 1.0) || o.block_precision < 0 || o.block_precision > 2 ||
      !(o.mu >= 0.0) || (o.mu > 0.0 && !(o.prandtl > 0.0)) || o.precond_refresh < 0 || o.precond_refresh > 2 ||
      o.guess < 0 || o.guess > 2 || o.jv_precision < 0 || o.jv_precision > 1 || o.riemann < 0 || o.riemann > 1)
    return FR_ERR_INVALID_ARG;
  // the 3D path: Rusanov flux, no body force; the FD operator in FP64 or with
  // FP32 linear parts; element blocks for p <= 3 (5 (p+1)^3 = 40, 135 or 320
  // rows; 320-row blocks in FP32 or BF16 only), no learned guess
  if (o.riemann != 0 || o.guess == 2 || o.body_force_x != 0.0) return FR_ERR_UNSUPPORTED;
  if (o.block_columns < 0 || o.block_columns > 1) return FR_ERR_INVALID_ARG;
  if (o.block_columns == 1 && (!o.precond || o.block_precision == 0)) return FR_ERR_UNSUPPORTED;
  if (o.precond && (p > 3 || (p == 3 && o.block_precision == 0))) return FR_ERR_UNSUPPORTED;
  for (int i = 0; i < mesh->nx; ++i)
    if (!(mesh->x_edges[i + 1] > mesh->x_edges[i])) return FR_ERR_INVALID_ARG;
  for (int i = 0; i < mesh->ny; ++i)
    if (!(mesh->y_edges[i + 1] > mesh->y_edges[i])) return FR_ERR_INVALID_ARG;
  for (int i = 0; i < mesh->nz; ++i)
    if (!(mesh->z_edges[i + 1] > mesh->z_edges[i])) return FR_ERR_INVALID_ARG;
  fr_ctx* c = new (std::nothrow) fr_ctx();
  if (!c) return FR_ERR_CUDA;
  const int rc = create3d(mesh, p, &o, c);
  if (rc != FR_OK) {
    free_ctx(c);
    return rc;
  }
  *out = c;
  return FR_OK;
}

extern "C" int fr_dissipation_rate(fr_ctx* ctx, const double* U, double rho0, double* out, void* stream) {
  if (!ctx || !out) return FR_ERR_INVALID_ARG;
  FRK_TRY(check_vec(ctx, U, "U"));
  if (!ctx->dim3) return set_error(ctx, FR_ERR_UNSUPPORTED, "fr_dissipation_rate: 3D contexts only");
  if (!(rho0 > 0.0)) return set_error(ctx, FR_ERR_INVALID_ARG, "fr_dissipation_rate: rho0 must be > 0");
  cudaStream_t s = as_stream(stream);
  FRK_TRY(launch_f3_dissipation(ctx, U, ctx->diss, s));
  FRK_CUDA(ctx, cudaMemcpyAsync(ctx->h_scal, ctx->diss, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  FRK_CUDA(ctx, cudaStreamSynchronize(s));
  const double V = ctx->volume;
  out[0] = 2.0 * ctx->opts.mu / rho0 * ctx->h_scal[0] / V;
  out[1] = -ctx->h_scal[1] / (rho0 * V);
  out[2] = ctx->h_scal[2] / (rho0 * V);
  return FR_OK;
}

extern "C" int fr_set_wait_test(fr_ctx* ctx, unsigned polls, int skip_first_copy) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  if (skip_first_copy < 0 || skip_first_copy > 1)
    return set_error(ctx, FR_ERR_INVALID_ARG, "fr_set_wait_test: skip_first_copy must be 0 or 1");
  ctx->wait_polls = polls ? polls : kWaitPolls;
  ctx->test_skip_copy = skip_first_copy;
  return FR_OK;
}

extern "C" int fr_set_block_chunk(fr_ctx* ctx, long long n) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  const long long cap = ctx->dim3 && ctx->p == 3 ? (ctx->ne < kStageChunk3 ? ctx->ne : kStageChunk3) : ctx->ne;
  if (!ctx->mst || n < 1 || n > cap)
    return set_error(ctx, FR_ERR_INVALID_ARG, "fr_set_block_chunk: n must be in [1, %lld]", cap);
  ctx->blk_chunk = n;
  return FR_OK;
}

extern "C" void fr_default_vortex(fr_vortex* v) {
  if (!v) return;
  v->alpha = 5.0;
  v->phi = 0.5;
  v->mach = 0.5;
  v->rho_inf = 1.0;
  v->u_inf = 1.0;
  v->v_inf = 1.0;
  v->x0 = 0.0;
  v->y0 = 0.0;
}

extern "C" int fr_vortex_error(fr_ctx* ctx, const double* U, const fr_vortex* vortex, double t, double* err,
                               void* stream) {
  if (!ctx || !err) return FR_ERR_INVALID_ARG;
  FRK_TRY(check_vec(ctx, U, "U"));
  if (!vortex) return set_error(ctx, FR_ERR_INVALID_ARG, "fr_vortex_error: vortex is NULL");
  if (ctx->dim3 || ctx->viscous)
    return set_error(ctx, FR_ERR_UNSUPPORTED, "fr_vortex_error: 2D Euler contexts only");
  if (!(vortex->phi > 0.0) || !(vortex->mach > 0.0) || !(vortex->rho_inf > 0.0) || !std::isfinite(vortex->alpha) ||
      !std::isfinite(vortex->u_inf) || !std::isfinite(vortex->v_inf) || !std::isfinite(vortex->x0) ||
      !std::isfinite(vortex->y0) || !std::isfinite(t) ||
      !(vortex->u_inf * vortex->u_inf + vortex->v_inf * vortex->v_inf > 0.0))
    return set_error(ctx, FR_ERR_INVALID_ARG,
                     "fr_vortex_error: phi, mach, rho_inf and the free-stream speed must be > 0, all finite");
  cudaStream_t s = as_stream(stream);
  FRK_TRY(launch_vortex_error(ctx, U, vortex, t, ctx->diss, s));
  FRK_CUDA(ctx, cudaMemcpyAsync(ctx->h_scal, ctx->diss, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  FRK_CUDA(ctx, cudaStreamSynchronize(s));
  for (int k = 0; k < 4; ++k) err[k] = std::sqrt(ctx->h_scal[k] / ctx->volume);
  return FR_OK;
}

extern "C" int fr_ctx_destroy(fr_ctx* ctx) {
  free_ctx(ctx);
  return FR_OK;
}

extern "C" const char* fr_last_error(const fr_ctx* ctx) { return ctx ? ctx->err : g_static_err; }

extern "C" long long fr_ndof(const fr_ctx* ctx) { return ctx ? ctx->ndof : 0; }

extern "C" int fr_residual(fr_ctx* ctx, const double* U, double* R, void* stream) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  FRK_TRY(check_vec(ctx, U, "U"));
  FRK_TRY(check_vec(ctx, R, "R"));
  if (U == R) return set_error(ctx, FR_ERR_INVALID_ARG, "fr_residual: U and R alias");
  return launch_residual(ctx, 0, U, nullptr, nullptr, nullptr, R, 0.0, nullptr, nullptr,
                         as_stream(stream));
}

extern "C" int fr_jv(fr_ctx* ctx, const double* U, const double* R0, const double* z, double shift,
                     double* y, void* stream) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  FRK_TRY(check_vec(ctx, U, "U"));
  FRK_TRY(check_vec(ctx, R0, "R0"));
  FRK_TRY(check_vec(ctx, z, "z"));
  FRK_TRY(check_vec(ctx, y, "y"));
  if (y == U || y == R0 || y == z) return set_error(ctx, FR_ERR_INVALID_ARG, "fr_jv: y aliases an input");
  cudaStream_t s = as_stream(stream);
  FRK_TRY(launch_linearize(ctx, U, s));
  FRK_TRY(launch_sumsq(ctx, U, ctx->scal + S_NU2, s));
  FRK_TRY(launch_sumsq(ctx, z, ctx->scal + S_NZ2, s, true));
  return launch_residual(ctx, 1, U, z, R0, nullptr, y, shift, ctx->scal + S_EPS, nullptr, s);
}

extern "C" int ejacobi_factor(fr_ctx* ctx, const double* U, const double* R0, double shift,
                              void* stream) {
  (void)R0;
  if (!ctx) return FR_ERR_INVALID_ARG;
  FRK_TRY(check_vec(ctx, U, "U"));
  if (!std::isfinite(shift)) return set_error(ctx, FR_ERR_INVALID_ARG, "shift is not finite");
  FRK_TRY(launch_block_factor(ctx, U, shift, as_stream(stream)));
  ctx->blocks_valid = 1;
  return FR_OK;
}

extern "C" int ejacobi_apply(fr_ctx* ctx, const double* r, double* z, void* stream) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  FRK_TRY(check_vec(ctx, r, "r"));
  FRK_TRY(check_vec(ctx, z, "z"));
  if (r == z) return set_error(ctx, FR_ERR_INVALID_ARG, "ejacobi_apply: r and z alias");
  if (!ctx->blocks_valid) return set_error(ctx, FR_ERR_INVALID_ARG, "ejacobi_apply before ejacobi_factor");
  const int saved = ctx->opts.precond;
  ctx->opts.precond = 1;
  const int rc = launch_block_apply(ctx, const_cast<double*>(r), nullptr, z, nullptr, nullptr,
                                    as_stream(stream));
  ctx->opts.precond = saved;
  return rc;
}

extern "C" int gmres_solve(fr_ctx* ctx, const double* U, const double* R0, double shift,
                           const double* b, double* x, int m, double rtol, int max_restarts,
                           fr_gmres_info* info, void* stream) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  FRK_TRY(check_vec(ctx, U, "U"));
  FRK_TRY(check_vec(ctx, R0, "R0"));
  FRK_TRY(check_vec(ctx, b, "b"));
  FRK_TRY(check_vec(ctx, x, "x"));
  if (m < 1 || m > ctx->opts.m_max) return set_error(ctx, FR_ERR_INVALID_ARG, "m = %d outside [1, %d]", m, ctx->opts.m_max);
  if (max_restarts < 0 || !(rtol >= 0.0)) return set_error(ctx, FR_ERR_INVALID_ARG, "bad rtol / max_restarts");
  if (x == b || x == U || x == R0) return set_error(ctx, FR_ERR_INVALID_ARG, "gmres_solve: x aliases an input");
  if (ctx->opts.precond && !ctx->blocks_valid)
    return set_error(ctx, FR_ERR_INVALID_ARG, "gmres_solve: call ejacobi_factor first (precond = 1)");
  fr_gmres_info loc{};
  const int rc = gmres_impl(ctx, U, R0, shift, b, x, m, rtol, max_restarts, false, &loc, as_stream(stream));
  if (info) *info = loc;
  return rc;
}

extern "C" long long fr_kernel_launches(void) { return frk::g_launches.load(); }

extern "C" int fr_profile_begin(fr_ctx* ctx, unsigned mask) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  Prof& P = ctx->prof;
  for (int f = 0; f < FR_KF_COUNT; ++f) {
    if (!(mask & (1u << f))) continue;
    if (!P.ev[f]) {
      P.ev[f] = new cudaEvent_t[2 * Prof::kPairs];
      for (int i = 0; i < 2 * Prof::kPairs; ++i) FRK_CUDA(ctx, cudaEventCreate(&P.ev[f][i]));
    }
    P.used[f] = 0;
    P.ms[f] = 0.0;
    P.n[f] = 0;
    P.skipped[f] = 0;
    P.bytes[f] = 0.0;
    P.flops[f] = 0.0;
  }
  P.mask = mask;
  return FR_OK;
}

extern "C" int fr_profile_end(fr_ctx* ctx, double* ms, long long* launches, double* bytes,
                              double* flops) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  Prof& P = ctx->prof;
  for (int f = 0; f < FR_KF_COUNT; ++f) {
    const bool on = (P.mask & (1u << f)) != 0;
    if (on) prof_harvest(ctx, f);
    if (ms) ms[f] = on ? P.ms[f] : 0.0;
    if (launches) launches[f] = on ? P.n[f] - P.skipped[f] : 0;
    if (bytes) bytes[f] = on ? P.bytes[f] : 0.0;
    if (flops) flops[f] = on ? P.flops[f] : 0.0;
  }
  P.mask = 0;
  return FR_OK;
}
