// fr_jv_noalloc: the finite-difference operator of fr_jv for callers that
// cannot allocate device memory.
//
// Its working memory (mesh edges and widths, the partial sums of the norm
// reductions, the FD step) lives in one file-scope static device array of
// fixed size, so a call allocates nothing.  Every GPU that loads the library
// holds that array until the process exits.  All calls share it and it keeps
// the last call's contents; calls that overlap on the GPU (two streams, two
// host threads) race on it.
#include "internal.cuh"

namespace frk {
namespace {

constexpr int kNoAllocMaxCells = 4096;  // largest nx and ny
// layout of the scratch array, in doubles
constexpr size_t kOffXE = 0;                                     // x edges (nx+1)
constexpr size_t kOffYE = kOffXE + kNoAllocMaxCells + 1;         // y edges (ny+1)
constexpr size_t kOffHX = kOffYE + kNoAllocMaxCells + 1;         // widths (nx)
constexpr size_t kOffHY = kOffHX + kNoAllocMaxCells;             // heights (ny)
constexpr size_t kOffPart = kOffHY + kNoAllocMaxCells;           // reduction partials
constexpr size_t kOffScal = kOffPart + (size_t)kVecBlocks * kMaxVec;
constexpr size_t kOffCount = kOffScal + S_COUNT;                 // completion counter
constexpr size_t kScratchDoubles = ((kOffCount + 1 + 31) / 32) * 32;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

__global__ void k_widths(double* scratch, int nx, int ny) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nx) scratch[kOffHX + i] = scratch[kOffXE + i + 1] - scratch[kOffXE + i];
  if (i < ny) scratch[kOffHY + i] = scratch[kOffYE + i + 1] - scratch[kOffYE + i];
}

// Device address of the scratch array on the current device, looked up on
// every call (the lookup allocates nothing, and a cached address would go
// stale after a device reset).  The first lookup on a device loads the
// library's device code there.
int scratch_for_device(double** out) {
  double* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    set_static_error("fr_jv_noalloc: cudaGetSymbolAddress failed");
    return FR_ERR_CUDA;
  }
  *out = p;
  return FR_OK;
}

// Stream-ordered body: clear the counter, bring the edges in, form the
// widths, then ||U||^2, ||z||^2 with the FD step, and the operator itself.
int run_jv(fr_ctx* ctx, const fr_mesh_desc* mesh, double* sp, const double* U, const double* R0,
           const double* z, double shift, double* y, cudaStream_t s) {
  FRK_CUDA(ctx, cudaMemsetAsync(ctx->red.counter, 0, sizeof(unsigned), s));
  FRK_CUDA(ctx, cudaMemcpyAsync(sp + kOffXE, mesh->x_edges, (ctx->nx + 1) * sizeof(double),
                                cudaMemcpyHostToDevice, s));
  FRK_CUDA(ctx, cudaMemcpyAsync(sp + kOffYE, mesh->y_edges, (ctx->ny + 1) * sizeof(double),
                                cudaMemcpyHostToDevice, s));
  const int mx = ctx->nx > ctx->ny ? ctx->nx : ctx->ny;
  count_launch();
  k_widths<<<(mx + 255) / 256, 256, 0, s>>>(sp, ctx->nx, ctx->ny);
  FRK_LAUNCHED(ctx);
  FRK_TRY(launch_sumsq(ctx, U, ctx->scal + S_NU2, s));
  FRK_TRY(launch_sumsq(ctx, z, ctx->scal + S_NZ2, s, true));
  return launch_residual(ctx, 1, U, z, R0, nullptr, y, shift, ctx->scal + S_EPS, nullptr, s);
}

}  // namespace
}  // namespace frk

using namespace frk;

extern "C" int fr_jv_noalloc(const fr_mesh_desc* mesh, int p, const fr_opts* opts, const double* U,
                             const double* R0, const double* z, double shift, double* y,
                             void* stream) {
  if (!mesh || !mesh->x_edges || !mesh->y_edges || !U || !R0 || !z || !y) {
    set_static_error("fr_jv_noalloc: null argument");
    return FR_ERR_INVALID_ARG;
  }
  if (mesh->nx < 2 || mesh->ny < 2 || mesh->nx > kNoAllocMaxCells || mesh->ny > kNoAllocMaxCells) {
    set_static_error("fr_jv_noalloc: nx and ny must lie in [2, 4096] (fixed scratch size)");
    return FR_ERR_INVALID_ARG;
  }
  if (p < 2 || p > 4) {
    set_static_error("fr_jv_noalloc: degree must be 2, 3 or 4");
    return FR_ERR_UNSUPPORTED;
  }
  if (y == U || y == R0 || y == z) {
    set_static_error("fr_jv_noalloc: y aliases an input");
    return FR_ERR_INVALID_ARG;
  }
  for (int i = 0; i < mesh->nx; ++i)
    if (!(mesh->x_edges[i + 1] > mesh->x_edges[i])) {
      set_static_error("fr_jv_noalloc: x edges must increase");
      return FR_ERR_INVALID_ARG;
    }
  for (int i = 0; i < mesh->ny; ++i)
    if (!(mesh->y_edges[i + 1] > mesh->y_edges[i])) {
      set_static_error("fr_jv_noalloc: y edges must increase");
      return FR_ERR_INVALID_ARG;
    }
  fr_opts o;
  fr_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.gamma > 1.0) || !(o.eps_rel > 0.0) || o.riemann < 0 || o.riemann > 1) {
    set_static_error("fr_jv_noalloc: bad gamma, eps_rel or riemann");
    return FR_ERR_INVALID_ARG;
  }
  // The product here is the periodic Euler one: a viscous or walled mesh, or
  // the FP32-linear-parts product (which needs per-context caches), would be
  // a different operator than fr_jv on a context made from the same inputs.
  if (mesh->wall_y || o.mu > 0.0 || o.jv_precision != 0) {
    set_static_error("fr_jv_noalloc: only the periodic Euler FP64 product (wall_y = 0, mu = 0, jv_precision = 0)");
    return FR_ERR_UNSUPPORTED;
  }
  // the edges are copied from the caller's (pageable, possibly temporary)
  // host arrays on the stream, which a graph capture could not replay
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(as_stream(stream), &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    set_static_error("fr_jv_noalloc: the stream is being captured (the call cannot be captured)");
    return FR_ERR_UNSUPPORTED;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_static_error("fr_jv_noalloc: cudaGetDevice failed");
    return FR_ERR_CUDA;
  }
  double* sp = nullptr;
  const int rc = scratch_for_device(&sp);
  if (rc != FR_OK) return rc;

  // A host-side view of the scratch with the fields the launchers use.
  fr_ctx c;
  c.device = dev;
  c.nx = mesh->nx;
  c.ny = mesh->ny;
  c.p = p;
  c.n1 = p + 1;
  c.np = c.n1 * c.n1;
  c.nb = 4 * c.np;
  c.ne = (long long)c.nx * c.ny;
  c.ndof = c.ne * c.nb;
  c.opts = o;
  build_tables(p, &c.tab);
  c.hx = sp + kOffHX;
  c.hy = sp + kOffHY;
  c.scal = sp + kOffScal;
  c.red.partials = sp + kOffPart;
  c.red.counter = reinterpret_cast<unsigned*>(sp + kOffCount);
  const int r = run_jv(&c, mesh, sp, U, R0, z, shift, y, as_stream(stream));
  if (r != FR_OK) set_static_error(c.err);
  return r;
}
