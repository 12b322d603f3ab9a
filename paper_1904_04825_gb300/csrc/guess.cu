// Stage-solve features for the learned initial guess, the guess itself, and
// capture of training pairs from the plain method's ROW stage solves.
//
// Features of element e for ROW stage i of step n with right-hand side b:
// [b_e / s, Y_i^{n-1}_e / s, Y_{i-1}^n_e / s] (the same stage's solution at
// the previous step and the previous stage's solution at this step, zero
// when absent) with s = ||b||_2 / sqrt(N).  The model predicts the change
// from the previous-step solution: x0 = Y_i^{n-1} + s * MLP(features), target
// (Y_i^n - Y_i^{n-1}) / s, so an imperfect model still starts GMRES near the
// previous-step guess.
#include "device.cuh"

struct fr_mlp;
extern "C" int fr_mlp_forward(fr_mlp* m, const float* X, int M, float* Y, int bf16, void* stream);

namespace frk {
namespace {

// X[r][0:nb) = b/s, [nb:2nb) = a1/s, [2nb:3nb) = a2/s (zero for a null a1 / a2)
// for the elements e = e0 + stride * r, r < count; T[r][0:nb) = (y - a1)/s when y != null.
__global__ void k_features(const double* __restrict__ b, const double* __restrict__ a1,
                           const double* __restrict__ a2, const double* __restrict__ y, int nb,
                           long long e0, long long stride, long long count, const double* nb2,
                           long long ndof, float* __restrict__ X, float* __restrict__ T) {
  const double s = sqrt(*nb2 / (double)ndof);
  const double is = s > 0.0 ? 1.0 / s : 1.0;
  const long long n = count * nb;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / nb;
    const int c = (int)(t % nb);
    const long long g = (e0 + stride * r) * nb + c;
    float* xr = X + r * 3 * nb;
    xr[c] = (float)(b[g] * is);
    xr[nb + c] = a1 ? (float)(a1[g] * is) : 0.f;
    xr[2 * nb + c] = a2 ? (float)(a2[g] * is) : 0.f;
    if (T) T[r * nb + c] = (float)((a1 ? y[g] - a1[g] : y[g]) * is);
  }
}

// x0 = a1 + s * out (a1 may be null)
__global__ void k_unscale(const float* __restrict__ out, const double* __restrict__ a1, const double* nb2,
                          long long ndof, double* __restrict__ x0) {
  const double s = sqrt(*nb2 / (double)ndof);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ndof; i += (long long)gridDim.x * blockDim.x)
    x0[i] = fma(s, (double)out[i], a1 ? a1[i] : 0.0);
}

unsigned grid_of(long long n) {
  long long g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

// Learned guess for one stage solve into x0 (device, ndof); a1 = the same
// stage's previous-step solution, a2 = the previous stage's solution (either
// may be null).
int stage_guess(fr_ctx* ctx, const double* b, const double* a1, const double* a2, double* x0,
                cudaStream_t s) {
  FRK_TRY(launch_sumsq(ctx, b, ctx->scal + S_GB2, s));
  count_launch();
  k_features<<<grid_of(ctx->ne * ctx->nb), 256, 0, s>>>(b, a1, a2, nullptr, ctx->nb, 0, 1, ctx->ne,
                                                      ctx->scal + S_GB2, ctx->ndof, ctx->gfeat, nullptr);
  FRK_LAUNCHED(ctx);
  const int rc = fr_mlp_forward(ctx->guess, ctx->gfeat, (int)ctx->ne, ctx->gout, 1, s);
  if (rc != FR_OK) return set_error(ctx, rc, "learned guess: MLP forward failed");
  count_launch();
  k_unscale<<<grid_of(ctx->ndof), 256, 0, s>>>(ctx->gout, a1, ctx->scal + S_GB2, ctx->ndof, x0);
  FRK_LAUNCHED(ctx);
  return FR_OK;
}

// Record (features, target) of the elements sampled from one finished stage.
int stage_capture(fr_ctx* ctx, const double* b, const double* a1, const double* a2, const double* y,
                  cudaStream_t s) {
  StageCapture& C = ctx->cap;
  if (!C.X || C.count >= C.max) return FR_OK;
  const long long stride = C.stride;
  const long long e0 = C.offset % stride;
  long long avail = (ctx->ne - e0 + stride - 1) / stride;
  if (avail > C.max - C.count) avail = C.max - C.count;
  if (avail <= 0) return FR_OK;
  FRK_TRY(launch_sumsq(ctx, b, ctx->scal + S_GB2, s));
  count_launch();
  k_features<<<grid_of(avail * ctx->nb), 256, 0, s>>>(b, a1, a2, y, ctx->nb, e0, stride, avail,
                                                    ctx->scal + S_GB2, ctx->ndof,
                                                    C.X + C.count * 3 * ctx->nb, C.T + C.count * ctx->nb);
  FRK_LAUNCHED(ctx);
  C.count += avail;
  C.offset += 1;
  return FR_OK;
}

}  // namespace frk

using namespace frk;

extern "C" int fr_attach_guess_model(fr_ctx* ctx, fr_mlp* model) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  ctx->guess = model;
  if (model && !ctx->gfeat) {
    FRK_CUDA(ctx, cudaMalloc(reinterpret_cast<void**>(&ctx->gfeat), (size_t)ctx->ne * 3 * ctx->nb * sizeof(float)));
    FRK_CUDA(ctx, cudaMalloc(reinterpret_cast<void**>(&ctx->gout), (size_t)ctx->ne * ctx->nb * sizeof(float)));
  }
  return FR_OK;
}

extern "C" int fr_set_stage_capture(fr_ctx* ctx, float* X, float* T, long long max_samples, int elem_stride) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  if ((X == nullptr) != (T == nullptr) || max_samples < 0 || elem_stride < 1)
    return set_error(ctx, FR_ERR_INVALID_ARG, "fr_set_stage_capture: bad arguments");
  ctx->cap.X = X;
  ctx->cap.T = T;
  ctx->cap.max = max_samples;
  ctx->cap.stride = elem_stride;
  ctx->cap.count = 0;
  ctx->cap.offset = 0;
  return FR_OK;
}

extern "C" long long fr_stage_capture_count(const fr_ctx* ctx) { return ctx ? ctx->cap.count : 0; }

extern "C" int fr_stage_features(fr_ctx* ctx, const double* b, const double* a1, const double* a2,
                                 float* X, void* stream) {
  if (!ctx || !b || !X) return FR_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  FRK_TRY(launch_sumsq(ctx, b, ctx->scal + S_GB2, s));
  count_launch();
  k_features<<<grid_of(ctx->ne * ctx->nb), 256, 0, s>>>(b, a1, a2, nullptr, ctx->nb, 0, 1, ctx->ne,
                                                      ctx->scal + S_GB2, ctx->ndof, X, nullptr);
  FRK_LAUNCHED(ctx);
  return FR_OK;
}
