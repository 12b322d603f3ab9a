// Stage-solve features for the learned initial guess, the guess itself, and
// capture of training pairs from the plain method's ROW stage solves.
//
// Features of element e for ROW stage i of step n with right-hand side b:
// [b_e / s, (b_e - b^{n-1}_e) / s, Y_i^{n-1}_e / s] (this stage's right-hand
// side and solution at the previous step, zero when absent) with
// s = ||b||_2 / sqrt(N).  The model predicts the change from the previous-step
// solution: x0 = Y_i^{n-1} + s * MLP(features), target (Y_i^n - Y_i^{n-1}) / s.
// The learned guess is kept only when ||b - A x0|| is below the residual of
// the previous-step guess (two extra FD products per stage).
#include "device.cuh"

struct fr_mlp;
extern "C" int fr_mlp_forward(fr_mlp* m, const float* X, int M, float* Y, int bf16, void* stream);

namespace frk {
namespace {

// X[r][0:nb) = b/s, [nb:2nb) = (b - bl)/s, [2nb:3nb) = yl/s (zero for a null
// bl / yl) for the elements e = e0 + stride * r, r < count; T[r][0:nb) =
// (y - yl)/s when y != null.
__global__ void k_features(const double* __restrict__ b, const double* __restrict__ bl,
                           const double* __restrict__ yl, const double* __restrict__ y, int nb,
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
    xr[nb + c] = bl ? (float)((b[g] - bl[g]) * is) : 0.f;
    xr[2 * nb + c] = yl ? (float)(yl[g] * is) : 0.f;
    if (T) T[r * nb + c] = (float)((yl ? y[g] - yl[g] : y[g]) * is);
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

int alloc_guess_buffers(fr_ctx* ctx);

// Learned guess for one stage solve into x0 (device, ndof) from (b, bl, yl)
// (bl / yl: previous-step right-hand side / solution of the stage).
int stage_guess(fr_ctx* ctx, const double* U, const double* R0, double shift, const double* b,
                const double* bl, const double* yl, double* x0, cudaStream_t s) {
  FRK_TRY(launch_sumsq(ctx, b, ctx->scal + S_GB2, s));
  count_launch();
  k_features<<<grid_of(ctx->ne * ctx->nb), 256, 0, s>>>(b, bl, yl, nullptr, ctx->nb, 0, 1, ctx->ne,
                                                      ctx->scal + S_GB2, ctx->ndof, ctx->gfeat, nullptr);
  FRK_LAUNCHED(ctx);
  const int rc = fr_mlp_forward(ctx->guess, ctx->gfeat, (int)ctx->ne, ctx->gout, 1, s);
  if (rc != FR_OK) return set_error(ctx, rc, "learned guess: MLP forward failed");
  count_launch();
  k_unscale<<<grid_of(ctx->ndof), 256, 0, s>>>(ctx->gout, yl, ctx->scal + S_GB2, ctx->ndof, x0);
  FRK_LAUNCHED(ctx);
  if (!yl) return FR_OK;
  // safeguard: residuals of the learned and of the previous-step guess
  double* r = ctx->buf[B_GUESS_R];
  FRK_TRY(launch_linearize(ctx, U, s));
  FRK_TRY(launch_sumsq(ctx, U, ctx->scal + S_NU2, s));
  FRK_TRY(launch_sumsq(ctx, x0, ctx->scal + S_NZ2, s, true));
  FRK_TRY(launch_residual(ctx, 2, U, x0, R0, b, r, shift, ctx->scal + S_EPS, nullptr, s));
  FRK_TRY(launch_sumsq(ctx, r, ctx->scal + S_GR1, s));
  FRK_TRY(launch_sumsq(ctx, yl, ctx->scal + S_NZ2, s, true));
  FRK_TRY(launch_residual(ctx, 2, U, yl, R0, b, r, shift, ctx->scal + S_EPS, nullptr, s));
  FRK_TRY(launch_sumsq(ctx, r, ctx->scal + S_GR2, s));
  FRK_CUDA(ctx, cudaMemcpyAsync(ctx->h_scal + 4, ctx->scal + S_GR1, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  FRK_CUDA(ctx, cudaStreamSynchronize(s));
  ctx->guess_used += ctx->h_scal[4] < ctx->h_scal[5] ? 1 : 0;
  ctx->guess_tried += 1;
  if (!(ctx->h_scal[4] < ctx->h_scal[5])) FRK_TRY(launch_copy(ctx, x0, yl, s));
  return FR_OK;
}

// Record (features, target) of the elements sampled from one finished stage.
int stage_capture(fr_ctx* ctx, const double* b, const double* bl, const double* yl, const double* y,
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
  k_features<<<grid_of(avail * ctx->nb), 256, 0, s>>>(b, bl, yl, y, ctx->nb, e0, stride, avail,
                                                    ctx->scal + S_GB2, ctx->ndof,
                                                    C.X + C.count * 3 * ctx->nb, C.T + C.count * ctx->nb);
  FRK_LAUNCHED(ctx);
  C.count += avail;
  C.offset += 1;
  return FR_OK;
}

}  // namespace frk

using namespace frk;

int frk::alloc_guess_buffers(fr_ctx* ctx) {
  if (!ctx->gfeat) {
    FRK_CUDA(ctx, cudaMalloc(reinterpret_cast<void**>(&ctx->gfeat), (size_t)ctx->ne * 3 * ctx->nb * sizeof(float)));
    FRK_CUDA(ctx, cudaMalloc(reinterpret_cast<void**>(&ctx->gout), (size_t)ctx->ne * ctx->nb * sizeof(float)));
  }
  for (double*& p : ctx->bhist)
    if (!p) {
      FRK_CUDA(ctx, cudaMalloc(reinterpret_cast<void**>(&p), (size_t)ctx->ndof * sizeof(double)));
      FRK_CUDA(ctx, cudaMemset(p, 0, (size_t)ctx->ndof * sizeof(double)));
    }
  return FR_OK;
}

extern "C" int fr_attach_guess_model(fr_ctx* ctx, fr_mlp* model) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  ctx->guess = model;
  if (model) FRK_TRY(alloc_guess_buffers(ctx));
  return FR_OK;
}

extern "C" int fr_reset_history(fr_ctx* ctx) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  ctx->hist_row = 0;
  return FR_OK;
}

extern "C" int fr_guess_stats(const fr_ctx* ctx, long long* tried, long long* used) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  if (tried) *tried = ctx->guess_tried;
  if (used) *used = ctx->guess_used;
  return FR_OK;
}

extern "C" int fr_set_stage_capture(fr_ctx* ctx, float* X, float* T, long long max_samples, int elem_stride) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  if ((X == nullptr) != (T == nullptr) || max_samples < 0 || elem_stride < 1)
    return set_error(ctx, FR_ERR_INVALID_ARG, "fr_set_stage_capture: bad arguments");
  if (X) FRK_TRY(alloc_guess_buffers(ctx));
  ctx->cap.X = X;
  ctx->cap.T = T;
  ctx->cap.max = max_samples;
  ctx->cap.stride = elem_stride;
  ctx->cap.count = 0;
  ctx->cap.offset = 0;
  return FR_OK;
}

extern "C" long long fr_stage_capture_count(const fr_ctx* ctx) { return ctx ? ctx->cap.count : 0; }

extern "C" int fr_stage_features(fr_ctx* ctx, const double* b, const double* bl, const double* yl,
                                 float* X, void* stream) {
  if (!ctx || !b || !X) return FR_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  FRK_TRY(launch_sumsq(ctx, b, ctx->scal + S_GB2, s));
  count_launch();
  k_features<<<grid_of(ctx->ne * ctx->nb), 256, 0, s>>>(b, bl, yl, nullptr, ctx->nb, 0, 1, ctx->ne,
                                                      ctx->scal + S_GB2, ctx->ndof, X, nullptr);
  FRK_LAUNCHED(ctx);
  return FR_OK;
}
