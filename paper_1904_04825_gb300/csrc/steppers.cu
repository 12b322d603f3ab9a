// Host control of the time integrators of Sec. 4 (ROW, ESDIRK with
// pseudo-transient continuation, BDF2).  Every vector operation is a kernel
// on the caller's stream; the host reads back only the scalars the method
// branches on (GMRES cycle status, ||F|| of each pseudo step).
#include <cmath>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <functional>
#include <new>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace frk {
namespace {

// ---- coefficient sets (the paper names them but prints none) --------------
// Rosenbrock sets in the form of Eq. Rosenbrock_General: omega (= gamma),
// a (stage arguments), c (stage right-hand sides), m (solution weights).
struct RowTab {
  int s = 0;
  double gamma = 0.0;
  double a[6][6] = {};
  double c[6][6] = {};
  double m[6] = {};
};

// Convert the Hairer-Wanner form (alpha, Gamma, b) to (a, c, m):
// a = alpha Gamma^-1, c = diag(1/gamma) - Gamma^-1, m = b Gamma^-1.
void from_alpha(int s, const double al[6][6], const double G[6][6], const double* b, RowTab* t) {
  double Gi[6][6] = {};
  // inverse of the lower-triangular Gamma by forward substitution
  for (int j = 0; j < s; ++j) {
    for (int i = 0; i < s; ++i) {
      double v = (i == j) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) v -= G[i][k] * Gi[k][j];
      Gi[i][j] = v / G[i][i];
    }
  }
  t->s = s;
  t->gamma = G[0][0];
  for (int i = 0; i < s; ++i) {
    for (int j = 0; j < s; ++j) {
      double v = 0.0;
      for (int k = 0; k < s; ++k) v += al[i][k] * Gi[k][j];
      t->a[i][j] = j < i ? v : 0.0;
      t->c[i][j] = j < i ? -Gi[i][j] : 0.0;
    }
  }
  for (int j = 0; j < s; ++j) {
    double v = 0.0;
    for (int i = 0; i < s; ++i) v += b[i] * Gi[i][j];
    t->m[j] = v;
  }
}

RowTab row_tableau(int order) {
  RowTab t;
  double al[6][6] = {}, G[6][6] = {}, b[6] = {};
  if (order == 2) {
    // 3 stages, order 2, stiffly accurate: W-order 2, stability function
    // matching exp(z) to third order (gamma: root of g^3 - 3g^2 + 3g/2 - 1/6).
    double g = 0.4;
    for (int it = 0; it < 60; ++it) g -= (g * g * g - 3 * g * g + 1.5 * g - 1.0 / 6.0) / (3 * g * g - 6 * g + 1.5);
    const double a21 = 2 * g, b2 = (0.5 - g) / a21, g21 = (g * g - g) / b2, b3 = g, b1 = 1.0 - b2 - b3;
    const double a31 = b1 / (1.0 - g), a32 = b2 / (1.0 - g);
    al[1][0] = a21; al[2][0] = a31; al[2][1] = a32;
    G[0][0] = G[1][1] = G[2][2] = g;
    G[1][0] = g21; G[2][0] = b1 - a31; G[2][1] = b2 - a32;
    b[0] = b1; b[1] = b2; b[2] = b3;
    from_alpha(3, al, G, b, &t);
  } else if (order == 3) {
    // ROS34PW2 (Rang & Angermann 2005)
    const double g = 4.3586652150845900e-01;
    al[1][0] = 8.7173304301691801e-01;
    al[2][0] = 8.4457060015369423e-01; al[2][1] = -1.1299064236484185e-01;
    al[3][0] = 0.0; al[3][1] = 0.0; al[3][2] = 1.0;
    for (int i = 0; i < 4; ++i) G[i][i] = g;
    G[1][0] = -8.7173304301691801e-01;
    G[2][0] = -9.0338057013044082e-01; G[2][1] = 5.4180672388095326e-02;
    G[3][0] = 2.4212380706095346e-01; G[3][1] = -1.2232505839045147e+00; G[3][2] = 5.4526025533510214e-01;
    b[0] = 2.4212380706095346e-01; b[1] = -1.2232505839045147e+00;
    b[2] = 1.5452602553351020e+00; b[3] = g;
    from_alpha(4, al, G, b, &t);
  } else {
    // RODASP (Steinebach 1995), entered in the transformed form
    t.s = 6;
    t.gamma = 0.25;
    const double r5[4] = {-7.170454962423024, -4.741636671481785, -16.31002631330971, -1.062004044111401};
    t.a[1][0] = 3.0;
    t.a[2][0] = 1.831036793486759; t.a[2][1] = 0.4955183967433795;
    t.a[3][0] = 2.304376582692669; t.a[3][1] = -0.05249275245743001; t.a[3][2] = -1.176798761832782;
    for (int j = 0; j < 4; ++j) { t.a[4][j] = r5[j]; t.a[5][j] = r5[j]; t.m[j] = r5[j]; }
    t.a[5][4] = 1.0;
    t.m[4] = 1.0; t.m[5] = 1.0;
    t.c[1][0] = -12.0;
    t.c[2][0] = -8.791795173947035; t.c[2][1] = -2.207865586973518;
    t.c[3][0] = 10.81793056857153; t.c[3][1] = 6.780270611428266; t.c[3][2] = 19.53485944642410;
    t.c[4][0] = 34.19095006749676; t.c[4][1] = 15.49671153725963; t.c[4][2] = 54.74760875964130;
    t.c[4][3] = 14.16005392148534;
    t.c[5][0] = 34.62605830930532; t.c[5][1] = 15.30084976114473; t.c[5][2] = 56.99955578662667;
    t.c[5][3] = 18.40807009793095; t.c[5][4] = -5.714285714285717;
  }
  return t;
}

struct EsdirkTab {
  int s = 0;
  double A[6][6] = {};
  double b[6] = {};
};

EsdirkTab esdirk_tableau(int order) {
  EsdirkTab t;
  if (order == 2) {
    const double g = 1.0 - std::sqrt(2.0) / 2.0, r = std::sqrt(2.0) / 4.0;
    t.s = 3;
    t.A[1][0] = g; t.A[1][1] = g;
    t.A[2][0] = r; t.A[2][1] = r; t.A[2][2] = g;
  } else if (order == 3) {
    const double g = 1767732205903.0 / 4055673282236.0;
    t.s = 4;
    t.A[1][0] = g; t.A[1][1] = g;
    t.A[2][0] = 2746238789719.0 / 10658868560708.0; t.A[2][1] = -640167445237.0 / 6845629431997.0;
    t.A[2][2] = g;
    t.A[3][0] = 1471266399579.0 / 7840856788654.0; t.A[3][1] = -4482444167858.0 / 7529755066697.0;
    t.A[3][2] = 11266239266428.0 / 11593286722821.0; t.A[3][3] = g;
  } else {
    const double q = 0.25;
    t.s = 6;
    t.A[1][0] = q; t.A[1][1] = q;
    t.A[2][0] = 8611.0 / 62500.0; t.A[2][1] = -1743.0 / 31250.0; t.A[2][2] = q;
    t.A[3][0] = 5012029.0 / 34652500.0; t.A[3][1] = -654441.0 / 2922500.0;
    t.A[3][2] = 174375.0 / 388108.0; t.A[3][3] = q;
    t.A[4][0] = 15267082809.0 / 155376265600.0; t.A[4][1] = -71443401.0 / 120774400.0;
    t.A[4][2] = 730878875.0 / 902184768.0; t.A[4][3] = 2285395.0 / 8070912.0; t.A[4][4] = q;
    t.A[5][0] = 82889.0 / 524892.0; t.A[5][1] = 0.0; t.A[5][2] = 15625.0 / 83664.0;
    t.A[5][3] = 69875.0 / 102672.0; t.A[5][4] = -2260.0 / 8211.0; t.A[5][5] = q;
  }
  for (int j = 0; j < t.s; ++j) t.b[j] = t.A[t.s - 1][j];
  return t;
}

// buffer roles
enum {
  B_R0 = 0, B_RHS, B_STAGE, B_RSTAGE, B_CONST, B_F, B_DQ, B_Q, B_RQ, B_NEW,
  B_Y0 = 10  // 6 stage vectors B_Y0 .. B_Y0+5
};
static_assert(B_GUESS_R == B_RSTAGE, "guess residual buffer");

int read_scalar(fr_ctx* ctx, const double* dev, double* host, cudaStream_t s) {
  FRK_CUDA(ctx, cudaMemcpyAsync(ctx->h_scal + 3, dev, sizeof(double), cudaMemcpyDeviceToHost, s));
  FRK_CUDA(ctx, cudaStreamSynchronize(s));
  *host = ctx->h_scal[3];
  return FR_OK;
}

// Linear solve with zero initial guess: x = A^{-1} b at tolerance tol.
int solve(fr_ctx* ctx, const double* U, const double* R0, double shift, const double* b, double* x,
          double tol, fr_step_stats* st, fr_gmres_info* info, cudaStream_t s) {
  FRK_TRY(launch_fill(ctx, x, 0.0, s));
  const int rc = gmres_impl(ctx, U, R0, shift, b, x, ctx->opts.gmres_m, tol,
                            ctx->opts.gmres_max_restarts, true, info, s);
  st->gmres_iters += info->iters;
  st->gmres_calls += 1;
  if (rc == FR_ERR_NOT_CONVERGED) {
    st->converged = 0;
    return FR_OK;  // the caller decides (ROW keeps going, PTC may reject)
  }
  return rc;
}

// Pseudo-transient continuation for F(q) = (q - cst)/(omega dt) - R(q) = 0
// (Sec. 4.4); q (in/out) starts from the given iterate; Rq receives R(q).
int ptc(fr_ctx* ctx, const double* cst, double omega_dt, double dt, double* q, double* Rq,
        const fr_ptc_opts& po, fr_step_stats* st, cudaStream_t s) {
  double* F = ctx->buf[B_F];
  double* dq = ctx->buf[B_DQ];
  double* nF2 = ctx->scal + S_NF2;
  auto eval_F = [&](double* Fn) -> int {
    FRK_TRY(launch_residual(ctx, 0, q, nullptr, nullptr, nullptr, Rq, 0.0, nullptr, nullptr, s));
    st->residual_evals += 1;
    const double* xs[3] = {q, cst, Rq};
    const double cs[3] = {1.0 / omega_dt, -1.0 / omega_dt, -1.0};
    FRK_TRY(launch_lincomb(ctx, F, 3, xs, cs, nF2, s));
    double v;
    FRK_TRY(read_scalar(ctx, nF2, &v, s));
    *Fn = std::sqrt(v);
    return FR_OK;
  };
  double Fn;
  FRK_TRY(eval_F(&Fn));
  if (!std::isfinite(Fn)) return set_error(ctx, FR_ERR_NONFINITE, "||F|| is not finite");
  const double F0 = Fn;
  double dtau = po.dtau_init > 0.0 ? po.dtau_init : dt;
  double dtau_max = po.dtau_max;
  int k = 0, rejections = 0;
  int formed_k = -1;          // pseudo iterate the staged blocks were formed at
  double blocks_shift = 0.0;  // shift of the current inverse blocks
  while (F0 > 0.0 && Fn / F0 >= po.tol_nl) {
    if (k >= po.max_iters) {
      st->converged = 0;
      return set_error(ctx, FR_ERR_NOT_CONVERGED, "PTC reached %d pseudo steps (||F||/||F0|| = %.3e)",
                       k, Fn / F0);
    }
    const double shift = 1.0 / dtau + 1.0 / omega_dt;
    if (ctx->opts.precond) {
      // blocks formed at the stage's first iterate (or every iterate with
      // precond_refresh = 1); a new shift only re-inverts the staged blocks
      if (k == 0 && rejections == 0 && formed_k < 0) {
        FRK_TRY(launch_block_factor(ctx, q, shift, s));
        formed_k = 0;
      } else if (ctx->opts.precond_refresh == 1 && formed_k != k) {
        FRK_TRY(launch_block_factor(ctx, q, shift, s));
        formed_k = k;
      } else if (ctx->opts.precond_refresh != 2 && blocks_shift != shift) {
        if (ctx->blk_chunk < ctx->ne) {
          // staged blocks are kept for one chunk of elements only: a new
          // shift forms the blocks again, at the current iterate
          FRK_TRY(launch_block_factor(ctx, q, shift, s));
          formed_k = k;
        } else {
          FRK_TRY(launch_block_reshift(ctx, shift, s));
        }
      }
      blocks_shift = shift;  // precond_refresh = 2 keeps the stage's first blocks and shift
    }
    ctx->blocks_valid = ctx->opts.precond;
    // b = -F into B_RHS
    const double* xs[1] = {F};
    const double cs[1] = {-1.0};
    FRK_TRY(launch_lincomb(ctx, ctx->buf[B_RHS], 1, xs, cs, nullptr, s));
    fr_gmres_info info{};
    const int conv_before = st->converged;
    FRK_TRY(solve(ctx, q, Rq, shift, ctx->buf[B_RHS], dq, po.tol_lin, st, &info, s));
    st->converged = conv_before;  // an inexact inner solve is not a failure of the step
    if (info.relres > po.reject_above) {
      ++rejections;
      ++st->rejections;
      if (rejections > po.max_rejections) {
        st->converged = 0;
        return set_error(ctx, FR_ERR_PTC_STALLED, "PTC: %d rejected pseudo steps", rejections);
      }
      dtau_max *= 0.5;
      dtau = std::fmin(dtau, dtau_max);
      continue;
    }
    const double* xq[2] = {q, dq};
    const double cq[2] = {1.0, 1.0};
    FRK_TRY(launch_lincomb(ctx, q, 2, xq, cq, nullptr, s));
    double Fnew;
    FRK_TRY(eval_F(&Fnew));
    if (!std::isfinite(Fnew)) return set_error(ctx, FR_ERR_NONFINITE, "||F|| is not finite");
    dtau = Fnew > 0.0 ? std::fmin(dtau * Fn / Fnew, dtau_max) : dtau_max;
    Fn = Fnew;
    ++k;
    ++st->ptc_iters;
  }
  return FR_OK;
}


// ROW prologue: R0 = R(q^n) and the element blocks at shift 1/(gamma dt).
int row_prologue(fr_ctx* ctx, const RowTab& t, double dt, const double* U, fr_step_stats* st,
                 cudaStream_t s) {
  FRK_TRY(launch_residual(ctx, 0, U, nullptr, nullptr, nullptr, ctx->buf[B_R0], 0.0, nullptr, nullptr, s));
  st->residual_evals += 1;
  if (ctx->opts.precond) {
    FRK_TRY(launch_block_factor(ctx, U, 1.0 / (t.gamma * dt), s));
    ctx->blocks_valid = 1;
  }
  return FR_OK;
}

// Right-hand side of ROW stage i: R(q^n + sum a_ij Y_j) + (1/dt) sum c_ij Y_j.
int row_stage_rhs(fr_ctx* ctx, const RowTab& t, int i, double dt, const double* U, fr_step_stats* st,
                  const double** b_out, cudaStream_t s) {
  const double* Ri = ctx->buf[B_R0];
  bool any_a = false;
  for (int j = 0; j < i; ++j) any_a |= t.a[i][j] != 0.0;
  if (i > 0 && any_a) {
    const double* xs[7];
    double cs[7];
    xs[0] = U; cs[0] = 1.0;
    for (int j = 0; j < i; ++j) { xs[j + 1] = ctx->buf[B_Y0 + j]; cs[j + 1] = t.a[i][j]; }
    FRK_TRY(launch_lincomb(ctx, ctx->buf[B_STAGE], i + 1, xs, cs, nullptr, s));
    FRK_TRY(launch_residual(ctx, 0, ctx->buf[B_STAGE], nullptr, nullptr, nullptr, ctx->buf[B_RSTAGE],
                            0.0, nullptr, nullptr, s));
    st->residual_evals += 1;
    Ri = ctx->buf[B_RSTAGE];
  }
  const double* b = Ri;
  if (i > 0) {
    const double* xs[7];
    double cs[7];
    xs[0] = Ri; cs[0] = 1.0;
    for (int j = 0; j < i; ++j) { xs[j + 1] = ctx->buf[B_Y0 + j]; cs[j + 1] = t.c[i][j] / dt; }
    FRK_TRY(launch_lincomb(ctx, ctx->buf[B_RHS], i + 1, xs, cs, nullptr, s));
    b = ctx->buf[B_RHS];
  }
  *b_out = b;
  return FR_OK;
}

// q^{n+1} = q^n + sum m_j Y_j into B_NEW, its squared norm into S_NX2.
int row_combine(fr_ctx* ctx, const RowTab& t, const double* U, cudaStream_t s) {
  const double* xs[7];
  double cs[7];
  xs[0] = U; cs[0] = 1.0;
  for (int j = 0; j < t.s; ++j) { xs[j + 1] = ctx->buf[B_Y0 + j]; cs[j + 1] = t.m[j]; }
  return launch_lincomb(ctx, ctx->buf[B_NEW], t.s + 1, xs, cs, ctx->scal + S_NX2, s);
}

}  // namespace
}  // namespace frk

using namespace frk;

extern "C" int step_row(fr_ctx* ctx, int scheme, double dt, double* U, fr_step_stats* stats,
                        void* stream) {
  if (!ctx || !U) return set_error(ctx, FR_ERR_INVALID_ARG, "step_row: null argument");
  if (scheme < 2 || scheme > 4) return set_error(ctx, FR_ERR_INVALID_ARG, "step_row: scheme %d", scheme);
  if (!(dt > 0.0)) return set_error(ctx, FR_ERR_INVALID_ARG, "step_row: dt must be > 0");
  cudaStream_t s = as_stream(stream);
  const RowTab t = row_tableau(scheme);
  fr_step_stats st{};
  st.converged = 1;
  const bool hist = ctx->hist_row == scheme;  // stage solutions of the last step still in place
  ctx->hist_row = 0;
  const double shift = 1.0 / (t.gamma * dt);
  double* R0 = ctx->buf[B_R0];
  FRK_TRY(row_prologue(ctx, t, dt, U, &st, s));
  for (int i = 0; i < t.s; ++i) {
    double* Yi = ctx->buf[B_Y0 + i];
    const double* b = nullptr;
    FRK_TRY(row_stage_rhs(ctx, t, i, dt, U, &st, &b, s));
    fr_gmres_info info{};
    // this stage's solution and right-hand side at the previous step (still in
    // place when the last step was a ROW step of this scheme on this state)
    const bool learn = ctx->cap.X || (ctx->guess && ctx->opts.guess == 2);
    const double* ylast = nullptr;
    const double* blast = nullptr;
    if (hist && learn) {
      FRK_TRY(launch_copy(ctx, ctx->buf[B_STAGE], Yi, s));  // B_STAGE is free after R(U_i)
      ylast = ctx->buf[B_STAGE];
      blast = ctx->bhist[i];
    }
    int mode = ctx->opts.guess;
    if (mode == 2 && !ctx->guess) mode = 1;
    if (mode != 0 && !hist) mode = 0;
    if (mode == 0) {
      FRK_TRY(solve(ctx, U, R0, shift, b, Yi, ctx->opts.tol_lin, &st, &info, s));
    } else {
      // nonzero initial guess: the previous step's solution (mode 1) or the
      // learned one, kept only when its residual is below the previous-step
      // guess's (mode 2); GMRES still stops at tol_lin * ||b||
      if (mode == 2) FRK_TRY(stage_guess(ctx, U, R0, shift, b, blast, ylast, Yi, s));
      const int rc = gmres_impl(ctx, U, R0, shift, b, Yi, ctx->opts.gmres_m, ctx->opts.tol_lin,
                                ctx->opts.gmres_max_restarts, false, &info, s);
      st.gmres_iters += info.iters;
      st.gmres_calls += 1;
      if (rc == FR_ERR_NOT_CONVERGED) st.converged = 0;
      else FRK_TRY(rc);
    }
    FRK_TRY(stage_capture(ctx, b, blast, ylast, Yi, s));
    if (learn) FRK_TRY(launch_copy(ctx, ctx->bhist[i], b, s));
  }

  // q^{n+1} = q^n + sum m_j Y_j, checked before it overwrites U
  FRK_TRY(row_combine(ctx, t, U, s));
  double nn;
  FRK_TRY(read_scalar(ctx, ctx->scal + S_NX2, &nn, s));
  if (stats) *stats = st;
  if (!std::isfinite(nn)) return set_error(ctx, FR_ERR_NONFINITE, "step_row: new state not finite");
  FRK_TRY(launch_copy(ctx, U, ctx->buf[B_NEW], s));
  FRK_CUDA(ctx, cudaStreamSynchronize(s));
  ctx->hist_row = scheme;
  if (!st.converged) return set_error(ctx, FR_ERR_NOT_CONVERGED, "step_row: a stage solve did not converge");
  return FR_OK;
}

extern "C" int step_esdirk(fr_ctx* ctx, int scheme, double dt, double* U, const fr_ptc_opts* ptc_opts,
                           fr_step_stats* stats, void* stream) {
  if (!ctx || !U) return set_error(ctx, FR_ERR_INVALID_ARG, "step_esdirk: null argument");
  if (scheme < 2 || scheme > 4) return set_error(ctx, FR_ERR_INVALID_ARG, "step_esdirk: scheme %d", scheme);
  if (!(dt > 0.0)) return set_error(ctx, FR_ERR_INVALID_ARG, "step_esdirk: dt must be > 0");
  fr_ptc_opts po;
  fr_default_ptc_opts(&po);
  if (ptc_opts) po = *ptc_opts;
  cudaStream_t s = as_stream(stream);
  const EsdirkTab t = esdirk_tableau(scheme);
  const double omega = t.A[1][1];
  ctx->hist_row = 0;
  fr_step_stats st{};
  st.converged = 1;
  // stage residuals R(q_j) in B_Y0 + j
  FRK_TRY(launch_residual(ctx, 0, U, nullptr, nullptr, nullptr, ctx->buf[B_Y0], 0.0, nullptr, nullptr,
                          s));
  st.residual_evals += 1;
  double* q = ctx->buf[B_Q];
  FRK_TRY(launch_copy(ctx, q, U, s));
  int rc = FR_OK;
  for (int i = 1; i < t.s; ++i) {
    const double* xs[7];
    double cs[7];
    xs[0] = U; cs[0] = 1.0;
    for (int j = 0; j < i; ++j) { xs[j + 1] = ctx->buf[B_Y0 + j]; cs[j + 1] = dt * t.A[i][j]; }
    FRK_TRY(launch_lincomb(ctx, ctx->buf[B_CONST], i + 1, xs, cs, nullptr, s));
    rc = ptc(ctx, ctx->buf[B_CONST], omega * dt, dt, q, ctx->buf[B_Y0 + i], po, &st, s);
    if (rc != FR_OK && rc != FR_ERR_NOT_CONVERGED) {
      if (stats) *stats = st;
      return rc;
    }
  }
  const double* xs[7];
  double cs[7];
  xs[0] = U; cs[0] = 1.0;
  for (int j = 0; j < t.s; ++j) { xs[j + 1] = ctx->buf[B_Y0 + j]; cs[j + 1] = dt * t.b[j]; }
  FRK_TRY(launch_lincomb(ctx, ctx->buf[B_NEW], t.s + 1, xs, cs, ctx->scal + S_NX2, s));
  double nn;
  FRK_TRY(read_scalar(ctx, ctx->scal + S_NX2, &nn, s));
  if (stats) *stats = st;
  if (!std::isfinite(nn)) return set_error(ctx, FR_ERR_NONFINITE, "step_esdirk: new state not finite");
  FRK_TRY(launch_copy(ctx, U, ctx->buf[B_NEW], s));
  FRK_CUDA(ctx, cudaStreamSynchronize(s));
  if (!st.converged) return set_error(ctx, FR_ERR_NOT_CONVERGED, "step_esdirk: a stage did not converge");
  return FR_OK;
}

extern "C" int step_bdf2(fr_ctx* ctx, double dt, double* U, double* U_prev, int first_step,
                         const fr_ptc_opts* ptc_opts, fr_step_stats* stats, void* stream) {
  if (!ctx || !U || !U_prev) return set_error(ctx, FR_ERR_INVALID_ARG, "step_bdf2: null argument");
  if (!(dt > 0.0)) return set_error(ctx, FR_ERR_INVALID_ARG, "step_bdf2: dt must be > 0");
  fr_ptc_opts po;
  fr_default_ptc_opts(&po);
  if (ptc_opts) po = *ptc_opts;
  cudaStream_t s = as_stream(stream);
  fr_step_stats st{};
  st.converged = 1;
  ctx->hist_row = 0;
  double omega, a1, a2;
  if (first_step) { omega = 1.0; a1 = 1.0; a2 = 0.0; }
  else { omega = 2.0 / 3.0; a1 = 4.0 / 3.0; a2 = -1.0 / 3.0; }
  {
    const double* xs[2] = {U, U_prev};
    const double cs[2] = {a1, a2};
    FRK_TRY(launch_lincomb(ctx, ctx->buf[B_CONST], first_step ? 1 : 2, xs, cs, nullptr, s));
  }
  double* q = ctx->buf[B_Q];
  FRK_TRY(launch_copy(ctx, q, U, s));
  const int rc = ptc(ctx, ctx->buf[B_CONST], omega * dt, dt, q, ctx->buf[B_RQ], po, &st, s);
  if (stats) *stats = st;
  if (rc != FR_OK && rc != FR_ERR_NOT_CONVERGED) return rc;
  FRK_TRY(launch_sumsq(ctx, q, ctx->scal + S_NX2, s));
  double nn;
  FRK_TRY(read_scalar(ctx, ctx->scal + S_NX2, &nn, s));
  if (!std::isfinite(nn)) return set_error(ctx, FR_ERR_NONFINITE, "step_bdf2: new state not finite");
  FRK_TRY(launch_copy(ctx, U_prev, U, s));
  FRK_TRY(launch_copy(ctx, U, q, s));
  FRK_CUDA(ctx, cudaStreamSynchronize(s));
  if (rc != FR_OK || !st.converged) return set_error(ctx, FR_ERR_NOT_CONVERGED, "step_bdf2: PTC did not converge");
  return FR_OK;
}

extern "C" int step_ssprk3(fr_ctx* ctx, double dt, double* U, fr_step_stats* stats, void* stream) {
  if (!ctx || !U) return set_error(ctx, FR_ERR_INVALID_ARG, "step_ssprk3: null argument");
  if (!(dt > 0.0)) return set_error(ctx, FR_ERR_INVALID_ARG, "step_ssprk3: dt must be > 0");
  cudaStream_t s = as_stream(stream);
  fr_step_stats st{};
  st.converged = 1;
  double* u1 = ctx->buf[B_STAGE];
  double* u2 = ctx->buf[B_Q];
  double* r = ctx->buf[B_RSTAGE];
  // u1 = U + dt R(U)
  FRK_TRY(launch_residual(ctx, 0, U, nullptr, nullptr, nullptr, r, 0.0, nullptr, nullptr, s));
  {
    const double* xs[2] = {U, r};
    const double cs[2] = {1.0, dt};
    FRK_TRY(launch_lincomb(ctx, u1, 2, xs, cs, nullptr, s));
  }
  // u2 = 3/4 U + 1/4 u1 + dt/4 R(u1)
  FRK_TRY(launch_residual(ctx, 0, u1, nullptr, nullptr, nullptr, r, 0.0, nullptr, nullptr, s));
  {
    const double* xs[3] = {U, u1, r};
    const double cs[3] = {0.75, 0.25, 0.25 * dt};
    FRK_TRY(launch_lincomb(ctx, u2, 3, xs, cs, nullptr, s));
  }
  // U_new = 1/3 U + 2/3 u2 + 2 dt/3 R(u2), checked before it overwrites U
  FRK_TRY(launch_residual(ctx, 0, u2, nullptr, nullptr, nullptr, r, 0.0, nullptr, nullptr, s));
  {
    const double* xs[3] = {U, u2, r};
    const double cs[3] = {1.0 / 3.0, 2.0 / 3.0, 2.0 * dt / 3.0};
    FRK_TRY(launch_lincomb(ctx, ctx->buf[B_NEW], 3, xs, cs, ctx->scal + S_NX2, s));
  }
  st.residual_evals = 3;
  double nn;
  FRK_TRY(read_scalar(ctx, ctx->scal + S_NX2, &nn, s));
  if (stats) *stats = st;
  if (!std::isfinite(nn)) return set_error(ctx, FR_ERR_NONFINITE, "step_ssprk3: new state not finite");
  FRK_TRY(launch_copy(ctx, U, ctx->buf[B_NEW], s));
  FRK_CUDA(ctx, cudaStreamSynchronize(s));
  ctx->hist_row = 0;
  return FR_OK;
}

// ---------------------------------------------------------------------------
// Batches of independent instances (uneven meshes and degrees) advanced
// together: the per-instance kernels of each phase run concurrently on one
// stream per instance, and every GMRES cycle of all instances is one CUDA
// graph launch (captured once per stage, replayed every step).

struct fr_batch {
  std::vector<fr_ctx*> m;
  cudaStream_t main = nullptr;
  std::vector<cudaStream_t> st;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  double* status_dev = nullptr;   // [count][4] GMRES cycle status
  double* status_host = nullptr;  // pinned mirror
  int* fin_dev = nullptr;         // [count] stage solve finished (reset per stage)
  cudaGraphExec_t exec[6] = {};
  long long nodes[6] = {};
  // batched Arnoldi iterations: instance tables and CTA partitions (device),
  // one group per degree 2..4 for the apply and the FD operator
  unsigned char* tab_dev = nullptr;
  size_t tab_bytes = 0;
  int batched = 0;          // 1: the cycles use the batched launches
  int use_batched = 1;      // set to 0 to capture per-instance cycles
  std::vector<const double*> keyU;
  std::vector<int> keyCfg;  // vec_blocks, tile_variant of every instance
  double key_dt = 0.0;
  int key_scheme = 0;
  char err[256] = {0};
};

namespace frk {
namespace {

int batch_err(fr_batch* B, int code, const char* msg) {
  if (B) {
    std::strncpy(B->err, msg, sizeof(B->err) - 1);
    B->err[sizeof(B->err) - 1] = 0;
  }
  return code;
}

#define BATCH_CUDA(B, call)                                                        \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) return batch_err((B), FR_ERR_CUDA, cudaGetErrorString(e_)); \
  } while (0)

#define BATCH_TRY(B, k, expr)                                                       \
  do {                                                                             \
    int r_ = (expr);                                                               \
    if (r_ != FR_OK) return batch_err((B), r_, fr_last_error((B)->m[k]));          \
  } while (0)

void free_batch(fr_batch* B) {
  if (!B) return;
  for (auto& e : B->exec)
    if (e) cudaGraphExecDestroy(e);
  for (fr_ctx* c : B->m) fr_ctx_destroy(c);
  for (cudaStream_t s : B->st) cudaStreamDestroy(s);
  for (cudaEvent_t e : B->join) cudaEventDestroy(e);
  if (B->fork) cudaEventDestroy(B->fork);
  if (B->main) cudaStreamDestroy(B->main);
  cudaFree(B->status_dev);
  cudaFree(B->fin_dev);
  cudaFree(B->tab_dev);
  cudaFreeHost(B->status_host);
  delete B;
}

// fork every instance stream off the main stream / join them back
int fork_all(fr_batch* B) {
  BATCH_CUDA(B, cudaEventRecord(B->fork, B->main));
  for (cudaStream_t s : B->st) BATCH_CUDA(B, cudaStreamWaitEvent(s, B->fork, 0));
  return FR_OK;
}
int join_all(fr_batch* B) {
  for (size_t k = 0; k < B->st.size(); ++k) {
    BATCH_CUDA(B, cudaEventRecord(B->join[k], B->st[k]));
    BATCH_CUDA(B, cudaStreamWaitEvent(B->main, B->join[k], 0));
  }
  return FR_OK;
}

// Layout of the batched-iteration tables in tab_dev, per degree g = 2, 3, 4
// (the instances of one degree form a group whose Arnoldi iterations run as
// one chain of batched launches on a stream of its own):
// [BatchKrylov x n_g][vec starts n_g+1][BatchApply x n_g][apply starts n_g+1]
// [ResArgs x n_g][tile starts n_g+1].
struct BatchPlan {
  size_t off_kry[3] = {}, off_vstart[3] = {};
  size_t off_app[3] = {}, off_astart[3] = {}, off_res[3] = {}, off_rstart[3] = {};
  int n[3] = {}, nb[3] = {};
  int app_blocks[3] = {}, res_blocks[3] = {}, vec_blocks[3] = {};
  size_t bytes = 0;
};

size_t align16(size_t x) { return (x + 15) / 16 * 16; }

// whether every instance can take the batched Arnoldi launches: 2D Euler,
// degree 2..4, element-Jacobi on, the FP64 FD operator
bool batchable(const fr_batch* B) {
  for (const fr_ctx* c : B->m)
    if (c->dim3 || c->viscous || c->p < 2 || c->p > 4 || !c->opts.precond || c->opts.jv_precision != 0)
      return false;
  return true;
}

BatchPlan plan_of(const fr_batch* B) {
  BatchPlan P;
  const int K = (int)B->m.size();
  for (const fr_ctx* c : B->m) P.n[c->p - 2] += 1;
  (void)K;
  size_t o = 0;
  for (int g = 0; g < 3; ++g) {
    P.nb[g] = 4 * (g + 3) * (g + 3);
    P.off_kry[g] = o; o = align16(o + (size_t)P.n[g] * sizeof(BatchKrylov));
    P.off_vstart[g] = o; o = align16(o + (size_t)(P.n[g] + 1) * sizeof(int));
    P.off_app[g] = o; o = align16(o + (size_t)P.n[g] * batch_apply_bytes());
    P.off_astart[g] = o; o = align16(o + (size_t)(P.n[g] + 1) * sizeof(int));
    P.off_res[g] = o; o = align16(o + (size_t)P.n[g] * batch_residual_bytes());
    P.off_rstart[g] = o; o = align16(o + (size_t)(P.n[g] + 1) * sizeof(int));
  }
  P.bytes = o;
  return P;
}

// fill the tables for A = shift I - dR/dU at the states U (host mirror, then
// one copy; called outside graph capture)
int fill_tables(fr_batch* B, BatchPlan* P, double shift, double* const* U) {
  const int K = (int)B->m.size();
  std::vector<unsigned char> h(P->bytes, 0);
  int fill[3] = {0, 0, 0};
  int acc_a[3] = {0, 0, 0}, acc_r[3] = {0, 0, 0}, acc_v[3] = {0, 0, 0};
  for (int k = 0; k < K; ++k) {
    fr_ctx* c = B->m[k];
    const int g = c->p - 2, q = fill[g]++;
    reinterpret_cast<BatchKrylov*>(h.data() + P->off_kry[g])[q] = batch_krylov_args(c);
    reinterpret_cast<int*>(h.data() + P->off_vstart[g])[q] = acc_v[g];
    acc_v[g] += (int)vec_grid_of(c);
    int* astart = reinterpret_cast<int*>(h.data() + P->off_astart[g]);
    int* rstart = reinterpret_cast<int*>(h.data() + P->off_rstart[g]);
    BATCH_TRY(B, k, fill_batch_apply(c, reinterpret_cast<BatchApply*>(h.data() + P->off_app[g] + q * batch_apply_bytes())));
    BATCH_TRY(B, k, fill_batch_residual(c, U[k], c->buf[B_R0], shift,
                                        h.data() + P->off_res[g] + q * batch_residual_bytes()));
    const unsigned ga = apply_grid_of(c), gr = residual_grid_of(c);
    if (ga == 0 || gr == 0) return batch_err(B, FR_ERR_UNSUPPORTED, "batched launch grid");
    astart[q] = acc_a[g];
    acc_a[g] += (int)ga;
    rstart[q] = acc_r[g];
    acc_r[g] += (int)gr;
  }
  for (int g = 0; g < 3; ++g) {
    reinterpret_cast<int*>(h.data() + P->off_vstart[g])[P->n[g]] = acc_v[g];
    P->vec_blocks[g] = acc_v[g];
    reinterpret_cast<int*>(h.data() + P->off_astart[g])[P->n[g]] = acc_a[g];
    reinterpret_cast<int*>(h.data() + P->off_rstart[g])[P->n[g]] = acc_r[g];
    P->app_blocks[g] = acc_a[g];
    P->res_blocks[g] = acc_r[g];
  }
  if (!B->tab_dev || B->tab_bytes < P->bytes) {
    cudaFree(B->tab_dev);
    B->tab_dev = nullptr;
    BATCH_CUDA(B, cudaMalloc(&B->tab_dev, P->bytes));
    B->tab_bytes = P->bytes;
  }
  BATCH_CUDA(B, cudaMemcpy(B->tab_dev, h.data(), P->bytes, cudaMemcpyHostToDevice));
  return FR_OK;
}

// capture the graph of one GMRES cycle of stage i for all instances
int capture_cycle(fr_batch* B, int i, const RowTab& t, double dt, double* const* U) {
  const double shift = 1.0 / (t.gamma * dt);
  cudaGraph_t g = nullptr;
  // launches enqueued while capturing run only when the graph is replayed;
  // per-family event timing does not apply inside a graph
  const long long launches0 = fr_kernel_launches();
  std::vector<unsigned> masks(B->m.size());
  for (size_t k = 0; k < B->m.size(); ++k) {
    masks[k] = B->m[k]->prof.mask;
    B->m[k]->prof.mask = 0;
  }
  // batched Arnoldi iterations when every instance allows them: the tables
  // are filled before the capture (a plain copy)
  B->batched = B->use_batched && batchable(B);
  BatchPlan P;
  if (B->batched) {
    P = plan_of(B);
    FRK_TRY(fill_tables(B, &P, shift, U));
  }
  BATCH_CUDA(B, cudaStreamBeginCapture(B->main, cudaStreamCaptureModeRelaxed));
  int rc = fork_all(B);
  const int K = (int)B->m.size();
  if (!B->batched) {
    for (int k = 0; k < K && rc == FR_OK; ++k) {
      fr_ctx* c = B->m[k];
      const double* b = (i == 0) ? c->buf[B_R0] : (i > 0 ? c->buf[B_RHS] : nullptr);
      rc = gmres_cycle_enqueue(c, U[k], c->buf[B_R0], shift, b, c->buf[B_Y0 + i], c->opts.gmres_m,
                               c->opts.tol_lin, B->status_dev + 4 * k, B->fin_dev + k, B->st[k]);
      if (rc != FR_OK) rc = batch_err(B, rc, fr_last_error(c));
    }
  } else {
    // per instance: r = b - A x and the cycle set-up; then every Arnoldi
    // iteration of all instances as batched launches on the main stream
    // (instances whose cycle is done skip their CTAs' work on the device);
    // then per instance: back substitution, solution update, status
    for (int k = 0; k < K && rc == FR_OK; ++k) {
      fr_ctx* c = B->m[k];
      const double* b = (i == 0) ? c->buf[B_R0] : (i > 0 ? c->buf[B_RHS] : nullptr);
      rc = gmres_cycle_prologue(c, U[k], c->buf[B_R0], shift, b, c->buf[B_Y0 + i], c->opts.gmres_m,
                                c->opts.tol_lin, B->fin_dev + k, B->st[k]);
      if (rc != FR_OK) rc = batch_err(B, rc, fr_last_error(c));
    }
    if (rc == FR_OK) rc = join_all(B);
    const int m = B->m[0]->opts.gmres_m, prec = B->m[0]->opts.block_precision, rm = B->m[0]->opts.riemann;
    unsigned char* T = B->tab_dev;
    // the groups' launches in order on the main stream, iteration by iteration
    for (int j = 0; j < m && rc == FR_OK; ++j) {
      for (int g = 0; g < 3 && rc == FR_OK; ++g) {
        if (!P.n[g]) continue;
        rc = launch_batch_apply(P.nb[g], prec, reinterpret_cast<const BatchApply*>(T + P.off_app[g]),
                                reinterpret_cast<const int*>(T + P.off_astart[g]), P.n[g], P.app_blocks[g], j,
                                B->main);
        if (rc == FR_OK)
          rc = launch_batch_residual(g + 2, rm, T + P.off_res[g], reinterpret_cast<const int*>(T + P.off_rstart[g]),
                                     P.n[g], P.res_blocks[g], j, B->main);
        if (rc == FR_OK)
          rc = launch_batch_gs_givens(reinterpret_cast<const BatchKrylov*>(T + P.off_kry[g]),
                                      reinterpret_cast<const int*>(T + P.off_vstart[g]), P.n[g], P.vec_blocks[g], j,
                                      B->main);
        if (rc != FR_OK) rc = batch_err(B, rc, "batched Arnoldi launch failed");
      }
    }
    if (rc == FR_OK) rc = fork_all(B);
    for (int k = 0; k < K && rc == FR_OK; ++k) {
      fr_ctx* c = B->m[k];
      rc = gmres_cycle_epilogue(c, c->buf[B_Y0 + i], B->status_dev + 4 * k, B->fin_dev + k, B->st[k]);
      if (rc != FR_OK) rc = batch_err(B, rc, fr_last_error(c));
    }
  }
  if (rc == FR_OK) rc = join_all(B);
  if (rc == FR_OK && cudaMemcpyAsync(B->status_host, B->status_dev, B->m.size() * 4 * sizeof(double),
                                     cudaMemcpyDeviceToHost, B->main) != cudaSuccess)
    rc = batch_err(B, FR_ERR_CUDA, "status copy capture failed");
  const cudaError_t ee = cudaStreamEndCapture(B->main, &g);
  for (size_t k = 0; k < B->m.size(); ++k) B->m[k]->prof.mask = masks[k];
  count_launches(launches0 - fr_kernel_launches());
  if (rc != FR_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  BATCH_CUDA(B, ee);
  size_t nn = 0;
  cudaGraphGetNodes(g, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  long long kernels = 0;
  if (nn && cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
    for (size_t q = 0; q < nn; ++q) {
      cudaGraphNodeType ty;
      if (cudaGraphNodeGetType(nodes[q], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kernels;
    }
  if (B->exec[i]) cudaGraphExecDestroy(B->exec[i]);
  B->exec[i] = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&B->exec[i], g, 0);
  cudaGraphDestroy(g);
  BATCH_CUDA(B, ei);
  B->nodes[i] = kernels;
  return FR_OK;
}

}  // namespace
}  // namespace frk

extern "C" int fr_batch_create(int count, const fr_mesh_desc* meshes, const int* degrees, const fr_opts* opts,
                               fr_batch** out) {
  if (!out) return FR_ERR_INVALID_ARG;
  *out = nullptr;
  if (count < 1 || !meshes || !degrees) return FR_ERR_INVALID_ARG;
  if (opts && opts->guess != 0) return FR_ERR_UNSUPPORTED;  // batch stage solves start from zero
  fr_batch* B = new (std::nothrow) fr_batch();
  if (!B) return FR_ERR_CUDA;
  int rc = FR_OK;
  for (int k = 0; k < count && rc == FR_OK; ++k) {
    fr_ctx* c = nullptr;
    rc = fr_ctx_create(&meshes[k], degrees[k], opts, &c);
    if (rc == FR_OK) B->m.push_back(c);
  }
  if (rc == FR_OK && cudaStreamCreateWithFlags(&B->main, cudaStreamNonBlocking) != cudaSuccess) rc = FR_ERR_CUDA;
  if (rc == FR_OK && cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess) rc = FR_ERR_CUDA;
  for (int k = 0; k < count && rc == FR_OK; ++k) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) rc = FR_ERR_CUDA;
    else B->st.push_back(s);
    if (rc == FR_OK && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) rc = FR_ERR_CUDA;
    else if (rc == FR_OK) B->join.push_back(e);
  }
  if (rc == FR_OK && cudaMalloc(&B->status_dev, (size_t)count * 4 * sizeof(double)) != cudaSuccess) rc = FR_ERR_CUDA;
  if (rc == FR_OK && cudaMallocHost(&B->status_host, (size_t)count * 4 * sizeof(double)) != cudaSuccess) rc = FR_ERR_CUDA;
  if (rc == FR_OK && cudaMalloc(&B->fin_dev, (size_t)count * sizeof(int)) != cudaSuccess) rc = FR_ERR_CUDA;
  if (rc != FR_OK) {
    free_batch(B);
    return rc;
  }
  *out = B;
  return FR_OK;
}

extern "C" int fr_batch_destroy(fr_batch* B) {
  free_batch(B);
  return FR_OK;
}

extern "C" const char* fr_batch_last_error(const fr_batch* B) { return B ? B->err : "invalid batch"; }

extern "C" int fr_batch_set_batched(fr_batch* B, int on) {
  if (!B || on < 0 || on > 1) return FR_ERR_INVALID_ARG;
  if (B->use_batched != on) {
    B->use_batched = on;
    for (auto& e : B->exec)
      if (e) { cudaGraphExecDestroy(e); e = nullptr; }
  }
  return FR_OK;
}

extern "C" int fr_batch_cycle_kernels(const fr_batch* B, long long* kernels) {
  if (!B || !kernels) return FR_ERR_INVALID_ARG;
  *kernels = 0;
  for (long long n : B->nodes) *kernels = n > *kernels ? n : *kernels;
  return FR_OK;
}

extern "C" fr_ctx* fr_batch_member(fr_batch* B, int k) {
  if (!B || k < 0 || k >= (int)B->m.size()) return nullptr;
  return B->m[k];
}

extern "C" int fr_batch_step_row(fr_batch* B, int scheme, double dt, double* const* U, fr_step_stats* stats,
                                 void* stream) {
  if (!B || !U) return FR_ERR_INVALID_ARG;
  if (scheme < 2 || scheme > 4 || !(dt > 0.0)) return batch_err(B, FR_ERR_INVALID_ARG, "bad scheme or dt");
  const int K = (int)B->m.size();
  for (int k = 0; k < K; ++k)
    if (!U[k]) return batch_err(B, FR_ERR_INVALID_ARG, "null state");
  const RowTab t = row_tableau(scheme);
  std::vector<fr_step_stats> st(K);
  for (auto& s : st) s.converged = 1;
  // order the batch after the caller's stream
  cudaStream_t caller = as_stream(stream);
  BATCH_CUDA(B, cudaEventRecord(B->fork, caller));
  BATCH_CUDA(B, cudaStreamWaitEvent(B->main, B->fork, 0));
  // (re)capture the cycle graphs when the states, dt or scheme changed
  std::vector<int> cfg(2 * K);
  for (int k = 0; k < K; ++k) {
    cfg[2 * k] = B->m[k]->vec_blocks;
    cfg[2 * k + 1] = B->m[k]->tile_variant;
  }
  bool same = B->key_scheme == scheme && B->key_dt == dt && (int)B->keyU.size() == K && B->keyCfg == cfg;
  for (int k = 0; same && k < K; ++k) same = B->keyU[k] == U[k];
  if (!same) {
    B->keyCfg = cfg;
    for (auto& e : B->exec)
      if (e) { cudaGraphExecDestroy(e); e = nullptr; }
    B->keyU.assign(U, U + K);
    B->key_dt = dt;
    B->key_scheme = scheme;
  }
  FRK_TRY(fork_all(B));
  for (int k = 0; k < K; ++k) {
    B->m[k]->hist_row = 0;
    BATCH_TRY(B, k, row_prologue(B->m[k], t, dt, U[k], &st[k], B->st[k]));
  }
  for (int i = 0; i < t.s; ++i) {
    for (int k = 0; k < K; ++k) {
      const double* b = nullptr;
      BATCH_TRY(B, k, row_stage_rhs(B->m[k], t, i, dt, U[k], &st[k], &b, B->st[k]));
      BATCH_TRY(B, k, launch_fill(B->m[k], B->m[k]->buf[B_Y0 + i], 0.0, B->st[k]));
    }
    FRK_TRY(join_all(B));
    BATCH_CUDA(B, cudaMemsetAsync(B->fin_dev, 0, (size_t)K * sizeof(int), B->main));
    if (!B->exec[i]) FRK_TRY(capture_cycle(B, i, t, dt, U));
    std::vector<int> conv(K, 0), cycles(K, 0);
    const int max_restarts = B->m[0]->opts.gmres_max_restarts;
    for (int cyc = 0; cyc <= max_restarts; ++cyc) {
      BATCH_CUDA(B, cudaGraphLaunch(B->exec[i], B->main));
      count_launches(B->nodes[i]);
      BATCH_CUDA(B, cudaStreamSynchronize(B->main));
      bool all = true;
      for (int k = 0; k < K; ++k) {
        const double* q = B->status_host + 4 * k;
        if (q[0] < 0.0) return batch_err(B, FR_ERR_TIMEOUT, "a kernel's bounded wait for its copies gave up");
        if (!std::isfinite(q[1])) return batch_err(B, FR_ERR_NONFINITE, "batch GMRES residual not finite");
        if (conv[k]) continue;
        st[k].gmres_iters += (int)q[0];
        if (q[0] > 0) cycles[k] += 1;
        if (q[1] <= q[2]) conv[k] = 1;
        all = all && conv[k];
      }
      if (all) break;
    }
    for (int k = 0; k < K; ++k) {
      st[k].gmres_calls += 1;
      if (!conv[k]) st[k].converged = 0;
    }
    FRK_TRY(fork_all(B));
  }
  for (int k = 0; k < K; ++k) BATCH_TRY(B, k, row_combine(B->m[k], t, U[k], B->st[k]));
  FRK_TRY(join_all(B));
  for (int k = 0; k < K; ++k)
    BATCH_CUDA(B, cudaMemcpyAsync(B->status_host + 4 * k, B->m[k]->scal + S_NX2, sizeof(double),
                                  cudaMemcpyDeviceToHost, B->main));
  BATCH_CUDA(B, cudaStreamSynchronize(B->main));
  for (int k = 0; k < K; ++k)
    if (!std::isfinite(B->status_host[4 * k]))
      return batch_err(B, FR_ERR_NONFINITE, "batch: a new state is not finite");
  FRK_TRY(fork_all(B));
  for (int k = 0; k < K; ++k) BATCH_TRY(B, k, launch_copy(B->m[k], U[k], B->m[k]->buf[B_NEW], B->st[k]));
  FRK_TRY(join_all(B));
  BATCH_CUDA(B, cudaEventRecord(B->fork, B->main));
  BATCH_CUDA(B, cudaStreamWaitEvent(caller, B->fork, 0));
  BATCH_CUDA(B, cudaStreamSynchronize(B->main));
  bool ok = true;
  for (int k = 0; k < K; ++k) {
    if (stats) stats[k] = st[k];
    ok = ok && st[k].converged;
  }
  if (!ok) return batch_err(B, FR_ERR_NOT_CONVERGED, "batch: a stage solve did not converge");
  return FR_OK;
}

// ---------------------------------------------------------------------------
// Batched ESDIRK / BDF2: every pseudo-transient iteration of an instance
// takes host decisions (acceptance, SER, rejection) on its own residual
// norms, so the instances cannot share one graph.  Instead a pool of host
// threads takes instances from a shared counter and runs each instance's
// step on that instance's stream; the kernels of different instances
// overlap on the device and their host waits overlap on the CPU.

namespace frk {
namespace {

int run_members(fr_batch* B, void* stream, int threads, const std::function<int(int)>& fn) {
  const int K = (int)B->m.size();
  cudaStream_t caller = as_stream(stream);
  BATCH_CUDA(B, cudaEventRecord(B->fork, caller));
  for (cudaStream_t s : B->st) BATCH_CUDA(B, cudaStreamWaitEvent(s, B->fork, 0));
  std::vector<int> rc(K, FR_OK);
  std::atomic<int> next{0};
  auto work = [&]() {
    for (int k = next.fetch_add(1); k < K; k = next.fetch_add(1)) rc[k] = fn(k);
  };
  int T = threads > 0 ? threads : (int)std::thread::hardware_concurrency();
  if (T < 1) T = 1;
  if (T > K) T = K;
  std::vector<std::thread> pool;
  for (int t = 1; t < T; ++t) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
  for (size_t k = 0; k < B->st.size(); ++k) {
    BATCH_CUDA(B, cudaEventRecord(B->join[k], B->st[k]));
    BATCH_CUDA(B, cudaStreamWaitEvent(caller, B->join[k], 0));
  }
  // most severe status first: hard errors, then non-convergence
  int worst = FR_OK;
  for (int k = 0; k < K; ++k) {
    if (rc[k] == FR_OK) continue;
    const bool soft = rc[k] == FR_ERR_NOT_CONVERGED || rc[k] == FR_ERR_PTC_STALLED;
    const bool worst_soft = worst == FR_OK || worst == FR_ERR_NOT_CONVERGED || worst == FR_ERR_PTC_STALLED;
    if (worst == FR_OK || (worst_soft && !soft)) {
      worst = rc[k];
      char msg[256];
      std::snprintf(msg, sizeof(msg), "instance %d: %s", k, fr_last_error(B->m[k]));
      batch_err(B, rc[k], msg);
    }
  }
  return worst;
}

}  // namespace
}  // namespace frk

extern "C" int fr_batch_step_esdirk(fr_batch* B, int scheme, double dt, double* const* U, const fr_ptc_opts* ptc,
                                    int threads, fr_step_stats* stats, void* stream) {
  if (!B || !U) return FR_ERR_INVALID_ARG;
  if (scheme < 2 || scheme > 4 || !(dt > 0.0)) return batch_err(B, FR_ERR_INVALID_ARG, "bad scheme or dt");
  const int K = (int)B->m.size();
  for (int k = 0; k < K; ++k)
    if (!U[k]) return batch_err(B, FR_ERR_INVALID_ARG, "null state");
  return run_members(B, stream, threads, [&](int k) {
    fr_step_stats st{};
    const int r = step_esdirk(B->m[k], scheme, dt, U[k], ptc, &st, B->st[k]);
    if (stats) stats[k] = st;
    return r;
  });
}

extern "C" int fr_batch_step_bdf2(fr_batch* B, double dt, double* const* U, double* const* U_prev, int first_step,
                                  const fr_ptc_opts* ptc, int threads, fr_step_stats* stats, void* stream) {
  if (!B || !U || !U_prev) return FR_ERR_INVALID_ARG;
  if (!(dt > 0.0)) return batch_err(B, FR_ERR_INVALID_ARG, "bad dt");
  const int K = (int)B->m.size();
  for (int k = 0; k < K; ++k)
    if (!U[k] || !U_prev[k]) return batch_err(B, FR_ERR_INVALID_ARG, "null state");
  return run_members(B, stream, threads, [&](int k) {
    fr_step_stats st{};
    const int r = step_bdf2(B->m[k], dt, U[k], U_prev[k], first_step, ptc, &st, B->st[k]);
    if (stats) stats[k] = st;
    return r;
  });
}

// ---------------------------------------------------------------------------
// Launch configuration: grid of the streaming vector kernels and the element
// tile of the Euler residual kernel, set by hand or measured.

extern "C" int fr_set_launch_config(fr_ctx* ctx, int vec_blocks, int tile_variant) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  if (vec_blocks < 1 || vec_blocks > kRedBlocks || tile_variant < 0 || tile_variant > 1)
    return set_error(ctx, FR_ERR_INVALID_ARG, "launch config: vec_blocks in [1, 4096], tile_variant 0 or 1");
  ctx->vec_blocks = vec_blocks;
  ctx->tile_variant = tile_variant;
  return FR_OK;
}

extern "C" int fr_get_launch_config(const fr_ctx* ctx, int* vec_blocks, int* tile_variant) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  if (vec_blocks) *vec_blocks = ctx->vec_blocks;
  if (tile_variant) *tile_variant = ctx->tile_variant;
  return FR_OK;
}

namespace frk {
namespace {
// candidate grids: 1..8 CTAs per SM on the 152 SMs
constexpr int kTuneGrids[] = {152, 304, 456, 608, 912, 1216};

int time_cycles(fr_ctx* ctx, const double* U, double shift, int reps, cudaEvent_t e0, cudaEvent_t e1,
                float* ms, cudaStream_t s) {
  double* b = ctx->buf[B_R0];
  double* x = ctx->buf[B_Y0];
  const int m = ctx->opts.gmres_m;
  // one warm-up cycle, then `reps` timed ones, each from x = 0
  for (int r = 0; r <= reps; ++r) {
    FRK_TRY(launch_fill(ctx, x, 0.0, s));
    if (r == 1) FRK_CUDA(ctx, cudaEventRecord(e0, s));
    FRK_TRY(gmres_cycle_enqueue(ctx, U, b, shift, b, x, m, 0.0, ctx->scal + S_ST0, nullptr, s));
  }
  FRK_CUDA(ctx, cudaEventRecord(e1, s));
  FRK_CUDA(ctx, cudaEventSynchronize(e1));
  FRK_CUDA(ctx, cudaEventElapsedTime(ms, e0, e1));
  *ms /= (float)reps;
  return FR_OK;
}
}  // namespace
}  // namespace frk

extern "C" int fr_autotune(fr_ctx* ctx, const double* U, double shift, int reps, double* ms_best,
                           double* ms_default, void* stream) {
  if (!ctx || !U) return FR_ERR_INVALID_ARG;
  if (reps < 1) reps = 1;
  if (!(shift >= 0.0)) return set_error(ctx, FR_ERR_INVALID_ARG, "autotune: shift must be >= 0");
  cudaStream_t s = as_stream(stream);
  const unsigned mask = ctx->prof.mask;
  ctx->prof.mask = 0;
  const int vb0 = ctx->vec_blocks, tv0 = ctx->tile_variant;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = FR_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    rc = set_error(ctx, FR_ERR_CUDA, "autotune: event creation failed");
  // the cycle's operator: R(U) and the element blocks at this shift
  if (rc == FR_OK)
    rc = launch_residual(ctx, 0, U, nullptr, nullptr, nullptr, ctx->buf[B_R0], 0.0, nullptr, nullptr, s);
  if (rc == FR_OK && ctx->opts.precond) {
    rc = launch_block_factor(ctx, U, shift, s);
    if (rc == FR_OK) ctx->blocks_valid = 1;
  }
  float best = 0.f, dflt = 0.f;
  int best_vb = vb0, best_tv = tv0;
  if (rc == FR_OK) rc = time_cycles(ctx, U, shift, reps, e0, e1, &dflt, s);
  best = dflt;
  const int ntv = (ctx->viscous || ctx->dim3) ? 1 : 2;  // the viscous and 3D residuals have one tile shape
  for (int tv = 0; tv < ntv && rc == FR_OK; ++tv)
    for (int vb : kTuneGrids) {
      ctx->vec_blocks = vb;
      ctx->tile_variant = tv;
      float ms = 0.f;
      rc = time_cycles(ctx, U, shift, reps, e0, e1, &ms, s);
      if (rc != FR_OK) break;
      if (ms < best) {
        best = ms;
        best_vb = vb;
        best_tv = tv;
      }
    }
  ctx->vec_blocks = rc == FR_OK ? best_vb : vb0;
  ctx->tile_variant = rc == FR_OK ? best_tv : tv0;
  ctx->prof.mask = mask;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc != FR_OK) return rc;
  if (ms_best) *ms_best = best;
  if (ms_default) *ms_default = dflt;
  return FR_OK;
}
