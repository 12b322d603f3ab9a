// Internal declarations shared by the translation units of libfrjfnk.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>

#include "frjfnk.h"

namespace frk {

constexpr int kMaxN = 7;          // p <= 6 (2D Euler); p <= 4 with viscous terms and in 3D
constexpr int kThreads = 256;     // default block size of the vector kernels
constexpr int kMaxVec = 64;       // largest Krylov basis slice handled per call (m_max + 1)
constexpr int kVecBlocks = 456;   // default grid of the streaming vector kernels (3 x 152 SMs)
constexpr int kRedBlocks = 4096;  // capacity of the partial-sum buffer (blocks)
constexpr long long kStageChunk3 = 4096;  // elements per FP64 staging chunk of 3D degree-3 blocks

// 1D tables of Sec. 3 on Gauss-Legendre points, passed to kernels by value.
//   Dt[i][k] = D_ik - g_L'(xi_i) l_k(-1) - g_R'(xi_i) l_k(+1)
// folds the local-flux traces F^l(+-1) into the derivative matrix, so the
// corrected divergence is  sum_k Dt_ik F_k + g_L'_i F^num_L + g_R'_i F^num_R.
struct Tables {
  double D[kMaxN][kMaxN];   // D_ik = l_k'(xi_i)
  double Dt[kMaxN][kMaxN];
  double lm[kMaxN];   // l_k(-1)
  double lp[kMaxN];   // l_k(+1)
  double dgL[kMaxN];  // g_L'(xi_i)
  double dgR[kMaxN];  // g_R'(xi_i)
  double xi[kMaxN];   // solution points
  double w[kMaxN];    // quadrature weights
};

// Deterministic two-stage reduction scratch: per-block partial sums and a
// completion counter (the last block to finish sums the partials in a fixed
// order and resets the counter).
struct Reduce {
  double* partials;   // [kRedBlocks][kMaxVec]
  unsigned* counter;
};

// GMRES cycle state kept on the device so a whole cycle is launched without
// host round trips.
struct GmresDev {
  double* H;        // (m_max+1) x m_max, column-major: H[j*(m_max+1) + i]
  double* cs;       // Givens cosines [m_max]
  double* sn;       // Givens sines [m_max]
  double* g;        // rotated rhs [m_max+1]
  double* y;        // least-squares solution [m_max]
  double* h1;       // first Gram-Schmidt coefficients [kMaxVec]
  double* h2;       // second (re-orthogonalisation) coefficients [kMaxVec]
  double* invh;     // 1/||v_j|| of the not-yet-normalised basis vector j [m_max+1]
  int* done;        // cycle finished (converged or breakdown)
  int* rflag;       // [m_max] 1 if iteration j needed the second Gram-Schmidt pass
  int* k;           // iterations done in this cycle
  double* res;      // |g_k|
  double* target;   // rtol * ||b||
  int ldh;          // m_max + 1
};

// Per-instance arguments of the batched Arnoldi-step kernels (the basis of
// the instance, its GMRES state, its reduction scratch and ||w||^2 slot).
struct BatchKrylov {
  double* V;        // basis, ldv = n
  long long n;
  GmresDev gd;
  Reduce red;
  double* nw2;      // ||w||^2 of the current Arnoldi vector
  double eta2;      // second Gram-Schmidt pass when ||w_new||^2 < eta2 ||w_old||^2
};

// Device scalars (sums of squares) used by the FD step and GMRES.
enum Scal { S_NU2 = 0, S_NZ2, S_NW2, S_NB2, S_NR2, S_NF2, S_NX2, S_EPS, S_IEPS, S_GB2, S_GU2, S_GR1, S_GR2, S_ST0, S_ST1, S_ST2, S_ST3, S_COUNT };  // S_ST*: one GMRES cycle status

// FD step eps = eps_rel (1 + ||U||) / ||z|| (or eps_fixed), written once per
// product as (eps, 1/eps) by the kernel that finishes ||z||^2.
struct EpsArgs {
  const double* nU2;  // ||U||^2
  double eps_rel;
  double eps_fixed;
  double* out;        // [eps, 1/eps], nullptr: not needed
};

}  // namespace frk

namespace frk {
// CUDA-event timing of kernel families (measurement only).
struct Prof {
  unsigned mask = 0;
  static constexpr int kPairs = 2048;
  cudaEvent_t* ev[FR_KF_COUNT] = {};  // 2 * kPairs events per family
  int used[FR_KF_COUNT] = {};
  double ms[FR_KF_COUNT] = {};
  long long n[FR_KF_COUNT] = {};
  long long skipped[FR_KF_COUNT] = {};  // launches that found the GMRES cycle finished
  double bytes[FR_KF_COUNT] = {};       // algorithmic bytes of the timed launches
  double flops[FR_KF_COUNT] = {};       // algorithmic flops of the timed launches
};
}  // namespace frk

struct fr_mlp;

namespace frk {
// Training-pair capture of ROW stage solves (features and scaled targets).
struct StageCapture {
  float* X = nullptr;       // [max][3 nb]
  float* T = nullptr;       // [max][nb]
  long long max = 0, count = 0, offset = 0;
  int stride = 1;           // sample every stride-th element, rotating the offset per stage
};
}  // namespace frk

struct fr_ctx {
  int device = 0;
  int nx = 0, ny = 0, p = 0, n1 = 0, np = 0, nb = 0;
  int dim3 = 0;              // 3D hexahedral Navier-Stokes path (5 variables, Np = (p+1)^3)
  int nz = 1;
  double* hz = nullptr;      // 3D: [nz] element depths (device)
  double volume = 0.0;       // 3D: volume of the periodic box
  double* diss = nullptr;    // 3D: the three quadrature sums of the dissipation rate
  long long ne = 0, ndof = 0;
  fr_opts opts{};
  frk::Tables tab{};
  double* hx = nullptr;      // [nx] element widths (device)
  double* hy = nullptr;      // [ny] element heights (device)
  double* xo = nullptr;      // 2D: [nx] left edges of the element columns (device)
  double* yo = nullptr;      // 2D: [ny] bottom edges of the element rows (device)
  double box[4] = {};        // 2D: x_edges[0], x_edges[nx], y_edges[0], y_edges[ny]
  int wall_y = 0;            // isothermal no-slip walls at the y ends (viscous runs)
  int viscous = 0;           // Navier-Stokes (BR2) residual instead of Euler
  double* tb = nullptr;      // viscous: face traces (q, grad q) of every element
  double* mst = nullptr;     // viscous: staging of the FD element blocks before inversion
  double* rloc = nullptr;    // viscous: R(U) at the linearisation point of the blocks
  float* r0f = nullptr;      // FP32 block columns: element-local R(U) of one staging chunk
  float* tbf = nullptr;      // FP32 block columns: FP32 copy of the 3D trace buffer
  // 3D A z with FP32 linear parts: caches at the linearisation point and FP32 buffers
  double* lin3_tb = nullptr;
  double* lin3_fb = nullptr;
  double* lin3_g = nullptr;
  double* lin3_f = nullptr;
  float* lin3_tbz = nullptr;
  float* lin3_fbz = nullptr;
  double* lin3_gc = nullptr;
  double staged_shift = 0.0; // shift the staged blocks in mst were formed with
  long long blk_chunk = 0;   // elements whose staged blocks mst holds at once (ne unless staged in chunks)
  int hist_row = 0;          // ROW order of the last step if its stage solutions are intact
  fr_mlp* guess = nullptr;   // learned initial-guess model (ROW stages), or null
  float* gfeat = nullptr;    // [ne][3 nb] features for the guess
  float* gout = nullptr;     // [ne][nb] model output
  double* bhist[6] = {};     // right-hand sides of the last ROW step's stages (guess features)
  long long guess_tried = 0, guess_used = 0;
  frk::StageCapture cap;
  double* blocks = nullptr;  // [ne][nb][nb] inverse blocks, column-major per element
  int blocks_valid = 0;
  double* V = nullptr;       // (m_max+1) x ndof Krylov basis
  double* z = nullptr;       // preconditioned basis vector
  double* buf[16] = {};      // stepper buffers, ndof each
  double* scal = nullptr;    // frk::S_COUNT device scalars
  double* fb = nullptr;      // Navier-Stokes face data [ne][3][n1][8] (q_com, f_n)
  double* lin_fg = nullptr;  // mixed A z: F(U), G(U) at the points [ne][8][np]
  double* lin_fx = nullptr;  // mixed A z: per element's west face point (q-, q+, f^num) [ne][n1][12]
  double* lin_fy = nullptr;  // mixed A z: per element's south face point, same layout
  int num_sms = 1;           // SMs of the device (persistent grids)
  int* kerr = nullptr;       // device flag: a kernel's bounded wait gave up
  unsigned wait_polls = 1u << 22;  // poll limit of the element-Jacobi apply's bounded waits
  int test_skip_copy = 0;    // test hook: the apply leaves one copy unissued (see fr_set_wait_test)
  int vec_blocks = frk::kVecBlocks;  // grid of the streaming vector kernels (autotuned)
  int tile_variant = 0;      // element-tile shape of the Euler residual kernel (autotuned)
  frk::Reduce red{};
  frk::GmresDev gd{};
  int* h_stat = nullptr;     // pinned host mirror: done, k
  double* h_scal = nullptr;  // pinned host mirror of a few doubles
  frk::Prof prof;
  cudaEvent_t chunk_ev[2] = {nullptr, nullptr};  // GMRES look-ahead status events
  char err[512] = {0};
};

namespace frk {

int set_error(fr_ctx* ctx, int code, const char* fmt, ...);
// message returned by fr_last_error(NULL) (calls without a context)
void set_static_error(const char* msg);

#define FRK_CUDA(ctx, call)                                                           \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return ::frk::set_error((ctx), FR_ERR_CUDA, "%s failed: %s (%s:%d)", #call,     \
                              cudaGetErrorString(e_), __FILE__, __LINE__);           \
  } while (0)

#define FRK_LAUNCHED(ctx)                                                             \
  do {                                                                               \
    cudaError_t e_ = cudaGetLastError();                                             \
    if (e_ != cudaSuccess)                                                           \
      return ::frk::set_error((ctx), FR_ERR_CUDA, "kernel launch failed: %s (%s:%d)", \
                              cudaGetErrorString(e_), __FILE__, __LINE__);           \
  } while (0)

#define FRK_TRY(expr)         \
  do {                        \
    int r_ = (expr);          \
    if (r_ != FR_OK) return r_; \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Launch accounting: every kernel launch goes through prof_begin / prof_end.
void count_launch();
void count_launches(long long n);
void prof_begin(fr_ctx* ctx, int family, cudaStream_t s);
void prof_end(fr_ctx* ctx, int family, cudaStream_t s);

void prof_work(fr_ctx* ctx, int family, double bytes, double flops);

struct ProfScope {
  fr_ctx* c;
  int f;
  cudaStream_t s;
  ProfScope(fr_ctx* ctx, int family, cudaStream_t st, double bytes = 0.0, double flops = 0.0)
      : c(ctx), f(family), s(st) {
    prof_begin(c, f, s);
    prof_work(c, f, bytes, flops);
  }
  ~ProfScope() { prof_end(c, f, s); }
};

// Algorithmic work per launch (counting rules; see the launch sites).
double residual_flops_per_element(int p);
double ns_residual_flops_per_element(int p);
double jv_flops_per_element(const fr_ctx* ctx);  // Euler or Navier-Stokes
double factor_flops_per_element(int p);

// ---- launchers implemented in the .cu files --------------------------------
// residual.cu: mode 0: out = R(U); mode 1: out = A z; mode 2: out = b - A z
// eps2 points at the device pair (eps, 1/eps) of the product (modes 1, 2)
// mixed-precision A z (jv_precision 1): cache F(U), G(U) and the face states
// and common fluxes at U for the following modes 1 / 2; no-op otherwise
int launch_linearize(fr_ctx* ctx, const double* U, cudaStream_t s);
int launch_residual(fr_ctx* ctx, int mode, const double* U, const double* z, const double* R0,
                    const double* b, double* out, double shift, const double* eps2,
                    const int* done, cudaStream_t s);
// blocks.cu
int launch_block_factor(fr_ctx* ctx, const double* U, double shift, cudaStream_t s);
int launch_block_apply(fr_ctx* ctx, double* r, const double* scale, double* z, double* sumsq,
                       const int* done, cudaStream_t s, bool with_eps = false);
int launch_solution_update(fr_ctx* ctx, double* x, cudaStream_t s);
// krylov.cu
int launch_sumsq(fr_ctx* ctx, const double* x, double* out, cudaStream_t s, bool with_eps = false);
EpsArgs eps_args(fr_ctx* ctx, bool on);
int launch_lincomb(fr_ctx* ctx, double* out, int nterms, const double* const* xs,
                   const double* coefs, double* sumsq, cudaStream_t s);
int launch_copy(fr_ctx* ctx, double* dst, const double* src, cudaStream_t s);
int launch_fill(fr_ctx* ctx, double* dst, double v, cudaStream_t s);
int gmres_impl(fr_ctx* ctx, const double* U, const double* R0, double shift, const double* b,
               double* x, int m, double rtol, int max_restarts, bool x_is_zero,
               fr_gmres_info* info, cudaStream_t s);
// fin (device int, may be NULL): set by the cycle once the solve met its
// tolerance; a cycle that finds it set does no work (for replayed graphs).
int gmres_cycle_enqueue(fr_ctx* ctx, const double* U, const double* R0, double shift, const double* b,
                        double* x, int m, double rtol, double* status, int* fin, cudaStream_t s);
// the cycle's parts (batches enqueue the Arnoldi iterations of all instances
// as batched launches between them)
int gmres_cycle_prologue(fr_ctx* ctx, const double* U, const double* R0, double shift, const double* b,
                         double* x, int m, double rtol, int* fin, cudaStream_t s);
int gmres_cycle_epilogue(fr_ctx* ctx, double* x, double* status, int* fin, cudaStream_t s);
// batched Arnoldi-step kernels (krylov.cu, blocks.cu, residual.cu); the
// instance tables and CTA partitions are device arrays
BatchKrylov batch_krylov_args(fr_ctx* ctx);
unsigned vec_grid_of(const fr_ctx* ctx);
int launch_batch_gs_givens(const BatchKrylov* tab, const int* start, int ninst, int nblocks, int j, cudaStream_t s);
// apply: the per-instance launch grid of the block apply (blocks.cu) and the
// batched apply of the instances of one block size nb
struct BatchApply;
unsigned apply_grid_of(fr_ctx* ctx);
int fill_batch_apply(fr_ctx* ctx, BatchApply* out);
int launch_batch_apply(int nb, int prec, const BatchApply* tab, const int* start, int ninst, int nblocks, int j,
                       cudaStream_t s);
size_t batch_apply_bytes();
// residual: A z of Arnoldi iteration j into V_{j+1} for the instances of one degree
int fill_batch_residual(fr_ctx* ctx, const double* U, const double* R0, double shift, void* out);
size_t batch_residual_bytes();
unsigned residual_grid_of(const fr_ctx* ctx);
int launch_batch_residual(int p, int riemann, const void* tab, const int* start, int ninst, int nblocks, int j,
                          cudaStream_t s);
// tables.cu
void build_tables(int p, Tables* t);
// ns.cu (viscous path): mode 0 R, 1 A z, 2 b - A z; block formation + inversion
int launch_ns_residual(fr_ctx* ctx, int mode, const double* U, const double* z, const double* R0,
                       const double* b, double* out, double shift, const double* eps2,
                       const int* done, cudaStream_t s);
int launch_ns_factor(fr_ctx* ctx, const double* U, double shift, cudaStream_t s);
// fr3d.cu (3D path): mode 0 R, 1 A z, 2 b - A z; element blocks (p <= 2);
// quadrature sums (S^d:S^d, p div v, rho |v|^2/2) of the dissipation rate into out[0..2]
double ns3d_residual_flops_per_element(int p);
int launch_f3_residual(fr_ctx* ctx, int mode, const double* U, const double* z, const double* R0,
                       const double* b, double* out, double shift, const double* eps2,
                       const int* done, cudaStream_t s);
int launch_f3_factor(fr_ctx* ctx, const double* U, double shift, cudaStream_t s);
int launch_f3_dissipation(fr_ctx* ctx, const double* U, double* out, cudaStream_t s);
// vortex.cu: quadrature sums of (s_exact - s_num)^2 |J| w_i w_j for s = rho, u, v, p
// against the exact isentropic vortex into out[0..3]
int launch_vortex_error(fr_ctx* ctx, const double* U, const fr_vortex* vx, double t, double* out,
                        cudaStream_t s);
// blocks.cu: invert staged FP64 blocks (column-major M[c][row], dshift added to
// the diagonal) into ctx->blocks; re-invert the staged blocks at a new shift
int launch_block_invert(fr_ctx* ctx, const double* mst, double dshift, cudaStream_t s);
// caches of the 3D A z with FP32 linear parts at U (no-op unless jv_precision = 1)
int launch_f3_linearize(fr_ctx* ctx, const double* U, cudaStream_t s);
// invert the staged blocks of elements e0 .. e0 + n - 1 (mst holds them from its start)
int launch_block_invert_range(fr_ctx* ctx, const double* mst, double dshift, long long e0, long long n,
                              cudaStream_t s);
int launch_block_reshift(fr_ctx* ctx, double shift, cudaStream_t s);
// guess.cu (B_GUESS_R: stepper buffer free while a stage solve starts)
constexpr int B_GUESS_R = 3;
int stage_guess(fr_ctx* ctx, const double* U, const double* R0, double shift, const double* b,
                const double* bl, const double* yl, double* x0, cudaStream_t s);
int stage_capture(fr_ctx* ctx, const double* b, const double* bl, const double* yl, const double* y,
                  cudaStream_t s);

}  // namespace frk
