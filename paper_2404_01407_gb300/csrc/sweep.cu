// Fused block-Jacobi sweep over the mean flow and every harmonic.
//
// Paper: arXiv 2404.01407, "Solution Update" -- the block-diagonal inversion
// "performed point by point" (block Jacobi) of Eq. lhs_mean / Eq. lhs_lin with
// the harmonic LHS of Eq. precon_linear, K_l = K + i omega_l V I, sharing one
// J across all systems:
//   x_i <- (J_ii + (D_i + i omega_k V_i) I)^-1 (B_i - sum_j J_ij x_j).
//
// Design (GB300): one thread per (node, system).  Each thread streams the
// node's off-diagonal blocks (shared by the node's K threads through L1),
// gathers the neighbours' Re/Im columns of its system, accumulates the
// off-diagonal product in registers and solves its shifted diagonal system
// in registers.  The sweeps run in the per-node Hessenberg basis prepared by
// fnlh_prepare (x = Q x~), where the diagonal block of system k is
// H_i + i omega_k V_i I and the solve costs O(b^2).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "sweep_kernel.cuh"

namespace fnlh {

struct SweepArgs {
  int32_t n;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const void* offd;  // rotated blocks, TJ
  const void* hess;  // [n][b][b] T
  const double* vol;
  const void* Bt;    // [n][C][b] T, rotated right-hand side
  const void* Xin;   // [n][C][b] T (not read when x_zero)
  void* Xout;        // [n][C][b] T
  int32_t x_zero;
  Systems sys;
};

template <int BS, typename TJ, typename T>
__global__ void __launch_bounds__(256) k_sweep(const __grid_constant__ SweepArgs a) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int K = a.sys.K;
  if (g >= (long long)a.n * K) return;
  const int i = (int)(g / K);
  const int k = (int)(g - (long long)i * K);
  sweep_pair<BS, TJ, T>(a.row_ptr, a.col_idx, (const TJ*)a.offd, (const T*)a.hess, a.vol, (const T*)a.Bt,
                        (const T*)a.Xin, (T*)a.Xout, a.sys.C, i, k, a.sys.omega[k], a.x_zero != 0);
}

// y_i[c] = Q_i^T x_i[c]  (into the Hessenberg basis), one thread per (node, column).
template <int BS, typename TO>
__global__ void __launch_bounds__(256) k_rotate_in(long long count, int C, const double* __restrict__ rot,
                                                   const double* __restrict__ x, TO* __restrict__ y) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= count) return;
  const long long i = g / C;
  const double* Q = rot + i * BS * BS;
  double v[BS];
#pragma unroll
  for (int t = 0; t < BS; ++t) v[t] = x[g * BS + t];
#pragma unroll
  for (int r = 0; r < BS; ++r) {
    double acc = 0.0;
#pragma unroll
    for (int t = 0; t < BS; ++t) acc += Q[t * BS + r] * v[t];
    y[g * BS + r] = (TO)acc;
  }
}

// x_i[c] (+)= Q_i y_i[c]  (back to the original basis, FP64), one thread per (node, column).
template <int BS, typename TI>
__global__ void __launch_bounds__(256) k_rotate_out(long long count, int C, const double* __restrict__ rot,
                                                    const TI* __restrict__ y, double* __restrict__ x, int accumulate) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= count) return;
  const long long i = g / C;
  const double* Q = rot + i * BS * BS;
  double v[BS];
#pragma unroll
  for (int t = 0; t < BS; ++t) v[t] = (double)y[g * BS + t];
#pragma unroll
  for (int r = 0; r < BS; ++r) {
    double acc = accumulate ? x[g * BS + r] : 0.0;
#pragma unroll
    for (int t = 0; t < BS; ++t) acc += Q[r * BS + t] * v[t];
    x[g * BS + r] = acc;
  }
}

static inline unsigned blocks_for(long long count, int threads) {
  return (unsigned)((count + threads - 1) / threads);
}

template <int BS, typename TO>
int rotate_in(int n, int C, const double* rot, const double* x, TO* y, cudaStream_t s) {
  const long long count = (long long)n * C;
  if (count == 0) return FNLH_OK;
  k_rotate_in<BS, TO><<<blocks_for(count, 256), 256, 0, s>>>(count, C, rot, x, y);
  FNLH_LAUNCH_CHECK();
  return FNLH_OK;
}

template <int BS, typename TI>
int rotate_out(int n, int C, const double* rot, const TI* y, double* x, int accumulate, cudaStream_t s) {
  const long long count = (long long)n * C;
  if (count == 0) return FNLH_OK;
  k_rotate_out<BS, TI><<<blocks_for(count, 256), 256, 0, s>>>(count, C, rot, y, x, accumulate);
  FNLH_LAUNCH_CHECK();
  return FNLH_OK;
}

template <int BS, typename TJ, typename T>
int sweep_launch(const SweepArgs& a, int threads, cudaStream_t s) {
  const long long count = (long long)a.n * a.sys.K;
  if (count == 0) return FNLH_OK;
  if (threads <= 0) threads = 256;
  k_sweep<BS, TJ, T><<<blocks_for(count, threads), threads, 0, s>>>(a);
  FNLH_LAUNCH_CHECK();
  return FNLH_OK;
}

// Everything a sweep needs, resolved from the prep blob for one precision.
struct SweepOperands {
  const void* offd;
  const void* hess;
  const double* rot;
};

int sweep_operands(const fnlh_jacobian* J, int precision, SweepOperands* o) {
  const PrepLayout L = prep_layout(J->n_nodes, J->nnz, J->block, J->prep_flags);
  o->rot = at<double>(J->prep, L.rot);
  if (precision == FNLH_F64) {
    if (L.offd64 == (size_t)-1) return FNLH_ERR_WORKSPACE;
    o->offd = at<double>(J->prep, L.offd64);
    o->hess = at<double>(J->prep, L.hess);
  } else {
    const size_t off = (precision == FNLH_F32) ? L.offd32 : L.offd16;
    if (off == (size_t)-1 || L.hessf == (size_t)-1) return FNLH_ERR_WORKSPACE;
    o->offd = (const char*)J->prep + off;
    o->hess = at<float>(J->prep, L.hessf);
  }
  return FNLH_OK;
}

Systems make_systems(int n_harm, const double* omega) {
  Systems s;
  s.K = 1 + n_harm;
  s.C = 1 + 2 * n_harm;
  for (int k = 0; k < kMaxSys; ++k) s.omega[k] = 0.0;
  for (int k = 1; k <= n_harm; ++k) s.omega[k] = omega[k - 1];
  return s;
}

// Optional timing events around the sweep launches (fnlh_set_sweep_events).
static thread_local cudaEvent_t g_ev_begin = nullptr, g_ev_end = nullptr;

void set_sweep_events(cudaEvent_t b, cudaEvent_t e) {
  g_ev_begin = b;
  g_ev_end = e;
}

static inline int mark(cudaEvent_t ev, cudaStream_t s) {
  if (ev && g_ev_begin && g_ev_end) FNLH_CUDA_TRY(cudaEventRecord(ev, s));
  return FNLH_OK;
}

// Runs `sweeps` sweeps between the ping-pong buffers x0/x1 starting from x0
// (or from zero when x_zero), returns the buffer holding the result.
template <int BS, typename TJ, typename T>
int run_sweeps(const fnlh_mesh* m, const SweepOperands& op, const Systems& sys, const T* Bt, T* x0, T* x1,
               int sweeps, int x_zero, int threads, cudaStream_t s, T** result) {
  SweepArgs a;
  a.n = m->n_nodes;
  a.row_ptr = m->row_ptr;
  a.col_idx = m->col_idx;
  a.offd = op.offd;
  a.hess = op.hess;
  a.vol = m->vol;
  a.Bt = Bt;
  a.sys = sys;
  T* cur = x0;
  T* nxt = x1;
  int rc = mark(g_ev_begin, s);
  if (rc) return rc;
  for (int it = 0; it < sweeps; ++it) {
    a.Xin = cur;
    a.Xout = nxt;
    a.x_zero = (it == 0) ? x_zero : 0;
    rc = sweep_launch<BS, TJ, T>(a, threads, s);
    if (rc) return rc;
    T* t = cur;
    cur = nxt;
    nxt = t;
  }
  *result = cur;
  return mark(g_ev_end, s);
}

template <int BS, typename TJ, typename T>
int relax_typed(const fnlh_mesh* m, const fnlh_jacobian* J, int n_harm, const double* omega, const double* B,
                double* X, int sweeps, int precision, void* ws, cudaStream_t s) {
  SweepOperands op;
  int rc = sweep_operands(J, precision, &op);
  if (rc) return rc;
  const Systems sys = make_systems(n_harm, omega);
  const WsLayout W = ws_layout(J->n_nodes, BS, n_harm, precision);
  T* bt = at<T>(ws, W.vec[0]);
  T* x0 = at<T>(ws, W.vec[1]);
  T* x1 = at<T>(ws, W.vec[2]);
  const int n = J->n_nodes;
  if ((rc = rotate_in<BS, T>(n, sys.C, op.rot, B, bt, s))) return rc;
  if ((rc = rotate_in<BS, T>(n, sys.C, op.rot, X, x0, s))) return rc;
  T* res = x0;
  if ((rc = run_sweeps<BS, TJ, T>(m, op, sys, bt, x0, x1, sweeps, 0, 0, s, &res))) return rc;
  return rotate_out<BS, T>(n, sys.C, op.rot, res, X, 0, s);
}

int relax_impl(const fnlh_mesh* m, const fnlh_jacobian* J, int n_harm, const double* omega, const double* B,
               double* X, int sweeps, int precision, void* ws, cudaStream_t s) {
  if (J->block == 5) {
    if (precision == FNLH_F64) return relax_typed<5, double, double>(m, J, n_harm, omega, B, X, sweeps, precision, ws, s);
    if (precision == FNLH_F32) return relax_typed<5, float, float>(m, J, n_harm, omega, B, X, sweeps, precision, ws, s);
    return relax_typed<5, __nv_bfloat16, float>(m, J, n_harm, omega, B, X, sweeps, precision, ws, s);
  }
  if (precision == FNLH_F64) return relax_typed<6, double, double>(m, J, n_harm, omega, B, X, sweeps, precision, ws, s);
  if (precision == FNLH_F32) return relax_typed<6, float, float>(m, J, n_harm, omega, B, X, sweeps, precision, ws, s);
  return relax_typed<6, __nv_bfloat16, float>(m, J, n_harm, omega, B, X, sweeps, precision, ws, s);
}

// ------------------------------------------------------------------ solve

int residual_launch(const fnlh_mesh* m, const fnlh_jacobian* J, const Systems& sys, const double* B,
                    const double* X, double* r, float* r32rot, const double* rot, double* norms, void* ws,
                    cudaStream_t s);

struct Check {
  double rel[kMaxSys];
  double first_max;
};

// Evaluates the residual, copies the norms to the host and classifies them.
static int check_norms(const double* hn, int K, double tol, Check* ck, bool first, bool* converged) {
  double worst = 0.0;
  bool finite = true;
  for (int k = 0; k < K; ++k) {
    const double rr = hn[2 * k], bb = hn[2 * k + 1];
    if (!(rr == rr) || !(bb == bb) || rr > 1e300 || bb > 1e300) finite = false;
    ck->rel[k] = (bb > 0.0) ? sqrt(rr / bb) : sqrt(rr);
    worst = fmax(worst, ck->rel[k]);
  }
  if (!finite) return FNLH_ERR_NONFINITE;
  if (first) ck->first_max = worst;
  else if (worst > 1e3 * fmax(ck->first_max, 1e-300)) return FNLH_ERR_DIVERGED;
  *converged = worst <= tol;
  return FNLH_OK;
}

template <int BS, typename TJ, typename T>
int solve_typed(const fnlh_mesh* m, const fnlh_jacobian* J, int n_harm, const double* omega, const double* B,
                double* X, int precision, double tol, int inner, int max_checks, void* ws, int* checks_done,
                int* sweeps_done, double* rel_res, cudaStream_t s) {
  SweepOperands op;
  int rc = sweep_operands(J, precision, &op);
  if (rc) return rc;
  const Systems sys = make_systems(n_harm, omega);
  const WsLayout W = ws_layout(J->n_nodes, BS, n_harm, precision);
  const int n = J->n_nodes, K = sys.K;
  double* norms = at<double>(ws, W.norms);
  T* v0 = at<T>(ws, W.vec[0]);
  T* v1 = at<T>(ws, W.vec[1]);
  T* v2 = at<T>(ws, W.vec[2]);
  double hn[2 * kMaxSys];
  Check ck;
  int checks = 0, sweeps = 0;
  bool conv = false;
  const bool mixed = precision != FNLH_F64;
  if (!mixed) {
    // plain FP64 Jacobi: iterate in the rotated basis, check every `inner` sweeps
    if ((rc = rotate_in<BS, T>(n, sys.C, op.rot, B, v0, s))) return rc;
    if ((rc = rotate_in<BS, T>(n, sys.C, op.rot, X, v1, s))) return rc;
  }
  T* cur = v1;
  for (;;) {
    rc = residual_launch(m, J, sys, B, X, nullptr, mixed ? (float*)v0 : nullptr, op.rot, norms, ws, s);
    if (rc) return rc;
    FNLH_CUDA_TRY(cudaMemcpyAsync(hn, norms, sizeof(double) * 2 * K, cudaMemcpyDeviceToHost, s));
    FNLH_CUDA_TRY(cudaStreamSynchronize(s));
    rc = check_norms(hn, K, tol, &ck, checks == 0, &conv);
    ++checks;
    if (rc || conv || checks >= max_checks) break;
    T* res = nullptr;
    if (mixed) {
      // inner: A~ e = r~ from e = 0 (v1/v2 ping-pong), then x += Q e in FP64
      if ((rc = run_sweeps<BS, TJ, T>(m, op, sys, v0, v1, v2, inner, 1, 0, s, &res))) return rc;
      if ((rc = rotate_out<BS, T>(n, sys.C, op.rot, res, X, 1, s))) return rc;
    } else {
      T* other = (cur == v1) ? v2 : v1;
      if ((rc = run_sweeps<BS, TJ, T>(m, op, sys, v0, cur, other, inner, 0, 0, s, &res))) return rc;
      cur = res;
      if ((rc = rotate_out<BS, T>(n, sys.C, op.rot, res, X, 0, s))) return rc;
    }
    sweeps += inner;
  }
  if (checks_done) *checks_done = checks;
  if (sweeps_done) *sweeps_done = sweeps;
  if (rel_res)
    for (int k = 0; k < K; ++k) rel_res[k] = ck.rel[k];
  if (rc) return rc;
  return conv ? FNLH_OK : FNLH_ERR_NOT_CONVERGED;
}

int solve_impl(const fnlh_mesh* m, const fnlh_jacobian* J, int n_harm, const double* omega, const double* B,
               double* X, int precision, double tol, int inner, int max_checks, void* ws, int* checks_done,
               int* sweeps_done, double* rel_res, cudaStream_t s) {
#define FNLH_SOLVE(BS, TJ, T) \
  solve_typed<BS, TJ, T>(m, J, n_harm, omega, B, X, precision, tol, inner, max_checks, ws, checks_done, sweeps_done, rel_res, s)
  if (J->block == 5) {
    if (precision == FNLH_F64) return FNLH_SOLVE(5, double, double);
    if (precision == FNLH_F32) return FNLH_SOLVE(5, float, float);
    return FNLH_SOLVE(5, __nv_bfloat16, float);
  }
  if (precision == FNLH_F64) return FNLH_SOLVE(6, double, double);
  if (precision == FNLH_F32) return FNLH_SOLVE(6, float, float);
  return FNLH_SOLVE(6, __nv_bfloat16, float);
#undef FNLH_SOLVE
}

// ----------------------------------------------------------- batched rows
//
// Several blade rows (different meshes, block counts and harmonic counts) in
// one persistent launch per sweep.  The (node, system) pairs of every row are
// cut into tiles of `tile_pairs` consecutive pairs; a grid of
// SMs x ctas_per_sm CTAs walks the global tile list round-robin, so the
// rows' tails share one launch instead of each paying its own.  The row
// descriptors travel as a __grid_constant__ kernel parameter (no device
// memory, capturable in a CUDA graph).

constexpr int kMaxBatchRows = 8;

struct BatchRow {
  int32_t n, K, C, pad;
  long long tile0;  // first global tile of this row
  long long pairs;  // n K
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const void* offd;
  const void* hess;
  const double* vol;
  const void* Bt;
  void* x[2];       // ping-pong iterate buffers
  double omega[kMaxSys];
};

struct BatchArgs {
  int32_t n_rows, parity, x_zero, tile_pairs;
  long long n_tiles;
  BatchRow row[kMaxBatchRows];
};

template <int BS, typename TJ, typename T>
__global__ void __launch_bounds__(256) k_sweep_batched(const __grid_constant__ BatchArgs a) {
  for (long long t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
    int r = 0;
    while (r + 1 < a.n_rows && t >= a.row[r + 1].tile0) ++r;
    const BatchRow& R = a.row[r];
    const long long first = (t - R.tile0) * a.tile_pairs;
    for (int q = threadIdx.x; q < a.tile_pairs; q += blockDim.x) {
      const long long g = first + q;
      if (g >= R.pairs) break;
      const int i = (int)(g / R.K);
      const int k = (int)(g - (long long)i * R.K);
      sweep_pair<BS, TJ, T>(R.row_ptr, R.col_idx, (const TJ*)R.offd, (const T*)R.hess, R.vol, (const T*)R.Bt,
                            (const T*)R.x[a.parity], (T*)R.x[a.parity ^ 1], R.C, i, k, R.omega[k], a.x_zero != 0);
    }
  }
}

size_t batched_extra_bytes(int n_rows) { return n_rows > 0 ? 256 : 0; }

template <int BS, typename TJ, typename T>
int batched_typed(const fnlh_row* rows, int n_rows, int sweeps, int precision, const fnlh_tuning* tn, void* ws,
                  cudaStream_t s) {
  static thread_local BatchArgs a;  // large: kept off the stack (the launch copies it)
  std::memset(&a, 0, sizeof(a));
  int threads = (tn && tn->threads > 0) ? tn->threads : 256;
  int ctas_per_sm = (tn && tn->ctas_per_sm > 0) ? tn->ctas_per_sm : 4;
  int tile_pairs = (tn && tn->nodes_per_tile > 0) ? tn->nodes_per_tile : threads;
  if (threads > 256 || threads % 32) return FNLH_ERR_ARG;
  int dev = 0, sms = 0;
  FNLH_CUDA_TRY(cudaGetDevice(&dev));
  FNLH_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  size_t off = 256;
  long long tiles = 0;
  a.n_rows = n_rows;
  a.tile_pairs = tile_pairs;
  SweepOperands ops[kMaxBatchRows];
  for (int r = 0; r < n_rows; ++r) {
    const fnlh_row& R = rows[r];
    int rc = sweep_operands(R.J, precision, &ops[r]);
    if (rc) return rc;
    const Systems sys = make_systems(R.n_harm, R.omega);
    const WsLayout W = ws_layout(R.mesh->n_nodes, BS, R.n_harm, precision);
    char* base = (char*)ws + off;
    off += W.total;
    BatchRow& D = a.row[r];
    D.n = R.mesh->n_nodes;
    D.K = sys.K;
    D.C = sys.C;
    D.pairs = (long long)D.n * D.K;
    D.tile0 = tiles;
    tiles += (D.pairs + tile_pairs - 1) / tile_pairs;
    D.row_ptr = R.mesh->row_ptr;
    D.col_idx = R.mesh->col_idx;
    D.offd = ops[r].offd;
    D.hess = ops[r].hess;
    D.vol = R.mesh->vol;
    D.Bt = base + W.vec[0];
    D.x[0] = base + W.vec[1];
    D.x[1] = base + W.vec[2];
    for (int k = 0; k < kMaxSys; ++k) D.omega[k] = sys.omega[k];
    if ((rc = rotate_in<BS, T>(D.n, D.C, ops[r].rot, R.B, (T*)D.Bt, s))) return rc;
    if ((rc = rotate_in<BS, T>(D.n, D.C, ops[r].rot, R.X, (T*)D.x[0], s))) return rc;
  }
  a.n_tiles = tiles;
  const long long grid_ll = std::min<long long>(tiles, (long long)sms * ctas_per_sm);
  const unsigned grid = (unsigned)std::max<long long>(grid_ll, 1);
  {
    int rc = mark(g_ev_begin, s);
    if (rc) return rc;
  }
  for (int it = 0; it < sweeps; ++it) {
    a.parity = it & 1;
    a.x_zero = 0;
    if (tiles > 0) {
      k_sweep_batched<BS, TJ, T><<<grid, threads, 0, s>>>(a);
      FNLH_LAUNCH_CHECK();
    }
  }
  {
    int rc = mark(g_ev_end, s);
    if (rc) return rc;
  }
  const int fin = sweeps & 1;
  for (int r = 0; r < n_rows; ++r) {
    const BatchRow& D = a.row[r];
    int rc = rotate_out<BS, T>(D.n, D.C, ops[r].rot, (const T*)D.x[fin], rows[r].X, 0, s);
    if (rc) return rc;
  }
  return FNLH_OK;
}

int batched_impl(const fnlh_row* rows, int n_rows, int sweeps, int precision, const fnlh_tuning* tn, void* ws,
                 size_t ws_bytes, cudaStream_t s) {
  (void)ws_bytes;
  if (n_rows > kMaxBatchRows) return FNLH_ERR_UNSUPPORTED;
  const int b = rows[0].J->block;
  for (int r = 1; r < n_rows; ++r)
    if (rows[r].J->block != b) return FNLH_ERR_UNSUPPORTED;
  if (b == 5) {
    if (precision == FNLH_F64) return batched_typed<5, double, double>(rows, n_rows, sweeps, precision, tn, ws, s);
    if (precision == FNLH_F32) return batched_typed<5, float, float>(rows, n_rows, sweeps, precision, tn, ws, s);
    return batched_typed<5, __nv_bfloat16, float>(rows, n_rows, sweeps, precision, tn, ws, s);
  }
  if (precision == FNLH_F64) return batched_typed<6, double, double>(rows, n_rows, sweeps, precision, tn, ws, s);
  if (precision == FNLH_F32) return batched_typed<6, float, float>(rows, n_rows, sweeps, precision, tn, ws, s);
  return batched_typed<6, __nv_bfloat16, float>(rows, n_rows, sweeps, precision, tn, ws, s);
}

}  // namespace fnlh
