// C ABI of the FNLH library: argument validation and dispatch.
// Every entry point validates on the host and launches nothing on failure.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace fnlh {
int build_jacobian_impl(const fnlh_mesh*, const double*, const fnlh_params*, fnlh_jacobian*, cudaStream_t);
int prepare_impl(const fnlh_mesh*, fnlh_jacobian*, cudaStream_t);
int relax_impl(const fnlh_mesh*, const fnlh_jacobian*, int, const double*, const double*, const double*, double*,
               int, int, void*, cudaStream_t);
int solve_impl(const fnlh_mesh*, const fnlh_jacobian*, int, const double*, const double*, const double*, double*, int,
               double, int, int, int, void*, size_t, int*, int*, double*, cudaStream_t);
int residual_launch(const fnlh_mesh*, const fnlh_jacobian*, const Systems&, const double*, const double*, double*,
                    float*, const float*, int, double*, void*, cudaStream_t);
Systems make_systems(int n_harm, const double* omega, const double* sigma);
int batched_impl(const fnlh_row*, int, int, int, const fnlh_tuning*, void*, size_t, cudaStream_t);
int solve_batched_impl(const fnlh_row*, int, int, double, int, int, int, const fnlh_tuning*, void*, size_t, int*, int*,
                       double*, cudaStream_t);
size_t batched_extra_bytes(int n_rows);
void set_sweep_events(cudaEvent_t b, cudaEvent_t e);
int residual_noalloc_launch(const fnlh_mesh*, const fnlh_jacobian*, const Systems&, const double*, const double*,
                            double*, double*, cudaStream_t);
int ilu_factor_impl(const fnlh_mesh*, const fnlh_jacobian*, int, const double*, fnlh_ilu*, void*, cudaStream_t);
int solve_ilu_impl(const fnlh_mesh*, const fnlh_jacobian*, const fnlh_ilu*, int, const double*, const double*,
                   const double*, double*, double, int, int, void*, int*, double*, cudaStream_t);
}  // namespace fnlh

using namespace fnlh;

namespace {

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

int check_mesh(const fnlh_mesh* m, bool need_edges) {
  if (!m) return FNLH_ERR_ARG;
  if (m->n_nodes < 0 || m->n_edges < 0) return FNLH_ERR_ARG;
  if (m->n_nodes > 0 && (!m->row_ptr || !m->vol)) return FNLH_ERR_ARG;
  if (m->n_edges > 0 && !m->col_idx) return FNLH_ERR_ARG;
  if (need_edges && m->n_edges > 0 && (!m->csr_edge || !m->edge_nodes || !m->normals)) return FNLH_ERR_ARG;
  // node ids must leave the top three bits free: the kernels read them as the
  // tags of periodic edges and partition cuts
  if (m->n_nodes > (int32_t)kColMask) return FNLH_ERR_UNSUPPORTED;
  return FNLH_OK;
}

// A mesh with periodic edges or partitions is only read through the prep
// blob's tagged column copy.
int check_tags(const fnlh_mesh* m, const fnlh_jacobian* J) {
  if (!tagged_mesh(m)) return FNLH_OK;
  if (!J->prep || !J->prep_ready || !(J->prep_flags & FNLH_PREP_TAGS)) return FNLH_ERR_WORKSPACE;
  if (!aligned(J->prep, 256)) return FNLH_ERR_ARG;
  if (J->prep_bytes < fnlh_prep_bytes(J->n_nodes, J->nnz, J->block, J->prep_flags)) return FNLH_ERR_WORKSPACE;
  return FNLH_OK;
}

int check_jac(const fnlh_mesh* m, const fnlh_jacobian* J) {
  if (!J) return FNLH_ERR_ARG;
  if (J->block != 5 && J->block != 6) return FNLH_ERR_UNSUPPORTED;
  if (J->n_nodes != m->n_nodes || J->nnz != 2 * m->n_edges) return FNLH_ERR_ARG;
  if (J->n_nodes > 0 && (!J->diag || !J->D)) return FNLH_ERR_ARG;
  if (J->nnz > 0 && !J->offd) return FNLH_ERR_ARG;
  if (!aligned(J->offd, 16) || !aligned(J->diag, 16) || !aligned(J->D, 8)) return FNLH_ERR_ARG;
  return FNLH_OK;
}

int check_prep(const fnlh_jacobian* J, int precision) {
  if (!J->prep || !J->prep_ready) return FNLH_ERR_WORKSPACE;
  if (!aligned(J->prep, 256)) return FNLH_ERR_ARG;
  if (J->prep_bytes < fnlh_prep_bytes(J->n_nodes, J->nnz, J->block, J->prep_flags)) return FNLH_ERR_WORKSPACE;
  const int need = precision == FNLH_F64 ? FNLH_PREP_F64 : precision == FNLH_F32 ? FNLH_PREP_F32 : FNLH_PREP_BF16;
  if (!(J->prep_flags & need)) return FNLH_ERR_WORKSPACE;
  return FNLH_OK;
}

int check_systems(int n_harm, const double* omega, const double* sigma) {
  if (n_harm < 0) return FNLH_ERR_ARG;
  if (n_harm > FNLH_MAX_HARMONICS) return FNLH_ERR_UNSUPPORTED;
  if (n_harm > 0 && !omega) return FNLH_ERR_ARG;
  for (int k = 0; k < n_harm; ++k)
    if (!std::isfinite(omega[k]) || (sigma && !std::isfinite(sigma[k]))) return FNLH_ERR_ARG;
  return FNLH_OK;
}

int check_ws(void* ws, size_t bytes, int n, int b, int n_harm, int precision) {
  if (!ws) return FNLH_ERR_WORKSPACE;
  if (!aligned(ws, 256)) return FNLH_ERR_ARG;
  if (bytes < ws_layout(n, b, n_harm, precision).total) return FNLH_ERR_WORKSPACE;
  return FNLH_OK;
}

bool valid_precision(int p) { return p == FNLH_F64 || p == FNLH_F32 || p == FNLH_BF16; }

// The sweep kernels index (node, system) pairs with 32-bit arithmetic.
int check_pairs(int n_nodes, int n_harm) {
  return ((long long)n_nodes * (1 + n_harm) < (1LL << 31)) ? FNLH_OK : FNLH_ERR_UNSUPPORTED;
}

}  // namespace

// Named NVTX range over one entry point, so that a profiler's timeline (or
// ncu --nvtx-include) shows each library call as one span.  NVTX is
// header-only: without an attached tool a push/pop is a few instructions.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

#define FNLH_TRY(expr)       \
  do {                       \
    int _rc = (expr);        \
    if (_rc) return _rc;     \
  } while (0)

extern "C" {

const char* fnlh_strerror(int status) {
  switch (status) {
    case FNLH_OK: return "success";
    case FNLH_ERR_ARG: return "invalid argument";
    case FNLH_ERR_CUDA: return "CUDA runtime error";
    case FNLH_ERR_NONFINITE: return "non-finite residual";
    case FNLH_ERR_DIVERGED: return "residual diverged";
    case FNLH_ERR_TIMEOUT: return "bounded device wait timed out";
    case FNLH_ERR_UNSUPPORTED: return "unsupported block size or harmonic count";
    case FNLH_ERR_WORKSPACE: return "workspace or prep blob missing or too small";
    case FNLH_ERR_NOT_CONVERGED: return "tolerance not reached within the iteration limit";
    case FNLH_ERR_BAD_MESH: return "bad mesh (self loop, duplicate edge or node out of range)";
    default: return "unknown status";
  }
}

int fnlh_version(void) { return 100; }

int fnlh_mesh_build_csr(int32_t n_nodes, int32_t n_edges, const int32_t* edge_nodes, int32_t* row_ptr,
                        int32_t* col_idx, int32_t* csr_edge) {
  if (n_nodes < 0 || n_edges < 0 || !row_ptr) return FNLH_ERR_ARG;
  if (n_edges > 0 && (!edge_nodes || !col_idx || !csr_edge)) return FNLH_ERR_ARG;
  if ((long long)2 * n_edges > 0x7fffffffLL) return FNLH_ERR_UNSUPPORTED;
  std::vector<int32_t> deg((size_t)n_nodes + 1, 0);
  for (int32_t e = 0; e < n_edges; ++e) {
    const int32_t a = edge_nodes[2 * e], c = edge_nodes[2 * e + 1];
    if (a < 0 || c < 0 || a >= n_nodes || c >= n_nodes || a == c) return FNLH_ERR_BAD_MESH;
    deg[a + 1]++;
    deg[c + 1]++;
  }
  row_ptr[0] = 0;
  for (int32_t i = 0; i < n_nodes; ++i) row_ptr[i + 1] = row_ptr[i] + deg[i + 1];
  std::vector<int32_t> fill((size_t)n_nodes, 0);
  for (int32_t e = 0; e < n_edges; ++e) {
    const int32_t a = edge_nodes[2 * e], c = edge_nodes[2 * e + 1];
    int32_t pa = row_ptr[a] + fill[a]++, pc = row_ptr[c] + fill[c]++;
    col_idx[pa] = c;
    csr_edge[pa] = e;
    col_idx[pc] = a;
    csr_edge[pc] = e;
  }
  std::vector<std::pair<int32_t, int32_t>> tmp;
  for (int32_t i = 0; i < n_nodes; ++i) {
    const int32_t p0 = row_ptr[i], p1 = row_ptr[i + 1];
    tmp.clear();
    for (int32_t p = p0; p < p1; ++p) tmp.emplace_back(col_idx[p], csr_edge[p]);
    std::sort(tmp.begin(), tmp.end());
    for (int32_t p = p0; p < p1; ++p) {
      col_idx[p] = tmp[p - p0].first;
      csr_edge[p] = tmp[p - p0].second;
      if (p > p0 && col_idx[p] == col_idx[p - 1]) return FNLH_ERR_BAD_MESH;
    }
  }
  return FNLH_OK;
}

size_t fnlh_prep_bytes(int32_t n_nodes, int32_t nnz, int32_t block, int32_t prep_flags) {
  if (n_nodes < 0 || nnz < 0 || (block != 5 && block != 6)) return 0;
  return prep_layout(n_nodes, nnz, block, prep_flags).total;
}

size_t fnlh_solve_workspace_bytes(int32_t n_nodes, int32_t block, int32_t n_harm, int32_t precision,
                                  int32_t prep_flags) {
  const size_t base = fnlh_workspace_bytes(n_nodes, block, n_harm, precision);
  if (base == 0 || precision == FNLH_F64 || !(prep_flags & FNLH_PREP_FF)) return base;
  return ws_layout(n_nodes, block, n_harm, precision).total_ff;
}

size_t fnlh_workspace_bytes(int32_t n_nodes, int32_t block, int32_t n_harm, int32_t precision) {
  if (n_nodes < 0 || (block != 5 && block != 6) || n_harm < 0 || n_harm > FNLH_MAX_HARMONICS) return 0;
  if (!valid_precision(precision)) return 0;
  return ws_layout(n_nodes, block, n_harm, precision).total;
}

int fnlh_build_jacobian(const fnlh_mesh* mesh, const double* Q, const fnlh_params* params, fnlh_jacobian* J,
                        fnlh_stream_t stream) {
  NvtxRange range_("fnlh_build_jacobian");
  FNLH_TRY(check_mesh(mesh, true));
  FNLH_TRY(check_jac(mesh, J));
  if (!params || (mesh->n_nodes > 0 && !Q)) return FNLH_ERR_ARG;
  if (!(params->cfl > 0.0) || !(params->gamma > 1.0) || !(params->entropy_delta >= 0.0)) return FNLH_ERR_ARG;
  if (params->pseudo_time != 0 && params->pseudo_time != 1) return FNLH_ERR_ARG;
  if (params->pseudo_time == 1 && !(params->eps > 0.0)) return FNLH_ERR_ARG;
  J->prep_ready = 0;
  cudaStream_t s = (cudaStream_t)stream;
  FNLH_TRY(build_jacobian_impl(mesh, Q, params, J, s));
  if (J->prep) return fnlh_prepare(mesh, J, stream);
  return FNLH_OK;
}

int fnlh_prepare(const fnlh_mesh* mesh, fnlh_jacobian* J, fnlh_stream_t stream) {
  NvtxRange range_("fnlh_prepare");
  FNLH_TRY(check_mesh(mesh, false));
  FNLH_TRY(check_jac(mesh, J));
  if (!J->prep) return FNLH_ERR_WORKSPACE;
  if (!aligned(J->prep, 256)) return FNLH_ERR_ARG;
  if (J->prep_flags & ~(FNLH_PREP_F64 | FNLH_PREP_F32 | FNLH_PREP_BF16 | FNLH_PREP_TAGS | FNLH_PREP_FF))
    return FNLH_ERR_ARG;
  if (J->prep_bytes < fnlh_prep_bytes(J->n_nodes, J->nnz, J->block, J->prep_flags)) return FNLH_ERR_WORKSPACE;
  if (tagged_mesh(mesh) && !(J->prep_flags & FNLH_PREP_TAGS)) return FNLH_ERR_WORKSPACE;
  if (mesh->periodic) FNLH_TRY(check_mesh(mesh, true));  // passage tags come from csr_edge and edge_nodes
  FNLH_TRY(prepare_impl(mesh, J, (cudaStream_t)stream));
  J->prep_ready = 1;
  return FNLH_OK;
}

int fnlh_relax(const fnlh_mesh* mesh, const fnlh_jacobian* J, int32_t n_harm, const double* omega,
               const double* sigma, const double* B, double* X, int32_t sweeps, int32_t precision, void* workspace,
               size_t workspace_bytes, fnlh_stream_t stream) {
  NvtxRange range_("fnlh_relax");
  FNLH_TRY(check_mesh(mesh, false));
  FNLH_TRY(check_jac(mesh, J));
  if (!valid_precision(precision) || sweeps < 0) return FNLH_ERR_ARG;
  FNLH_TRY(check_systems(n_harm, omega, sigma));
  FNLH_TRY(check_prep(J, precision));
  FNLH_TRY(check_tags(mesh, J));
  if (mesh->n_nodes > 0 && (!B || !X)) return FNLH_ERR_ARG;
  FNLH_TRY(check_ws(workspace, workspace_bytes, mesh->n_nodes, J->block, n_harm, precision));
  FNLH_TRY(check_pairs(mesh->n_nodes, n_harm));
  return relax_impl(mesh, J, n_harm, omega, sigma, B, X, sweeps, precision, workspace, (cudaStream_t)stream);
}

int fnlh_residual(const fnlh_mesh* mesh, const fnlh_jacobian* J, int32_t n_harm, const double* omega,
                  const double* sigma, const double* B, const double* X, double* r, double* norms, void* workspace,
                  size_t workspace_bytes, fnlh_stream_t stream) {
  NvtxRange range_("fnlh_residual");
  FNLH_TRY(check_mesh(mesh, false));
  FNLH_TRY(check_jac(mesh, J));
  FNLH_TRY(check_systems(n_harm, omega, sigma));
  FNLH_TRY(check_tags(mesh, J));
  if (!norms || (mesh->n_nodes > 0 && (!B || !X))) return FNLH_ERR_ARG;
  if (!workspace) return FNLH_ERR_WORKSPACE;
  if (!aligned(workspace, 256)) return FNLH_ERR_ARG;
  const WsLayout W = ws_layout(mesh->n_nodes, J->block, n_harm, FNLH_F64);
  if (workspace_bytes < W.vec[0]) return FNLH_ERR_WORKSPACE;  // partials only
  const Systems sys = make_systems(n_harm, omega, sigma);
  return residual_launch(mesh, J, sys, B, X, r, nullptr, nullptr, 0, norms, workspace, (cudaStream_t)stream);
}

int fnlh_solve(const fnlh_mesh* mesh, const fnlh_jacobian* J, int32_t n_harm, const double* omega,
               const double* sigma, const double* B, double* X, int32_t precision, double tol, int32_t inner_sweeps,
               int32_t max_checks, int32_t flags, void* workspace, size_t workspace_bytes, int32_t* checks_done,
               int32_t* sweeps_done, double* rel_res, fnlh_stream_t stream) {
  NvtxRange range_("fnlh_solve");
  FNLH_TRY(check_mesh(mesh, false));
  FNLH_TRY(check_jac(mesh, J));
  if (!valid_precision(precision) || !(tol >= 0.0) || inner_sweeps < 1 || max_checks < 1) return FNLH_ERR_ARG;
  if (flags & ~(FNLH_SOLVE_ZERO_GUESS | FNLH_SOLVE_MASK_CONVERGED)) return FNLH_ERR_ARG;
  FNLH_TRY(check_systems(n_harm, omega, sigma));
  FNLH_TRY(check_prep(J, precision));
  FNLH_TRY(check_tags(mesh, J));
  if (mesh->n_nodes > 0 && (!B || !X)) return FNLH_ERR_ARG;
  FNLH_TRY(check_ws(workspace, workspace_bytes, mesh->n_nodes, J->block, n_harm, precision));
  FNLH_TRY(check_pairs(mesh->n_nodes, n_harm));
  return solve_impl(mesh, J, n_harm, omega, sigma, B, X, precision, tol, inner_sweeps, max_checks, flags, workspace,
                    workspace_bytes, checks_done, sweeps_done, rel_res, (cudaStream_t)stream);
}

size_t fnlh_batched_extra_bytes(int32_t n_rows) { return n_rows > 0 ? batched_extra_bytes(n_rows) : 0; }

int fnlh_relax_batched(const fnlh_row* rows, int32_t n_rows, int32_t sweeps, int32_t precision,
                       const fnlh_tuning* tuning, void* workspace, size_t workspace_bytes, fnlh_stream_t stream) {
  NvtxRange range_("fnlh_relax_batched");
  if (!rows || n_rows < 1 || sweeps < 0 || !valid_precision(precision)) return FNLH_ERR_ARG;
  size_t need = batched_extra_bytes(n_rows);
  for (int r = 0; r < n_rows; ++r) {
    const fnlh_row& R = rows[r];
    FNLH_TRY(check_mesh(R.mesh, false));
    FNLH_TRY(check_jac(R.mesh, R.J));
    FNLH_TRY(check_systems(R.n_harm, R.omega, R.sigma));
    FNLH_TRY(check_prep(R.J, precision));
    FNLH_TRY(check_tags(R.mesh, R.J));
    if (R.mesh->n_nodes > 0 && (!R.B || !R.X)) return FNLH_ERR_ARG;
    FNLH_TRY(check_pairs(R.mesh->n_nodes, R.n_harm));
    need += ws_layout(R.mesh->n_nodes, R.J->block, R.n_harm, precision).total;
  }
  if (!workspace) return FNLH_ERR_WORKSPACE;
  if (!aligned(workspace, 256)) return FNLH_ERR_ARG;
  if (workspace_bytes < need) return FNLH_ERR_WORKSPACE;
  return batched_impl(rows, n_rows, sweeps, precision, tuning, workspace, workspace_bytes, (cudaStream_t)stream);
}

int fnlh_solve_batched(const fnlh_row* rows, int32_t n_rows, int32_t precision, double tol, int32_t inner_sweeps,
                       int32_t max_checks, int32_t flags, const fnlh_tuning* tuning, void* workspace,
                       size_t workspace_bytes, int32_t* checks_done, int32_t* sweeps_done, double* rel_res,
                       fnlh_stream_t stream) {
  NvtxRange range_("fnlh_solve_batched");
  if (!rows || n_rows < 1 || !valid_precision(precision)) return FNLH_ERR_ARG;
  if (!(tol >= 0.0) || inner_sweeps < 1 || max_checks < 1) return FNLH_ERR_ARG;
  if (flags & ~(FNLH_SOLVE_ZERO_GUESS | FNLH_SOLVE_MASK_CONVERGED)) return FNLH_ERR_ARG;
  size_t need = batched_extra_bytes(n_rows);
  for (int r = 0; r < n_rows; ++r) {
    const fnlh_row& R = rows[r];
    FNLH_TRY(check_mesh(R.mesh, false));
    FNLH_TRY(check_jac(R.mesh, R.J));
    FNLH_TRY(check_systems(R.n_harm, R.omega, R.sigma));
    FNLH_TRY(check_prep(R.J, precision));
    FNLH_TRY(check_tags(R.mesh, R.J));
    // plain FP64 Jacobi on the truncated sweeps would not reach the full system's solution
    if (precision == FNLH_F64 && R.mesh->part) return FNLH_ERR_UNSUPPORTED;
    if (R.mesh->n_nodes > 0 && (!R.B || !R.X)) return FNLH_ERR_ARG;
    FNLH_TRY(check_pairs(R.mesh->n_nodes, R.n_harm));
    need += ws_layout(R.mesh->n_nodes, R.J->block, R.n_harm, precision).total;
  }
  if (!workspace) return FNLH_ERR_WORKSPACE;
  if (!aligned(workspace, 256)) return FNLH_ERR_ARG;
  if (workspace_bytes < need) return FNLH_ERR_WORKSPACE;
  return solve_batched_impl(rows, n_rows, precision, tol, inner_sweeps, max_checks, flags, tuning, workspace,
                            workspace_bytes, checks_done, sweeps_done, rel_res, (cudaStream_t)stream);
}

int fnlh_residual_noalloc(const fnlh_mesh* mesh, const fnlh_jacobian* J, int32_t n_harm, const double* omega,
                          const double* sigma, const double* B, const double* X, double* r, double* norms,
                          fnlh_stream_t stream) {
  NvtxRange range_("fnlh_residual_noalloc");
  FNLH_TRY(check_mesh(mesh, false));
  FNLH_TRY(check_jac(mesh, J));
  FNLH_TRY(check_systems(n_harm, omega, sigma));
  FNLH_TRY(check_tags(mesh, J));
  if (!norms || (mesh->n_nodes > 0 && (!B || !X))) return FNLH_ERR_ARG;
  const Systems sys = make_systems(n_harm, omega, sigma);
  return residual_noalloc_launch(mesh, J, sys, B, X, r, norms, (cudaStream_t)stream);
}

int fnlh_mesh_color(int32_t n_nodes, const int32_t* row_ptr, const int32_t* col_idx, int32_t max_colors,
                    int32_t* color, int32_t* order, int32_t* color_ptr, int32_t* n_colors) {
  if (n_nodes < 0 || max_colors < 1 || !row_ptr || !color || !order || !color_ptr || !n_colors) return FNLH_ERR_ARG;
  if (n_nodes > 0 && row_ptr[n_nodes] > 0 && !col_idx) return FNLH_ERR_ARG;
  std::vector<int32_t> used((size_t)max_colors + 1, -1);
  int32_t top = 0;
  for (int32_t i = 0; i < n_nodes; ++i) {
    for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
      const int32_t j = col_idx[p];
      if (j < 0 || j >= n_nodes) return FNLH_ERR_BAD_MESH;
      if (j < i && color[j] < max_colors) used[color[j]] = i;
    }
    int32_t c = 0;
    while (c < max_colors && used[c] == i) ++c;
    if (c >= max_colors) return FNLH_ERR_UNSUPPORTED;
    color[i] = c;
    top = std::max(top, c + 1);
  }
  *n_colors = top;
  for (int32_t c = 0; c <= top; ++c) color_ptr[c] = 0;
  for (int32_t i = 0; i < n_nodes; ++i) color_ptr[color[i] + 1]++;
  for (int32_t c = 0; c < top; ++c) color_ptr[c + 1] += color_ptr[c];
  std::vector<int32_t> fill(color_ptr, color_ptr + top + 1);
  for (int32_t i = 0; i < n_nodes; ++i) order[fill[color[i]]++] = i;
  return FNLH_OK;
}

size_t fnlh_ilu_bytes(int32_t n_nodes, int32_t block, int32_t n_harm, int32_t precision) {
  if (n_nodes < 0 || (block != 5 && block != 6) || n_harm < 0 || n_harm > FNLH_MAX_HARMONICS) return 0;
  if (precision != FNLH_F64 && precision != FNLH_F32) return 0;
  const size_t elem = precision == FNLH_F64 ? 8 : 4;
  return (size_t)n_nodes * (1 + (size_t)n_harm) * block * block * 2 * elem;
}

static int check_ilu(const fnlh_mesh* mesh, const fnlh_jacobian* J, const fnlh_ilu* ilu, int n_harm) {
  if (!ilu) return FNLH_ERR_ARG;
  if (ilu->precision != FNLH_F64 && ilu->precision != FNLH_F32) return FNLH_ERR_ARG;
  if (ilu->n_colors < 1 && mesh->n_nodes > 0) return FNLH_ERR_ARG;
  if (mesh->n_nodes > 0 && (!ilu->color || !ilu->order || !ilu->color_ptr || !ilu->factor)) return FNLH_ERR_ARG;
  if (!aligned(ilu->factor, 16)) return FNLH_ERR_ARG;
  if (ilu->factor_bytes < fnlh_ilu_bytes(mesh->n_nodes, J->block, n_harm, ilu->precision)) return FNLH_ERR_WORKSPACE;
  for (int c = 0; c < ilu->n_colors; ++c)
    if (ilu->color_ptr[c] > ilu->color_ptr[c + 1]) return FNLH_ERR_ARG;
  if (mesh->n_nodes > 0 && (ilu->color_ptr[0] != 0 || ilu->color_ptr[ilu->n_colors] != mesh->n_nodes))
    return FNLH_ERR_ARG;
  return FNLH_OK;
}

int fnlh_ilu_factor(const fnlh_mesh* mesh, const fnlh_jacobian* J, int32_t n_harm, const double* omega, fnlh_ilu* ilu,
                    void* workspace, size_t workspace_bytes, fnlh_stream_t stream) {
  NvtxRange range_("fnlh_ilu_factor");
  FNLH_TRY(check_mesh(mesh, false));
  FNLH_TRY(check_jac(mesh, J));
  FNLH_TRY(check_systems(n_harm, omega, nullptr));
  FNLH_TRY(check_tags(mesh, J));
  FNLH_TRY(check_ilu(mesh, J, ilu, n_harm));
  if (ilu->precision == FNLH_F32) FNLH_TRY(check_prep(J, FNLH_F32));  // rotated FP32 blocks
  FNLH_TRY(check_ws(workspace, workspace_bytes, mesh->n_nodes, J->block, n_harm, FNLH_F64));
  FNLH_TRY(check_pairs(mesh->n_nodes, n_harm));
  ilu->ready = 0;
  if (mesh->n_nodes == 0) {
    ilu->n_harm = n_harm;
    ilu->ready = 1;
    return FNLH_OK;
  }
  return ilu_factor_impl(mesh, J, n_harm, omega, ilu, workspace, (cudaStream_t)stream);
}

int fnlh_solve_ilu(const fnlh_mesh* mesh, const fnlh_jacobian* J, const fnlh_ilu* ilu, int32_t n_harm,
                   const double* omega, const double* sigma, const double* B, double* X, double tol,
                   int32_t max_iterations, int32_t flags, void* workspace, size_t workspace_bytes,
                   int32_t* iterations_done, double* rel_res, fnlh_stream_t stream) {
  NvtxRange range_("fnlh_solve_ilu");
  FNLH_TRY(check_mesh(mesh, false));
  FNLH_TRY(check_jac(mesh, J));
  FNLH_TRY(check_systems(n_harm, omega, sigma));
  FNLH_TRY(check_tags(mesh, J));
  FNLH_TRY(check_ilu(mesh, J, ilu, n_harm));
  if (!ilu->ready || ilu->n_harm != n_harm) return FNLH_ERR_WORKSPACE;
  if (ilu->precision == FNLH_F32) FNLH_TRY(check_prep(J, FNLH_F32));
  if (!(tol >= 0.0) || max_iterations < 0) return FNLH_ERR_ARG;
  if (flags & ~(FNLH_SOLVE_ZERO_GUESS | FNLH_SOLVE_MASK_CONVERGED)) return FNLH_ERR_ARG;
  if (mesh->n_nodes > 0 && (!B || !X)) return FNLH_ERR_ARG;
  FNLH_TRY(check_ws(workspace, workspace_bytes, mesh->n_nodes, J->block, n_harm, FNLH_F64));
  FNLH_TRY(check_pairs(mesh->n_nodes, n_harm));
  return solve_ilu_impl(mesh, J, ilu, n_harm, omega, sigma, B, X, tol, max_iterations, flags, workspace,
                        iterations_done, rel_res, (cudaStream_t)stream);
}

int fnlh_prep_structured(const fnlh_jacobian* J, int32_t* structured, fnlh_stream_t stream) {
  if (!J || !structured) return FNLH_ERR_ARG;
  *structured = 0;
  const int32_t* info = prep_info(J);
  if (!info) return FNLH_ERR_WORKSPACE;
  if (J->block != 6) return FNLH_OK;
  int32_t h = 1;
  cudaStream_t s = (cudaStream_t)stream;
  FNLH_CUDA_TRY(cudaMemcpyAsync(&h, info, sizeof(h), cudaMemcpyDeviceToHost, s));
  FNLH_CUDA_TRY(cudaStreamSynchronize(s));
  *structured = (h == 0) ? 1 : 0;
  return FNLH_OK;
}

int fnlh_set_sweep_events(void* begin, void* end) {
  if ((begin == nullptr) != (end == nullptr)) return FNLH_ERR_ARG;
  set_sweep_events((cudaEvent_t)begin, (cudaEvent_t)end);
  return FNLH_OK;
}

}  // extern "C"
