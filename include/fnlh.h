/*
 * fnlh.h -- C ABI of the GB300 (sm_103a) shared-Jacobian FNLH linear solver.
 *
 * Paper: X. Wang, L. di Mare et al., "Convergence Acceleration of
 * Favre-Averaged Non-Linear Harmonic Method", arXiv 2404.01407.
 *
 * The library relaxes, all at once, the sparse linear systems formed in one
 * implicit RK stage by the mean flow and by every time-linearised harmonic
 * (Eq. lhs_mean and Eq. lhs_lin, with the implicit left-hand side of
 * Eq. precon / Eq. precon_linear):
 *
 *     A_k x_k = B_k,   A_k = J + D I + i omega_k V I,   k = 0..N
 *
 * J = dR/dQ is the first-order approximate residual Jacobian assembled from
 * immediate neighbours ("Generalized RK Scheme for The Mean Flow"), D the
 * scalar pseudo-time diagonal V_i/dt_i, V the control volume, omega_0 = 0 the
 * mean flow.  One J and one D serve the mean flow and all harmonics, so no
 * allocation here grows with N ("Solution Update": the LHS memory of all
 * harmonics is shared).  The Gamma*alpha_k factor of Eq. lhs_mean is the
 * caller's: scale B by Gamma*alpha_k to obtain the paper's update.
 *
 * Conventions
 * -----------
 *  - Every array argument is DEVICE memory owned by the caller unless the
 *    comment says "host".  The library allocates no device memory: scratch
 *    space is the caller's `workspace` (size from fnlh_workspace_bytes) and
 *    derived Jacobian data is the caller's `prep` blob (size from
 *    fnlh_prep_bytes).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    asynchronous on it, except the ones documented as synchronising.
 *  - Vectors X, B, r use the real layout [n][C][b], C = 1 + 2N: column 0 is
 *    the mean flow, columns 2l-1 and 2l are Re and Im of harmonic l, whose
 *    angular frequency is omega[l-1] (the +i omega sign of Eq. phi_fft).
 *  - Phase-lagged periodic boundaries (Eq. lhs_lin; the inter-blade phase
 *    angle makes each harmonic's LHS different without changing its
 *    sparsity): on a mesh with `periodic` edges, harmonic l couples node i to
 *    the image of node j in the neighbouring blade passage, so its
 *    off-diagonal term is J_ij e^{i s sigma[l-1]} x_j, s = +1 (next passage)
 *    or -1 (previous) as seen from node i.  sigma (HOST [n_harm], radians,
 *    nullable = all 0, i.e. plain periodicity) sits beside omega in every
 *    call; J and its memory stay shared.  The mean flow carries no phase.
 *  - Blocks are row-major b x b, b = 5 (Euler) or 6 (Euler + one turbulence
 *    equation).  Off-diagonal blocks are stored in CSR order [nnz][b][b];
 *    within a row the neighbours are sorted ascending.
 *  - Return value: FNLH_OK (0) or a negative FNLH_ERR_* code; arguments are
 *    validated on the host before anything is launched, and nothing is
 *    launched when validation fails.
 */
#ifndef FNLH_H
#define FNLH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void *fnlh_stream_t; /* a cudaStream_t */

enum fnlh_status {
    FNLH_OK = 0,
    FNLH_ERR_ARG = -1,           /* invalid argument (null pointer, size, range) */
    FNLH_ERR_CUDA = -2,          /* a CUDA runtime call or kernel launch failed */
    FNLH_ERR_NONFINITE = -3,     /* a residual norm is NaN or Inf */
    FNLH_ERR_DIVERGED = -4,      /* residual grew by more than 1e3 over its start */
    FNLH_ERR_TIMEOUT = -5,       /* reserved: a bounded device wait gave up (no kernel here waits) */
    FNLH_ERR_UNSUPPORTED = -6,   /* block size not 5 or 6, too many harmonics */
    FNLH_ERR_WORKSPACE = -7,     /* workspace or prep blob too small / missing */
    FNLH_ERR_NOT_CONVERGED = -8, /* iteration limit reached above tolerance */
    FNLH_ERR_BAD_MESH = -9       /* self loop, duplicate edge, node out of range */
};

/* Precision of a relaxation (storage of the off-diagonal blocks / iterate). */
enum fnlh_precision {
    FNLH_F64 = 0,  /* FP64 blocks, FP64 iterate and arithmetic */
    FNLH_F32 = 1,  /* FP32 blocks, FP32 iterate and arithmetic */
    FNLH_BF16 = 2  /* BF16 blocks, FP32 iterate and arithmetic */
};

/* Which derived off-diagonal copies fnlh_prepare writes (bit mask). */
enum fnlh_prep_flags {
    FNLH_PREP_F64 = 1,
    FNLH_PREP_F32 = 2,
    FNLH_PREP_BF16 = 4,
    /* a copy of col_idx whose top three bits tag each entry: the passage
     * offset of a periodic edge, and whether it crosses a partition; required
     * by every call on a mesh with `periodic` or `part` */
    FNLH_PREP_TAGS = 8,
    /* float-float copies (each FP64 entry as an FP32 pair hi + lo, |entry - hi - lo| <= 2^-48 |entry|) of
     * the off-diagonal blocks and of J_ii + D_i I in the original basis: with them, and the workspace of
     * fnlh_solve_workspace_bytes, the intermediate residual checks of a mixed-precision fnlh_solve run on
     * the FP32 units (see fnlh_solve; likewise fnlh_solve_batched and the FP32 fnlh_solve_ilu) */
    FNLH_PREP_FF = 16
};

#define FNLH_MAX_HARMONICS 64

/* Edge-based node-centred mesh (paper, "Brief Description of Hydra": an
 * edge data structure with dual-face normals).  Device arrays. */
typedef struct fnlh_mesh {
    int32_t n_nodes;
    int32_t n_edges;
    const int32_t *edge_nodes; /* [E][2] node pair (i, j) of each edge */
    const double *normals;     /* [E][3] dual-face normal n_ij, pointing from i to j */
    const double *vol;         /* [n] control volume V_i (spectral term i omega V) */
    const int32_t *row_ptr;    /* [n+1] CSR of the symmetric neighbour graph */
    const int32_t *col_idx;    /* [2E] neighbour of each CSR entry, ascending per row */
    const int32_t *csr_edge;   /* [2E] edge of each CSR entry */
    /* [E] nullable: passage of node j of the edge as seen from node i across a
     * periodic boundary: +1 the next passage, -1 the previous, 0 none (an
     * ordinary edge); other values count by their sign.  The normal of such
     * an edge points to the image of j.  Needs a prep blob with
     * FNLH_PREP_TAGS.  (Every mesh needs n_nodes < 2^29.) */
    const int8_t *periodic;
    /* [n] nullable: partition of each node -- the domain decomposition of a
     * parallel run.  As in the paper's decomposition (Implementation: the
     * entries that couple nodes of different partitions are ignored), the
     * sweeps drop every coupling between partitions, so each partition
     * relaxes on its own, while the residual keeps them all; fnlh_solve then
     * corrects the truncated sweeps with the full residual at every
     * precision.  Needs FNLH_PREP_TAGS. */
    const int32_t *part;
} fnlh_mesh;

/* Jacobian construction parameters. */
typedef struct fnlh_params {
    double gamma;         /* ratio of specific heats (1.4) */
    double cfl;           /* pseudo-time CFL number sigma_CFL */
    double entropy_delta; /* entropy fix: f(l) = max(|l|, delta (|u_n| + a|n|)); 0.1 */
    int32_t pseudo_time;  /* 0: scalar D_i = V_i/dt_i; 1: block P/(eps sigma_CFL) of Eq. precon */
    double eps;           /* relaxation factor eps of Eq. precon (0.6) */
} fnlh_params;

/* The shared operator.  offd/diag/D are written by fnlh_build_jacobian or
 * supplied by the caller; prep is the caller-allocated derived blob
 * (fnlh_prep_bytes) that fnlh_prepare fills with per-node Hessenberg factors
 * and the off-diagonal copies named by prep_flags. */
typedef struct fnlh_jacobian {
    int32_t n_nodes;
    int32_t nnz;       /* = 2 E */
    int32_t block;     /* b: 5 or 6 */
    double *offd;      /* [nnz][b][b] J_ij */
    double *diag;      /* [n][b][b]   J_ii */
    double *D;         /* [n]         pseudo-time diagonal */
    void *prep;        /* derived data, fnlh_prep_bytes(n, nnz, b, prep_flags) bytes */
    size_t prep_bytes;
    int32_t prep_flags; /* FNLH_PREP_* mask */
    int32_t prep_ready; /* set to 1 by fnlh_prepare, 0 by fnlh_build_jacobian */
} fnlh_jacobian;

/* One blade row of a batched relaxation (fnlh_relax_batched). */
typedef struct fnlh_row {
    const fnlh_mesh *mesh;
    const fnlh_jacobian *J;
    int32_t n_harm;
    const double *omega; /* host [n_harm] */
    const double *B;     /* [n][C][b] right-hand sides */
    double *X;           /* [n][C][b] in: x0, out: x */
    const double *sigma; /* host [n_harm] inter-blade phase angles, or NULL */
} fnlh_row;

/* Launch shape of the batched sweep kernel (0 = library default). */
typedef struct fnlh_tuning {
    int32_t threads;      /* threads per CTA = (node, system) pairs per tile; 32..256, multiple of 32 */
    int32_t ctas_per_sm;  /* 0: one CTA per tile; > 0: persistent grid of SMs x this CTAs;
                             FNLH_TUNING_PER_ROW: every row its own single-row launches (threads unused) */
    int32_t reserved[2];
} fnlh_tuning;

/* fnlh_tuning.ctas_per_sm: rows large enough to fill the GPU on their own
 * gain nothing from sharing a launch, and the single-row kernels are the
 * faster ones for them (the FP64 one solves the mean flow on a real-only
 * path); the autotuner weighs this mode against the shared launches. */
#define FNLH_TUNING_PER_ROW (-1)

/* Human-readable text of a status code (static storage). */
const char *fnlh_strerror(int status);

/* Library version as 10000*major + 100*minor + patch. */
int fnlh_version(void);

/* HOST helper: CSR of the neighbour graph from an edge list.
 * edge_nodes (host [E][2]); outputs (host) row_ptr [n+1], col_idx [2E],
 * csr_edge [2E], neighbours ascending within each row.  Rejects self loops,
 * duplicate edges and out-of-range nodes with FNLH_ERR_BAD_MESH. */
int fnlh_mesh_build_csr(int32_t n_nodes, int32_t n_edges, const int32_t *edge_nodes,
                        int32_t *row_ptr, int32_t *col_idx, int32_t *csr_edge);

/* Bytes of the derived blob for fnlh_prepare. */
size_t fnlh_prep_bytes(int32_t n_nodes, int32_t nnz, int32_t block, int32_t prep_flags);

/* Bytes of scratch space the calls below need for this problem size when
 * they run at `precision` (FNLH_F64 gives the largest size, enough for any
 * precision; fnlh_residual alone needs the FNLH_F32 size).  0 on bad input. */
size_t fnlh_workspace_bytes(int32_t n_nodes, int32_t block, int32_t n_harm, int32_t precision);

/* Assemble J (off-diagonal and diagonal blocks) and D from the conservative
 * state Q [n][b] (rho, rho u, rho v, rho w, rho E[, rho nu]) -- the
 * first-order, immediate-neighbour residual Jacobian of Eq. precon:
 *   J_ij = 1/2 (A(Q_j, n_ij) - |A|(Qbar_ij, n_ij))
 *   J_ii = 1/2 sum_j |A|(Qbar_ij, n_ij) + 1/2 |A|(Q_i, n_b),  n_b = -sum_j n_ij
 *   D_i  = (sum_j lambda(Qbar_ij, n_ij) + lambda(Q_i, n_b)) / CFL
 * A = d(F.n)/dQ of the Euler flux (six equations: frozen turbulence row
 * advected at u_n, its J_ii entry doubled), |A| its matrix absolute value with
 * the entropy fix, lambda = |u_n| + a|n|, Qbar the arithmetic mean.  With
 * params->pseudo_time = 1, D = 0 and J_ii is scaled by 1 + 1/(eps CFL).
 * Then, if J->prep is set, runs fnlh_prepare.  Asynchronous. */
int fnlh_build_jacobian(const fnlh_mesh *mesh, const double *Q, const fnlh_params *params,
                        fnlh_jacobian *J, fnlh_stream_t stream);

/* Derived data for the sweeps: per node an orthogonal Q_i with
 * Q_i^T (J_ii + D_i I) Q_i upper Hessenberg, and the off-diagonal blocks
 * rotated into that basis, Q_i^T J_ij Q_j, in the precisions of prep_flags.
 * With b = 6 and frozen turbulence (column 5 zero in rows 0..4 of J_ii: the
 * mean-flow equations do not see the turbulence variable) Q_i keeps that
 * structure, and when every block has it the FP64 sweeps and the residual
 * skip the structural zeros (fnlh_prep_structured tells);
 * with FNLH_PREP_TAGS the tagged column copy (from the mesh's periodic flags
 * and partition; FNLH_ERR_WORKSPACE when the mesh has either and the flag is
 * missing).  Depends only on J, D and the mesh, so it is
 * independent of the number of harmonics and of their phase angles.
 * Call after changing offd/diag/D yourself.  Asynchronous. */
int fnlh_prepare(const fnlh_mesh *mesh, fnlh_jacobian *J, fnlh_stream_t stream);

/* `sweeps` undamped block-Jacobi sweeps ("Solution Update": block-diagonal
 * inversion point by point) on every system at once:
 *   x_i <- (J_ii + (D_i + i omega_k V_i) I)^-1 (B_i - sum_j J_ij x_j)
 * omega: HOST [n_harm]; sigma: HOST [n_harm] phase angles or NULL (see
 * Conventions).  B, X: FP64 [n][C][b]; X holds x0 on entry, the
 * result on return.  precision selects the block copy and arithmetic of the
 * sweeps (FNLH_F64 needs FNLH_PREP_F64, etc.).  Asynchronous. */
int fnlh_relax(const fnlh_mesh *mesh, const fnlh_jacobian *J, int32_t n_harm, const double *omega,
               const double *sigma, const double *B, double *X, int32_t sweeps, int32_t precision,
               void *workspace, size_t workspace_bytes, fnlh_stream_t stream);

/* FP64 linear residual r_k = B_k - A_k x_k (the quantity of the paper's
 * linear-solve stopping rule, Results / Table fnlh_para) and, per system k,
 * norms[2k] = ||r_k||_2^2, norms[2k+1] = ||B_k||_2^2 (complex 2-norm over all
 * n b entries).  r (nullable) [n][C][b]; norms [2K] device.  The sums are
 * reduced in a fixed order, so repeated calls give identical bits.
 * Asynchronous. */
int fnlh_residual(const fnlh_mesh *mesh, const fnlh_jacobian *J, int32_t n_harm,
                  const double *omega, const double *sigma, const double *B, const double *X,
                  double *r, double *norms, void *workspace, size_t workspace_bytes,
                  fnlh_stream_t stream);

/* fnlh_solve flags */
#define FNLH_SOLVE_ZERO_GUESS 1     /* start from x0 = 0 (X is overwritten; the first residual is B) */
#define FNLH_SOLVE_MASK_CONVERGED 2 /* systems already at tol are not swept again (their x is kept) */

/* Workspace bytes of fnlh_solve: fnlh_workspace_bytes, plus for FNLH_F32 /
 * FNLH_BF16 with FNLH_PREP_FF in prep_flags the float-float shadows of B and
 * x ([n][C][b] FP32 pairs each) that its float-float checks read.  0 for an
 * unsupported block size, harmonic count or precision. */
size_t fnlh_solve_workspace_bytes(int32_t n_nodes, int32_t block, int32_t n_harm, int32_t precision,
                                  int32_t prep_flags);

/* Solve every system to ||r_k|| <= tol ||B_k||.  With x0 = 0 and tol = 1e-2 this is
 * the paper's linear-solve rule (Results, Table fnlh_para: the residual drops
 * two orders of magnitude from its initial value; max_checks and inner_sweeps
 * bound the iterations).  precision FNLH_F64: plain FP64
 * Jacobi with an FP64 residual check every `inner_sweeps` sweeps.
 * FNLH_F32 / FNLH_BF16: defect correction -- FP64 residual r = B - A x,
 * `inner_sweeps` sweeps on A e = r with the low-precision blocks and FP32
 * arithmetic from e = 0 (r and e rotated in FP32), then x += e with the sum in
 * FP64; repeated.  Float-float checks: when J's prep blob holds FNLH_PREP_FF
 * and the workspace has fnlh_solve_workspace_bytes, every check of a mixed
 * solve after the first evaluates B - A x in float-float arithmetic on the
 * FP32 units (about 44 bits: its norms agree with the FP64 residual's to
 * ~1e-5 relative at a 1e-8 residual) -- except that a check is always made,
 * or confirmed, with the FP64 residual before the solve reports convergence:
 * a float-float check at tol is followed at once by an FP64 one, and when the
 * residual's decay (the last two checks' ratio) predicts the next check at
 * or below 2 tol, the next check is FP64 directly.  On a mesh with
 * `periodic` the float-float residual applies the phase factor of Eq.
 * lhs_lin to the product of each periodic entry (FNLH_PREP_TAGS as usual).
 * On a mesh with `part` the FP64 solve is a defect
 * correction too (inner FP64 sweeps without the cross-partition couplings,
 * FP64 residual with them).  X: in x0 (ignored with FNLH_SOLVE_ZERO_GUESS), out x.
 * SYNCHRONISING (reads the norms after every check).  Outputs (host, each
 * nullable): *checks_done residual checks (a float-float check and the FP64
 * residual that confirms it count as one), *sweeps_done total sweeps,
 * rel_res [K] final ||r_k||/||B_k||.  Returns FNLH_ERR_NOT_CONVERGED after
 * max_checks checks above tol, FNLH_ERR_NONFINITE / FNLH_ERR_DIVERGED on a
 * non-finite or growing (x1e3) residual. */
int fnlh_solve(const fnlh_mesh *mesh, const fnlh_jacobian *J, int32_t n_harm, const double *omega,
               const double *sigma, const double *B, double *X, int32_t precision, double tol,
               int32_t inner_sweeps,
               int32_t max_checks, int32_t flags, void *workspace, size_t workspace_bytes,
               int32_t *checks_done, int32_t *sweeps_done, double *rel_res, fnlh_stream_t stream);

/* Batched form: `sweeps` sweeps of fnlh_relax on several blade rows of
 * different sizes and harmonic counts (the multi-row FNLH setting of the
 * paper's Results) with one kernel launch per sweep over a tile list
 * spanning every row (one CTA per tile, or a persistent grid) -- two when
 * FP32/BF16 rows that stage their blocks in shared memory (K >= 6 systems)
 * are mixed with rows that do not.  At most 8
 * rows, all with the same block size.  tuning may be NULL (defaults).  workspace: at
 * least the sum of fnlh_workspace_bytes of the rows plus
 * fnlh_batched_extra_bytes(n_rows).  Asynchronous, graph-capturable. */
int fnlh_relax_batched(const fnlh_row *rows, int32_t n_rows, int32_t sweeps, int32_t precision,
                       const fnlh_tuning *tuning, void *workspace, size_t workspace_bytes,
                       fnlh_stream_t stream);

size_t fnlh_batched_extra_bytes(int32_t n_rows);

/* Batched fnlh_solve: every system of every row to ||r|| <= tol ||B||, all
 * rows checked together.  FNLH_F64: plain Jacobi with the FP64 residual of
 * every row every `inner_sweeps` sweeps (rows with `part` are rejected with
 * FNLH_ERR_UNSUPPORTED: use a low precision).  FNLH_F32 / FNLH_BF16: defect
 * correction -- FP64 residual of every row, then `inner_sweeps` batched
 * launches over all rows from e = 0, then x += Q e per row.  flags, outputs
 * and errors as fnlh_solve; rel_res (host, nullable) holds the rows' systems
 * one row after the other.  workspace as fnlh_relax_batched, with each row's
 * fnlh_workspace_bytes taken at `precision`.  When every row's prep blob has
 * FNLH_PREP_FF and the workspace holds the sum of
 * the rows' fnlh_solve_workspace_bytes plus fnlh_batched_extra_bytes, the
 * intermediate checks of a mixed solve run in float-float as in fnlh_solve
 * (the check that ends the solve is FP64).  SYNCHRONISING. */
int fnlh_solve_batched(const fnlh_row *rows, int32_t n_rows, int32_t precision, double tol,
                       int32_t inner_sweeps, int32_t max_checks, int32_t flags, const fnlh_tuning *tuning,
                       void *workspace, size_t workspace_bytes, int32_t *checks_done, int32_t *sweeps_done,
                       double *rel_res, fnlh_stream_t stream);

/* Allocation-free variant of fnlh_residual (the paper has no counterpart).
 *
 * Same arguments, results and fixed-order sums as fnlh_residual, minus the
 * workspace: the per-block partial sums live in a device array built into
 * the library (1,264,640 bytes on every device that loads it, kept until the
 * process exits), which covers every valid harmonic count.  It is meant for
 * callers that cannot allocate device memory -- for instance a host code
 * whose memory pool owns the whole device budget, or a caller inside a CUDA
 * stream capture, where cudaMalloc is not allowed -- and therefore cannot
 * provide the workspace fnlh_residual needs.  The call allocates nothing.
 * Every call looks up the array's address in the current context (a lookup
 * that allocates nothing); the first call on a device may also load the
 * library's device code there, so make that first call before any stream
 * capture.  All
 * calls share the one array: calls that may run at the same time on the GPU
 * (other streams or host threads) race on it and must be serialised by the
 * caller.  A problem too large for the array (impossible for
 * n_harm <= FNLH_MAX_HARMONICS) returns FNLH_ERR_UNSUPPORTED. */
int fnlh_residual_noalloc(const fnlh_mesh *mesh, const fnlh_jacobian *J, int32_t n_harm,
                          const double *omega, const double *sigma, const double *B,
                          const double *X, double *r, double *norms, fnlh_stream_t stream);

/* ------------------------------------------------------------------ ILU(0)
 *
 * The paper's implicit smoother ("Generalized RK Scheme": the LHS of every
 * stage is inverted approximately by ILU(0) iterations, each partition of a
 * parallel run factored on its own).  Here block ILU(0) in multicolour order:
 * the nodes are grouped by colour (no two neighbours share one), so each
 * triangular solve is a sequence of parallel colour passes.  On a pattern
 * without triangles (three pairwise adjacent nodes; hexahedral edge graphs
 * have none) elimination changes only the pivot blocks,
 *     P_i = A_ii - sum_{j of an earlier colour} A_ij P_j^-1 A_ji,
 * with L_ij = A_ij P_j^-1 and U_ij = A_ij, so the factor is one inverse pivot
 * block per node and system and J supplies every off-diagonal block.  A_ij
 * carries the phase-lag factor on periodic entries (the pivots do not depend
 * on it: an edge's two couplings carry opposite phases) and is dropped
 * between partitions (`part`). */

/* HOST helper: greedy colouring of the neighbour graph in node order (each
 * node takes the smallest colour none of its earlier neighbours has), and the
 * nodes grouped by colour: order[color_ptr[c] .. color_ptr[c+1]) are the nodes
 * of colour c, ascending.  row_ptr/col_idx: host CSR (untagged); color, order
 * [n]; color_ptr [max_colors + 1].  FNLH_ERR_UNSUPPORTED if more than
 * max_colors colours are needed. */
int fnlh_mesh_color(int32_t n_nodes, const int32_t *row_ptr, const int32_t *col_idx, int32_t max_colors,
                    int32_t *color, int32_t *order, int32_t *color_ptr, int32_t *n_colors);

typedef struct fnlh_ilu {
    int32_t n_colors;
    const int32_t *color;     /* [n] device: colour of every node */
    const int32_t *order;     /* [n] device: nodes grouped by colour, colour 0 first */
    const int32_t *color_ptr; /* HOST [n_colors + 1]: order[color_ptr[c] .. color_ptr[c+1]) have colour c */
    void *factor;             /* device, fnlh_ilu_bytes(n, b, n_harm, precision) bytes */
    size_t factor_bytes;
    int32_t precision;        /* FNLH_F64: FP64 factor and passes on J's FP64 blocks.  FNLH_F32:
                                 FP32 factor and passes in the per-node Schur basis of the sweeps
                                 on the prep blob's FP32 blocks (needs FNLH_PREP_F32; the same
                                 smoother, ILU(0) being invariant under that change of basis),
                                 pivots formed in FP64 from the stored FP32 inverses of earlier
                                 colours, FP64 residual and x += Q e with the sum in FP64 */
    int32_t n_harm;           /* systems the factor holds (set by fnlh_ilu_factor) */
    int32_t ready;            /* set to 1 by fnlh_ilu_factor */
} fnlh_ilu;

/* Bytes of the factor: n (1 + n_harm) b^2 complex values of the precision. */
size_t fnlh_ilu_bytes(int32_t n_nodes, int32_t block, int32_t n_harm, int32_t precision);

/* Factor every system (omega: HOST [n_harm]) into ilu->factor.  Uses J's FP64
 * blocks in the original basis (no prep needed, except FNLH_PREP_TAGS on a
 * mesh with periodic edges or partitions).  SYNCHRONISING: first checks on the
 * device that neighbours have different colours and `order` groups every node
 * once by colour (FNLH_ERR_BAD_MESH), and that the pattern, without the
 * couplings between partitions, has no triangle (FNLH_ERR_UNSUPPORTED: block
 * ILU(0) would then need off-diagonal factors); FNLH_ERR_NONFINITE on a
 * singular pivot.  workspace: fnlh_workspace_bytes(n, b, n_harm, FNLH_F64). */
int fnlh_ilu_factor(const fnlh_mesh *mesh, const fnlh_jacobian *J, int32_t n_harm, const double *omega,
                    fnlh_ilu *ilu, void *workspace, size_t workspace_bytes, fnlh_stream_t stream);

/* ILU(0) iterations x <- x + (L U)^-1 (B - A x) on every system with the
 * factor of fnlh_ilu_factor (same n_harm and omega); the FP64 residual keeps
 * every coupling.  Before each iteration ||B_k - A_k x_k|| <= tol ||B_k|| for
 * all k ends the solve (with x0 = 0 and tol = 1e-2, max_iterations = 10: the
 * paper's rule).  flags: FNLH_SOLVE_ZERO_GUESS, FNLH_SOLVE_MASK_CONVERGED.
 * SYNCHRONISING.  Outputs (host, nullable): *iterations_done, rel_res [K].
 * Returns FNLH_ERR_NOT_CONVERGED after max_iterations, FNLH_ERR_NONFINITE /
 * FNLH_ERR_DIVERGED as fnlh_solve.  workspace: the FNLH_F64 size.  With an
 * FP32 factor and FNLH_PREP_FF in J's prep, the residual
 * of every iteration after the first is taken in float-float as in
 * fnlh_solve, and the one that ends the solve in FP64. */
int fnlh_solve_ilu(const fnlh_mesh *mesh, const fnlh_jacobian *J, const fnlh_ilu *ilu, int32_t n_harm,
                   const double *omega, const double *sigma, const double *B, double *X, double tol,
                   int32_t max_iterations, int32_t flags, void *workspace, size_t workspace_bytes,
                   int32_t *iterations_done, double *rel_res, fnlh_stream_t stream);

/* Whether fnlh_prepare certified the b = 6 frozen-turbulence zero pattern
 * (every block, diagonal and off-diagonal, has column 5 zero in rows 0..4):
 * *structured = 1 or 0.  FNLH_ERR_WORKSPACE without a prepared blob.
 * SYNCHRONISING (reads one word of the blob). */
int fnlh_prep_structured(const fnlh_jacobian *J, int32_t *structured, fnlh_stream_t stream);

/* Timing hook (not part of the paper): when both are non-NULL, every later
 * relaxation on this host thread records `begin` on its stream right before
 * its first sweep launch and `end` right after its last one (fnlh_solve_ilu:
 * around the colour passes of each iteration, so the pair brackets the last
 * one), so that the caller can time the sweep launches alone.  Events are cudaEvent_t created
 * by the caller; pass NULL, NULL to switch the hook off. */
int fnlh_set_sweep_events(void *begin, void *end);

#ifdef __cplusplus
}
#endif

#endif /* FNLH_H */
