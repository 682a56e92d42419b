/*
 * CPU FP64 oracle for the shared-Jacobian FNLH linear systems.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * CUDA library is checked against.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the library never calls it
 * and shares no code, header or table with it.
 *
 * What it computes (paper: arXiv 2404.01407, "Convergence Acceleration of
 * Favre-Averaged Non-Linear Harmonic Method"):
 *
 *  - The implicit left-hand side of the generalised RK scheme,
 *    K = P/(eps*sigma) + J  (Eq. precon), with J = dR/dQ the first-order
 *    approximate residual Jacobian built from immediate neighbours
 *    ("Generalized RK Scheme for The Mean Flow").  The paper does not print
 *    the first-order flux it linearises; this oracle uses a first-order
 *    upwind (matrix-dissipation) edge flux
 *        F_ij = 1/2 (F(Q_i) + F(Q_j)) . n_ij - 1/2 |A|(Qbar_ij, n_ij) (Q_j - Q_i)
 *    with |A| frozen, and a far-field closure face n_b = -sum_j n_ij per node,
 *    so that
 *        J_ij = 1/2 (A(Q_j, n_ij) - |A|(Qbar_ij, n_ij))
 *        J_ii = sum_j 1/2 (A(Q_i, n_ij) + |A|(Qbar_ij, n_ij))
 *               + 1/2 (A(Q_i, n_b) + |A|(Q_i, n_b)).
 *    A(Q, n) is d(F(Q).n)/dQ, evaluated here by complex-step
 *    differentiation of the flux itself (no hand-derived matrix).
 *    |A| is the matrix absolute value by Sylvester's formula over the three
 *    distinct eigenvalues u_n, u_n +- a|n|, with the entropy fix
 *    f(lambda) = max(|lambda|, delta (|u_n| + a|n|)).  With six equations the
 *    turbulence row is frozen (Hydra linearises with frozen turbulence) and
 *    its dissipation is the scalar f(u_n); the (6,6) diagonal entry of J_ii
 *    is doubled (turbulence-row dominance of the synthetic cases).
 *  - The scalar pseudo-time diagonal D_i = V_i / dt_i with the local time
 *    step dt_i = CFL V_i / (sum_j lambda_ij + lambda_b), lambda = |u_n| + a|n|.
 *    Alternatively (pseudo_block != 0) Eq. precon's block form: no D, and
 *    J_ii scaled by (1 + 1/(eps CFL)).
 *  - The systems of Eq. lhs_mean / Eq. lhs_lin (the Gamma*alpha_k factor is
 *    left to the caller): A_k = J + D I + i omega_k V I (Eq. precon_linear),
 *    omega_0 = 0 for the mean flow; solved by undamped block Jacobi, which the
 *    paper names for the block-diagonal inversion of the explicit scheme
 *    ("Solution Update"):
 *        x_i <- (J_ii + (D_i + i omega_k V_i) I)^-1 (B_i - sum_j J_ij x_j)
 *    every block solved by LU with partial pivoting.
 *  - The linear residual r_k = B_k - A_k x_k and its 2-norm, the quantity
 *    whose drop the paper's linear-solve stopping rule tests (Results,
 *    Table fnlh_para).
 *  - Phase-lagged periodic boundaries (Eq. lhs_lin and the text around
 *    Eq. precon_linear: the inter-blade phase angle changes each harmonic's
 *    LHS but not its sparsity).  A periodic edge joins node i to the image of
 *    node j in the neighbouring blade passage; the harmonic-l perturbation of
 *    that image is e^{i s sigma_l} x_j, s = +1 (next passage) or -1
 *    (previous).  So the off-diagonal term of harmonic l across such an edge
 *    is J_ij e^{i s sigma_l} x_j: J itself is unchanged and shared, the mean
 *    flow (plain periodicity) carries no phase.
 *  - Domain-truncated block Jacobi (Implementation, parallel decomposition:
 *    the entries that couple two nodes of different partitions are ignored,
 *    so that each partition's sub-system is solved on its own): with a
 *    partition id per node, the sweep drops J_ij x_j whenever i and j lie in
 *    different partitions.  The residual always keeps every coupling.
 *
 * Layout: X, B, r are real [n][C][b], C = 1 + 2N; column 0 is the mean flow,
 * columns 2l-1 / 2l are Re / Im of harmonic l (omega[l-1]).  Off-diagonal
 * blocks are stored row-major [nnz][b][b] in CSR order with neighbours sorted
 * ascending.
 *
 * Compile: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (no FMA
 * contraction, so every product and sum is rounded separately).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXB 6

typedef double complex cplx;

/* ---------------------------------------------------------------- flux */

/* Euler flux through the (unnormalised) face normal n; with six equations
 * the sixth conserved variable is advected, F_6 = Q_6 u_n. */
static void flux_dot_n(int b, const cplx *q, const double *n, double gamma, cplx *f)
{
    cplx rho = q[0];
    cplx u = q[1] / rho, v = q[2] / rho, w = q[3] / rho;
    cplx p = (gamma - 1.0) * (q[4] - 0.5 * (q[1] * u + q[2] * v + q[3] * w));
    cplx un = u * n[0] + v * n[1] + w * n[2];
    f[0] = q[0] * un;
    f[1] = q[1] * un + p * n[0];
    f[2] = q[2] * un + p * n[1];
    f[3] = q[3] * un + p * n[2];
    f[4] = (q[4] + p) * un;
    if (b == 6) f[5] = q[5] * un;
}

/* A(Q, n) = d(F(Q).n)/dQ by complex-step differentiation: column k is
 * Im(F(Q + i h e_k)) / h, exact to rounding for this rational flux. */
void oracle_flux_jacobian(int b, const double *q, const double *n, double gamma, double *A)
{
    const double h = 1e-30;
    for (int k = 0; k < b; k++) {
        cplx qc[MAXB], f[MAXB];
        for (int m = 0; m < b; m++) qc[m] = q[m];
        qc[k] += I * h;
        flux_dot_n(b, qc, n, gamma, f);
        for (int r = 0; r < b; r++) A[r * b + k] = cimag(f[r]) / h;
    }
    if (b == 6) {
        /* frozen turbulence: the mean-flow rows do not depend on Q_6 */
        for (int r = 0; r < 5; r++) A[r * b + 5] = 0.0;
    }
}

/* spectral radius |u_n| + a |n| */
double oracle_spectral_radius(const double *q, const double *n, double gamma)
{
    double rho = q[0], u = q[1] / rho, v = q[2] / rho, w = q[3] / rho;
    double p = (gamma - 1.0) * (q[4] - 0.5 * rho * (u * u + v * v + w * w));
    double a = sqrt(gamma * p / rho);
    double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    double un = u * n[0] + v * n[1] + w * n[2];
    return fabs(un) + a * nn;
}

/* |A|(Q, n) by Sylvester's formula on the 5x5 Euler block:
 *   |A| = sum_k f(l_k) prod_{m != k} (A - l_m I) / (l_k - l_m)
 * over the distinct eigenvalues l = (u_n, u_n + a|n|, u_n - a|n|).
 * Six equations: block diagonal with the scalar f(u_n) for the sixth row. */
void oracle_abs_jacobian(int b, const double *q, const double *n, double gamma, double delta, double *absA)
{
    memset(absA, 0, sizeof(double) * b * b);
    double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (nn == 0.0) return; /* zero face: A = 0, all eigenvalues 0 */
    double A[MAXB * MAXB];
    oracle_flux_jacobian(b, q, n, gamma, A);
    double rho = q[0], u = q[1] / rho, v = q[2] / rho, w = q[3] / rho;
    double p = (gamma - 1.0) * (q[4] - 0.5 * rho * (u * u + v * v + w * w));
    double a = sqrt(gamma * p / rho);
    double un = u * n[0] + v * n[1] + w * n[2];
    double lam[3] = {un, un + a * nn, un - a * nn};
    double fix = delta * (fabs(un) + a * nn);
    double f[3];
    for (int k = 0; k < 3; k++) f[k] = fabs(lam[k]) > fix ? fabs(lam[k]) : fix;

    for (int k = 0; k < 3; k++) {
        double M[25], T[25];
        for (int r = 0; r < 5; r++)
            for (int c = 0; c < 5; c++) M[r * 5 + c] = (r == c) ? 1.0 : 0.0;
        for (int m = 0; m < 3; m++) {
            if (m == k) continue;
            double s = 1.0 / (lam[k] - lam[m]);
            /* T = M (A - l_m I) s */
            for (int r = 0; r < 5; r++)
                for (int c = 0; c < 5; c++) {
                    double acc = 0.0;
                    for (int t = 0; t < 5; t++) {
                        double am = A[t * b + c] - ((t == c) ? lam[m] : 0.0);
                        acc += M[r * 5 + t] * am;
                    }
                    T[r * 5 + c] = acc * s;
                }
            memcpy(M, T, sizeof(M));
        }
        for (int r = 0; r < 5; r++)
            for (int c = 0; c < 5; c++) absA[r * b + c] += f[k] * M[r * 5 + c];
    }
    if (b == 6) absA[5 * b + 5] = f[0];
}

/* ---------------------------------------------------------------- mesh */

typedef struct {
    int j;
    int e;
    int sgn;
} nbr_t;

static int cmp_nbr(const void *a, const void *b)
{
    const nbr_t *x = (const nbr_t *)a, *y = (const nbr_t *)b;
    return (x->j > y->j) - (x->j < y->j);
}

/* neighbour lists from the edge list, sorted ascending; returns 0 or -1 on a
 * bad edge (self loop, out of range, duplicate). */
static int make_neighbours(int n, int E, const int32_t *edge_nodes, int32_t *row_ptr, nbr_t **out)
{
    for (int i = 0; i <= n; i++) row_ptr[i] = 0;
    for (int e = 0; e < E; e++) {
        int a = edge_nodes[2 * e], c = edge_nodes[2 * e + 1];
        if (a < 0 || c < 0 || a >= n || c >= n || a == c) return -1;
        row_ptr[a + 1]++;
        row_ptr[c + 1]++;
    }
    for (int i = 0; i < n; i++) row_ptr[i + 1] += row_ptr[i];
    nbr_t *nb = (nbr_t *)malloc(sizeof(nbr_t) * (size_t)(2 * (size_t)E + 1));
    int *fill = (int *)calloc((size_t)n + 1, sizeof(int));
    for (int e = 0; e < E; e++) {
        int a = edge_nodes[2 * e], c = edge_nodes[2 * e + 1];
        nb[row_ptr[a] + fill[a]++] = (nbr_t){c, e, +1};
        nb[row_ptr[c] + fill[c]++] = (nbr_t){a, e, -1};
    }
    free(fill);
    int bad = 0;
    for (int i = 0; i < n; i++) {
        qsort(nb + row_ptr[i], (size_t)(row_ptr[i + 1] - row_ptr[i]), sizeof(nbr_t), cmp_nbr);
        for (int p = row_ptr[i] + 1; p < row_ptr[i + 1]; p++)
            if (nb[p].j == nb[p - 1].j) bad = 1;
    }
    if (bad) {
        free(nb);
        return -1;
    }
    *out = nb;
    return 0;
}

/* Passage offset of the neighbour of every CSR entry (same order as the
 * col_idx that oracle_build_jacobian writes).  periodic[e] in {-1, 0, +1} is
 * the passage of the edge's second node as seen from its first; seen from
 * the second node the offset is the opposite. */
int oracle_phase_sides(int n, int E, const int32_t *edge_nodes, const int8_t *periodic, int32_t *row_ptr,
                       int8_t *side)
{
    nbr_t *nb = NULL;
    if (make_neighbours(n, E, edge_nodes, row_ptr, &nb) != 0) return -2;
    for (int p = 0; p < 2 * E; p++) side[p] = (int8_t)(nb[p].sgn * periodic[nb[p].e]);
    free(nb);
    return 0;
}

/* ------------------------------------------------------- Jacobian build */

int oracle_build_jacobian(int n, int E, int b, const int32_t *edge_nodes, const double *normals,
                          const double *Q, double gamma, double delta, double cfl,
                          int pseudo_block, double eps, int32_t *row_ptr, int32_t *col_idx,
                          double *offd, double *diag, double *D)
{
    if (b != 5 && b != 6) return -1;
    nbr_t *nb = NULL;
    if (make_neighbours(n, E, edge_nodes, row_ptr, &nb) != 0) return -2;
    const int bb = b * b;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        const double *qi = Q + (size_t)i * b;
        double *Pi = diag + (size_t)i * bb;
        double nbnd[3] = {0.0, 0.0, 0.0};
        double lsum = 0.0;
        double Ai[MAXB * MAXB], Aj[MAXB * MAXB], Ab[MAXB * MAXB];
        for (int t = 0; t < bb; t++) Pi[t] = 0.0;
        for (int p = row_ptr[i]; p < row_ptr[i + 1]; p++) {
            int j = nb[p].j, e = nb[p].e;
            col_idx[p] = j;
            double nij[3];
            for (int d = 0; d < 3; d++) nij[d] = nb[p].sgn * normals[3 * e + d];
            for (int d = 0; d < 3; d++) nbnd[d] -= nij[d];
            const double *qj = Q + (size_t)j * b;
            double qbar[MAXB];
            for (int m = 0; m < b; m++) qbar[m] = 0.5 * (qi[m] + qj[m]);
            oracle_flux_jacobian(b, qj, nij, gamma, Aj);
            oracle_flux_jacobian(b, qi, nij, gamma, Ai);
            oracle_abs_jacobian(b, qbar, nij, gamma, delta, Ab);
            double *Oij = offd + (size_t)p * bb;
            for (int t = 0; t < bb; t++) {
                Oij[t] = 0.5 * (Aj[t] - Ab[t]);
                Pi[t] += 0.5 * (Ai[t] + Ab[t]);
            }
            lsum += oracle_spectral_radius(qbar, nij, gamma);
        }
        /* far-field closure face */
        oracle_flux_jacobian(b, qi, nbnd, gamma, Ai);
        oracle_abs_jacobian(b, qi, nbnd, gamma, delta, Ab);
        for (int t = 0; t < bb; t++) Pi[t] += 0.5 * (Ai[t] + Ab[t]);
        lsum += oracle_spectral_radius(qi, nbnd, gamma);
        if (b == 6) Pi[5 * b + 5] *= 2.0;
        if (pseudo_block) {
            double s = 1.0 + 1.0 / (eps * cfl);
            for (int t = 0; t < bb; t++) Pi[t] *= s;
            D[i] = 0.0;
        } else {
            D[i] = lsum / cfl;
        }
    }
    free(nb);
    return 0;
}

/* ----------------------------------------------------------- block solves */

/* real LU with partial pivoting: solve M y = s (M destroyed) */
static int lu_solve_real(int b, double *M, double *s)
{
    for (int k = 0; k < b; k++) {
        int piv = k;
        for (int r = k + 1; r < b; r++)
            if (fabs(M[r * b + k]) > fabs(M[piv * b + k])) piv = r;
        if (M[piv * b + k] == 0.0) return -1;
        if (piv != k) {
            for (int c = 0; c < b; c++) {
                double t = M[k * b + c];
                M[k * b + c] = M[piv * b + c];
                M[piv * b + c] = t;
            }
            double t = s[k];
            s[k] = s[piv];
            s[piv] = t;
        }
        for (int r = k + 1; r < b; r++) {
            double l = M[r * b + k] / M[k * b + k];
            for (int c = k + 1; c < b; c++) M[r * b + c] -= l * M[k * b + c];
            s[r] -= l * s[k];
        }
    }
    for (int k = b - 1; k >= 0; k--) {
        double acc = s[k];
        for (int c = k + 1; c < b; c++) acc -= M[k * b + c] * s[c];
        s[k] = acc / M[k * b + k];
    }
    return 0;
}

/* complex LU with partial pivoting: solve M y = s (M destroyed) */
static int lu_solve_cplx(int b, cplx *M, cplx *s)
{
    for (int k = 0; k < b; k++) {
        int piv = k;
        for (int r = k + 1; r < b; r++)
            if (cabs(M[r * b + k]) > cabs(M[piv * b + k])) piv = r;
        if (M[piv * b + k] == 0.0) return -1;
        if (piv != k) {
            for (int c = 0; c < b; c++) {
                cplx t = M[k * b + c];
                M[k * b + c] = M[piv * b + c];
                M[piv * b + c] = t;
            }
            cplx t = s[k];
            s[k] = s[piv];
            s[piv] = t;
        }
        for (int r = k + 1; r < b; r++) {
            cplx l = M[r * b + k] / M[k * b + k];
            for (int c = k + 1; c < b; c++) M[r * b + c] -= l * M[k * b + c];
            s[r] -= l * s[k];
        }
    }
    for (int k = b - 1; k >= 0; k--) {
        cplx acc = s[k];
        for (int c = k + 1; c < b; c++) acc -= M[k * b + c] * s[c];
        s[k] = acc / M[k * b + k];
    }
    return 0;
}

/* -------------------------------------------------------------- Jacobi */

/* S -= sum_j J_ij x_j over row i for every column of the [C][b] row S.  With
 * side != NULL, harmonic l takes x_j times e^{i side[p] sigma[l-1]} on the
 * entries of periodic edges (phase-lagged boundary); the mean flow never.
 * With part != NULL, neighbours in another partition than i are skipped. */
static void subtract_offd(int i, int b, int n_harm, const int32_t *row_ptr, const int32_t *col_idx,
                          const double *offd, const int8_t *side, const double *sigma, const int32_t *part,
                          const double *X, double *S)
{
    const int C = 1 + 2 * n_harm, bb = b * b;
    const size_t row = (size_t)C * b;
    for (int p = row_ptr[i]; p < row_ptr[i + 1]; p++) {
        if (part && part[col_idx[p]] != part[i]) continue;
        const double *Jij = offd + (size_t)p * bb;
        const double *Xj = X + (size_t)col_idx[p] * row;
        const int s = side ? side[p] : 0;
        for (int c = 0; c < C; c++) {
            double xs[MAXB];
            for (int t = 0; t < b; t++) xs[t] = Xj[c * b + t];
            if (s != 0 && c > 0) {
                /* column c is Re (odd c) or Im (even c) of harmonic l */
                const int l = (c + 1) / 2;
                const double ang = s * sigma[l - 1];
                const double cs = cos(ang), sn = sin(ang);
                for (int t = 0; t < b; t++) {
                    const double re = Xj[(2 * l - 1) * b + t], im = Xj[(2 * l) * b + t];
                    xs[t] = (c % 2 == 1) ? cs * re - sn * im : sn * re + cs * im;
                }
            }
            for (int r = 0; r < b; r++) {
                double acc = 0.0;
                for (int t = 0; t < b; t++) acc += Jij[r * b + t] * xs[t];
                S[c * b + r] -= acc;
            }
        }
    }
}

/* One undamped block-Jacobi sweep per iteration, `sweeps` iterations;
 * X holds x^0 on entry and x^sweeps on return.  side / sigma (nullable):
 * phase-lagged periodic edges; part (nullable): partition of each node,
 * couplings across partitions dropped (subtract_offd).  Returns -1 on a
 * singular diagonal block. */
int oracle_jacobi(int n, int b, int n_harm, const int32_t *row_ptr, const int32_t *col_idx,
                  const double *offd, const double *diag, const double *D, const double *vol,
                  const double *omega, const int8_t *side, const double *sigma, const double *B, double *X,
                  int sweeps, const int32_t *part)
{
    const int C = 1 + 2 * n_harm, bb = b * b;
    const size_t row = (size_t)C * b;
    double *Xn = (double *)malloc(sizeof(double) * (size_t)n * row + 8);
    int fail = 0;
    for (int s = 0; s < sweeps; s++) {
#pragma omp parallel for schedule(static) reduction(| : fail)
        for (int i = 0; i < n; i++) {
            double S[(1 + 2 * 64) * MAXB];
            const double *Bi = B + (size_t)i * row;
            for (size_t t = 0; t < row; t++) S[t] = Bi[t];
            subtract_offd(i, b, n_harm, row_ptr, col_idx, offd, side, sigma, part, X, S);
            const double *Pi = diag + (size_t)i * bb;
            double *Yi = Xn + (size_t)i * row;
            /* mean flow: real system (omega = 0) */
            double M[MAXB * MAXB], y[MAXB];
            for (int t = 0; t < bb; t++) M[t] = Pi[t];
            for (int r = 0; r < b; r++) M[r * b + r] += D[i];
            for (int r = 0; r < b; r++) y[r] = S[r];
            if (lu_solve_real(b, M, y)) fail = 1;
            for (int r = 0; r < b; r++) Yi[r] = y[r];
            /* harmonics: complex systems */
            for (int k = 1; k <= n_harm; k++) {
                cplx Mc[MAXB * MAXB], yc[MAXB];
                cplx shift = D[i] + I * omega[k - 1] * vol[i];
                for (int t = 0; t < bb; t++) Mc[t] = Pi[t];
                for (int r = 0; r < b; r++) Mc[r * b + r] += shift;
                for (int r = 0; r < b; r++) yc[r] = S[(2 * k - 1) * b + r] + I * S[(2 * k) * b + r];
                if (lu_solve_cplx(b, Mc, yc)) fail = 1;
                for (int r = 0; r < b; r++) {
                    Yi[(2 * k - 1) * b + r] = creal(yc[r]);
                    Yi[(2 * k) * b + r] = cimag(yc[r]);
                }
            }
        }
        memcpy(X, Xn, sizeof(double) * (size_t)n * row);
    }
    free(Xn);
    return fail ? -1 : 0;
}

/* ------------------------------------------------------------ residual */

/* r_k = B_k - A_k x_k; norms[2k] = ||r_k||^2, norms[2k+1] = ||B_k||^2 (sums in
 * node order).  r may be NULL. */
int oracle_residual(int n, int b, int n_harm, const int32_t *row_ptr, const int32_t *col_idx,
                    const double *offd, const double *diag, const double *D, const double *vol,
                    const double *omega, const int8_t *side, const double *sigma, const double *B,
                    const double *X, double *r, double *norms)
{
    const int C = 1 + 2 * n_harm, K = 1 + n_harm, bb = b * b;
    const size_t row = (size_t)C * b;
    double *part = (double *)calloc((size_t)n * 2 * K + 1, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        double R[(1 + 2 * 64) * MAXB];
        const double *Bi = B + (size_t)i * row;
        const double *Xi = X + (size_t)i * row;
        for (size_t t = 0; t < row; t++) R[t] = Bi[t];
        subtract_offd(i, b, n_harm, row_ptr, col_idx, offd, side, sigma, NULL, X, R);
        const double *Pi = diag + (size_t)i * bb;
        for (int c = 0; c < C; c++)
            for (int rr = 0; rr < b; rr++) {
                double acc = 0.0;
                for (int t = 0; t < b; t++) acc += Pi[rr * b + t] * Xi[c * b + t];
                acc += D[i] * Xi[c * b + rr];
                R[c * b + rr] -= acc;
            }
        for (int k = 1; k <= n_harm; k++) {
            double wv = omega[k - 1] * vol[i];
            for (int rr = 0; rr < b; rr++) {
                /* (i w V)(xr + i xi) = -w V xi + i w V xr */
                R[(2 * k - 1) * b + rr] -= -wv * Xi[(2 * k) * b + rr];
                R[(2 * k) * b + rr] -= wv * Xi[(2 * k - 1) * b + rr];
            }
        }
        if (r)
            for (size_t t = 0; t < row; t++) r[(size_t)i * row + t] = R[t];
        double *pi = part + (size_t)i * 2 * K;
        for (int k = 0; k < K; k++) {
            int c0 = (k == 0) ? 0 : 2 * k - 1, nc = (k == 0) ? 1 : 2;
            double rs = 0.0, bs = 0.0;
            for (int c = c0; c < c0 + nc; c++)
                for (int rr = 0; rr < b; rr++) {
                    rs += R[c * b + rr] * R[c * b + rr];
                    bs += Bi[c * b + rr] * Bi[c * b + rr];
                }
            pi[2 * k] = rs;
            pi[2 * k + 1] = bs;
        }
    }
    for (int t = 0; t < 2 * K; t++) norms[t] = 0.0;
    for (int i = 0; i < n; i++)
        for (int t = 0; t < 2 * K; t++) norms[t] += part[(size_t)i * 2 * K + t];
    free(part);
    return 0;
}

/* -------------------------------------------------------------- ILU(0) */

/* Complex block inverse by Gauss-Jordan elimination with partial pivoting
 * (M destroyed).  Returns -1 on a zero pivot. */
static int inv_cplx(int b, cplx *M, cplx *Minv)
{
    for (int r = 0; r < b; r++)
        for (int c = 0; c < b; c++) Minv[r * b + c] = (r == c) ? 1.0 : 0.0;
    for (int k = 0; k < b; k++) {
        int piv = k;
        for (int r = k + 1; r < b; r++)
            if (cabs(M[r * b + k]) > cabs(M[piv * b + k])) piv = r;
        if (M[piv * b + k] == 0.0) return -1;
        for (int c = 0; c < b; c++) {
            cplx t = M[k * b + c];
            M[k * b + c] = M[piv * b + c];
            M[piv * b + c] = t;
            t = Minv[k * b + c];
            Minv[k * b + c] = Minv[piv * b + c];
            Minv[piv * b + c] = t;
        }
        const cplx d = M[k * b + k];
        for (int c = 0; c < b; c++) {
            M[k * b + c] /= d;
            Minv[k * b + c] /= d;
        }
        for (int r = 0; r < b; r++) {
            if (r == k) continue;
            const cplx f = M[r * b + k];
            for (int c = 0; c < b; c++) {
                M[r * b + c] -= f * M[k * b + c];
                Minv[r * b + c] -= f * Minv[k * b + c];
            }
        }
    }
    return 0;
}

/* C = A B for complex b x b blocks. */
static void mul_cplx(int b, const cplx *A, const cplx *B, cplx *C)
{
    for (int r = 0; r < b; r++)
        for (int c = 0; c < b; c++) {
            cplx acc = 0.0;
            for (int t = 0; t < b; t++) acc += A[r * b + t] * B[t * b + c];
            C[r * b + c] = acc;
        }
}

static int find_entry(const int32_t *row_ptr, const int32_t *col_idx, int i, int j)
{
    for (int p = row_ptr[i]; p < row_ptr[i + 1]; p++)
        if (col_idx[p] == j) return p;
    return -1;
}

/* Block ILU(0) of the matrix of one system -- the paper's implicit smoother
 * (Generalized RK scheme: "ILU(0)" approximate inversion of the LHS) -- in the
 * elimination order given by rank[] (rank[i] = position of node i), by the
 * row-oriented (IKJ) elimination restricted to the sparsity pattern:
 *
 *   for every row i in order, for every neighbour k of i earlier in the
 *   order (by increasing rank):
 *       L_ik = W_ik U_kk^-1,
 *       W_ij -= L_ik U_kj  for every j later than k in row k with (i, j) in the
 *                          pattern (j = i: the diagonal block),
 *
 * W starting as the system's matrix: A_ii = J_ii + (D_i + i omega V_i) I and
 * A_ij = J_ij e^{i side sigma} (phase-lagged periodic entries), with every
 * coupling between partitions dropped (part != NULL).  Out (interleaved
 * complex): Fdiag [n][b][b] = U_ii, Foffd [nnz][b][b] = L_ij (j earlier) or
 * U_ij (j later), zero for dropped entries.  Returns -1 on a zero pivot. */
int oracle_ilu_factor(int n, int b, const int32_t *row_ptr, const int32_t *col_idx, const double *offd,
                      const double *diag, const double *D, const double *vol, double omega,
                      const int8_t *side, double sigma, const int32_t *part, const int32_t *rank,
                      double *Fdiag, double *Foffd)
{
    const int bb = b * b;
    cplx *Wd = (cplx *)Fdiag, *Wo = (cplx *)Foffd;
    for (int i = 0; i < n; i++) {
        for (int t = 0; t < bb; t++) Wd[(size_t)i * bb + t] = diag[(size_t)i * bb + t];
        for (int r = 0; r < b; r++) Wd[(size_t)i * bb + r * b + r] += D[i] + I * omega * vol[i];
        for (int p = row_ptr[i]; p < row_ptr[i + 1]; p++) {
            const int j = col_idx[p];
            const int drop = part && part[i] != part[j];
            const cplx ph = (side && side[p]) ? cexp(I * (double)side[p] * sigma) : 1.0;
            for (int t = 0; t < bb; t++) Wo[(size_t)p * bb + t] = drop ? 0.0 : ph * offd[(size_t)p * bb + t];
        }
    }
    int *perm = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; i++) perm[rank[i]] = i;
    cplx Uinv[MAXB * MAXB], tmp[MAXB * MAXB], L[MAXB * MAXB], upd[MAXB * MAXB];
    int fail = 0;
    for (int pos = 0; pos < n; pos++) {
        const int i = perm[pos];
        /* earlier neighbours of i, by increasing rank */
        int lower[64], nl = 0;
        for (int p = row_ptr[i]; p < row_ptr[i + 1] && nl < 64; p++) {
            const int k = col_idx[p];
            if (rank[k] < rank[i] && !(part && part[k] != part[i])) lower[nl++] = p;
        }
        for (int a = 1; a < nl; a++)
            for (int c = a; c > 0 && rank[col_idx[lower[c]]] < rank[col_idx[lower[c - 1]]]; c--) {
                int t = lower[c];
                lower[c] = lower[c - 1];
                lower[c - 1] = t;
            }
        for (int a = 0; a < nl; a++) {
            const int pik = lower[a], k = col_idx[pik];
            for (int t = 0; t < bb; t++) tmp[t] = Wd[(size_t)k * bb + t];
            if (inv_cplx(b, tmp, Uinv)) fail = 1;
            mul_cplx(b, Wo + (size_t)pik * bb, Uinv, L);
            for (int q = row_ptr[k]; q < row_ptr[k + 1]; q++) {
                const int j = col_idx[q];
                if (rank[j] <= rank[k] || (part && part[j] != part[k])) continue;
                cplx *target = NULL;
                if (j == i) {
                    target = Wd + (size_t)i * bb;
                } else {
                    const int pij = find_entry(row_ptr, col_idx, i, j);
                    if (pij >= 0 && !(part && part[j] != part[i])) target = Wo + (size_t)pij * bb;
                }
                if (!target) continue; /* fill outside the pattern: dropped */
                mul_cplx(b, L, Wo + (size_t)q * bb, upd);
                for (int t = 0; t < bb; t++) target[t] -= upd[t];
            }
            for (int t = 0; t < bb; t++) Wo[(size_t)pik * bb + t] = L[t];
        }
    }
    free(perm);
    return fail ? -1 : 0;
}

/* y = (L U)^-1 r for the factors of oracle_ilu_factor (unit lower L):
 * forward z_i = r_i - sum_{k earlier} L_ik z_k, then backward
 * y_i = U_ii^-1 (z_i - sum_{j later} U_ij y_j), both in rank order.
 * r, y: interleaved complex [n][b]. */
int oracle_ilu_apply(int n, int b, const int32_t *row_ptr, const int32_t *col_idx, const int32_t *part,
                     const int32_t *rank, const double *Fdiag, const double *Foffd, const double *r, double *y)
{
    const int bb = b * b;
    const cplx *Ud = (const cplx *)Fdiag, *Fo = (const cplx *)Foffd;
    cplx *z = (cplx *)y;
    const cplx *rc = (const cplx *)r;
    int *perm = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; i++) perm[rank[i]] = i;
    for (int t = 0; t < n * b; t++) z[t] = rc[t];
    for (int pos = 0; pos < n; pos++) {
        const int i = perm[pos];
        for (int p = row_ptr[i]; p < row_ptr[i + 1]; p++) {
            const int k = col_idx[p];
            if (rank[k] >= rank[i] || (part && part[k] != part[i])) continue;
            for (int rr = 0; rr < b; rr++) {
                cplx acc = 0.0;
                for (int t = 0; t < b; t++) acc += Fo[(size_t)p * bb + rr * b + t] * z[(size_t)k * b + t];
                z[(size_t)i * b + rr] -= acc;
            }
        }
    }
    int fail = 0;
    for (int pos = n - 1; pos >= 0; pos--) {
        const int i = perm[pos];
        cplx t_[MAXB], M[MAXB * MAXB];
        for (int rr = 0; rr < b; rr++) t_[rr] = z[(size_t)i * b + rr];
        for (int p = row_ptr[i]; p < row_ptr[i + 1]; p++) {
            const int j = col_idx[p];
            if (rank[j] <= rank[i] || (part && part[j] != part[i])) continue;
            for (int rr = 0; rr < b; rr++) {
                cplx acc = 0.0;
                for (int t = 0; t < b; t++) acc += Fo[(size_t)p * bb + rr * b + t] * z[(size_t)j * b + t];
                t_[rr] -= acc;
            }
        }
        for (int t = 0; t < bb; t++) M[t] = Ud[(size_t)i * bb + t];
        if (lu_solve_cplx(b, M, t_)) fail = 1;
        for (int rr = 0; rr < b; rr++) z[(size_t)i * b + rr] = t_[rr];
    }
    free(perm);
    return fail ? -1 : 0;
}

void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
