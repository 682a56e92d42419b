// Jacobian assembly and sweep preparation (FP64).
//
// Paper: arXiv 2404.01407, Eq. precon (implicit K = P/(eps sigma) + J, where
// J = dR/dQ is an approximate, first-order Jacobian built from each node's
// immediate neighbours only) and "Solution Update" (J assembled once per
// nonlinear iteration and shared by the mean flow and every harmonic).
//
// Both kernels here run once per nonlinear iteration, off the sweep loop.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "schur.cuh"

namespace fnlh {

// Closed-form Euler flux Jacobian d(F.n)/dQ for conservative Q and an
// unnormalised face normal n; with six equations the sixth (turbulence)
// variable is advected at u_n and does not feed back (frozen turbulence).
template <int BS>
__device__ __forceinline__ void flux_jacobian(const double (&q)[BS], const double n[3], double gamma,
                                              double (&A)[BS][BS]) {
  const double rho = q[0], ir = 1.0 / rho;
  const double vel[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
  const double g1 = gamma - 1.0;
  const double ke = 0.5 * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]);
  const double p = g1 * (q[4] - rho * ke);
  const double H = (q[4] + p) * ir;
  const double phi = g1 * ke;
  const double un = vel[0] * n[0] + vel[1] * n[1] + vel[2] * n[2];
#pragma unroll
  for (int r = 0; r < BS; ++r)
#pragma unroll
    for (int c = 0; c < BS; ++c) A[r][c] = 0.0;
  A[0][1] = n[0];
  A[0][2] = n[1];
  A[0][3] = n[2];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    A[1 + r][0] = n[r] * phi - vel[r] * un;
#pragma unroll
    for (int c = 0; c < 3; ++c) A[1 + r][1 + c] = vel[r] * n[c] - g1 * vel[c] * n[r];
    A[1 + r][1 + r] += un;
    A[1 + r][4] = g1 * n[r];
  }
  A[4][0] = un * (phi - H);
#pragma unroll
  for (int c = 0; c < 3; ++c) A[4][1 + c] = H * n[c] - g1 * vel[c] * un;
  A[4][4] = gamma * un;
  if (BS == 6) {
    const double nu = q[BS - 1] * ir;
    A[BS - 1][0] = -nu * un;
    A[BS - 1][1] = nu * n[0];
    A[BS - 1][2] = nu * n[1];
    A[BS - 1][3] = nu * n[2];
    A[BS - 1][BS - 1] = un;
  }
}

// |A|(Q, n) with the entropy fix f(l) = max(|l|, delta (|u_n| + a|n|)) on the
// Euler block (the turbulence row gets the scalar f(u_n)); returns the
// spectral radius |u_n| + a|n|.  On the Euler block N = A - u_n I has rank two:
//   N = alpha p^T + beta q^T,  alpha = (1, v, H), beta = (0, n, u_n),
//                              p = (-u_n, n, 0), q = (phi, -(gamma-1) v, gamma-1),
// phi = (gamma-1)|v|^2/2, and the Gram products are p.alpha = q.beta = 0,
// p.beta = |n|^2, q.alpha = (gamma-1)(H - |v|^2/2) = a^2.  The spectral form
// |A| = sum_k f(l_k) P_k = f0 I + s2 N^2 + s1 N (projectors onto the
// eigenspaces of u_n and u_n +- c, c = a|n|, s2 = ((f+ + f-)/2 - f0)/c^2,
// s1 = (f+ - f-)/(2c)) therefore collapses to
//   |A| = f0 I + [alpha beta] C [p q]^T,   C = [[s1, s2 |n|^2], [s2 a^2, s1]],
// 70 multiply-adds instead of a 5x5 matrix product.
template <int BS>
__device__ __forceinline__ double abs_flux_jacobian(const double (&q)[BS], const double n[3], double gamma,
                                                    double delta, double (&M)[BS][BS]) {
#pragma unroll
  for (int r = 0; r < BS; ++r)
#pragma unroll
    for (int c = 0; c < BS; ++c) M[r][c] = 0.0;
  const double g1 = gamma - 1.0;
  const double ir = 1.0 / q[0];
  const double v[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
  const double ke = 0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  const double pr = g1 * (q[4] - q[0] * ke);
  const double a2 = gamma * pr * ir;
  const double un = v[0] * n[0] + v[1] * n[1] + v[2] * n[2];
  const double nn2 = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
  const double c = sqrt(a2) * sqrt(nn2);
  const double lam = fabs(un) + c;
  if (nn2 == 0.0) return lam;
  const double fix = delta * lam;
  const double f0 = fmax(fabs(un), fix), fp = fmax(fabs(un + c), fix), fm = fmax(fabs(un - c), fix);
  const double ic = 1.0 / c;
  const double s1 = 0.5 * (fp - fm) * ic;
  const double s2 = (0.5 * (fp + fm) - f0) * ic * ic;
  const double H = (q[4] + pr) * ir;
  const double alpha[5] = {1.0, v[0], v[1], v[2], H};
  const double beta[5] = {0.0, n[0], n[1], n[2], un};
  const double pv[5] = {-un, n[0], n[1], n[2], 0.0};
  const double qv[5] = {g1 * ke, -g1 * v[0], -g1 * v[1], -g1 * v[2], g1};
  const double c01 = s2 * nn2, c10 = s2 * a2;
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const double w0 = alpha[r] * s1 + beta[r] * c10;
    const double w1 = alpha[r] * c01 + beta[r] * s1;
#pragma unroll
    for (int k = 0; k < 5; ++k) M[r][k] = w0 * pv[k] + w1 * qv[k] + (r == k ? f0 : 0.0);
  }
  if (BS == 6) M[5][5] = f0;
  return lam;
}

struct BuildArgs {
  int32_t n;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const int32_t* csr_edge;
  const int32_t* edge_nodes;
  const double* normals;
  const double* Q;
  double* offd;
  double* diag;
  double* D;
  double gamma, cfl, delta, eps;
  int32_t pseudo_time;
};

// One thread per node: its off-diagonal row blocks, its diagonal block and
// D_i, accumulated in neighbour order (no atomics, deterministic).
template <int BS>
__global__ void __launch_bounds__(128) k_build_jacobian(BuildArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  double qi[BS];
#pragma unroll
  for (int m = 0; m < BS; ++m) qi[m] = a.Q[(size_t)i * BS + m];
  double P[BS][BS];
#pragma unroll
  for (int r = 0; r < BS; ++r)
#pragma unroll
    for (int c = 0; c < BS; ++c) P[r][c] = 0.0;
  double nb[3] = {0.0, 0.0, 0.0};
  double lsum = 0.0;
  const int p0 = a.row_ptr[i], p1 = a.row_ptr[i + 1];
  for (int p = p0; p < p1; ++p) {
    const int j = a.col_idx[p];
    const int e = a.csr_edge[p];
    const double sg = (a.edge_nodes[2 * e] == i) ? 1.0 : -1.0;
    const double n[3] = {sg * a.normals[3 * e], sg * a.normals[3 * e + 1], sg * a.normals[3 * e + 2]};
    nb[0] -= n[0];
    nb[1] -= n[1];
    nb[2] -= n[2];
    double qj[BS], qb[BS];
#pragma unroll
    for (int m = 0; m < BS; ++m) {
      qj[m] = a.Q[(size_t)j * BS + m];
      qb[m] = 0.5 * (qi[m] + qj[m]);
    }
    double M[BS][BS], Aj[BS][BS];
    lsum += abs_flux_jacobian<BS>(qb, n, a.gamma, a.delta, M);
    flux_jacobian<BS>(qj, n, a.gamma, Aj);
    double* o = a.offd + (size_t)p * BS * BS;
#pragma unroll
    for (int r = 0; r < BS; ++r)
#pragma unroll
      for (int c = 0; c < BS; ++c) {
        o[r * BS + c] = 0.5 * (Aj[r][c] - M[r][c]);
        P[r][c] += 0.5 * M[r][c];
      }
  }
  {
    double M[BS][BS];
    lsum += abs_flux_jacobian<BS>(qi, nb, a.gamma, a.delta, M);
#pragma unroll
    for (int r = 0; r < BS; ++r)
#pragma unroll
      for (int c = 0; c < BS; ++c) P[r][c] += 0.5 * M[r][c];
  }
  if (BS == 6) P[5][5] *= 2.0;
  const double scale = a.pseudo_time ? (1.0 + 1.0 / (a.eps * a.cfl)) : 1.0;
  double* d = a.diag + (size_t)i * BS * BS;
#pragma unroll
  for (int r = 0; r < BS; ++r)
#pragma unroll
    for (int c = 0; c < BS; ++c) d[r * BS + c] = P[r][c] * scale;
  a.D[i] = a.pseudo_time ? 0.0 : lsum / a.cfl;
}

// Per-node orthogonal basis for the sweeps, one thread per node:
// P_i = J_ii + D_i I is reduced to upper Hessenberg form by Householder
// reflections and then, by the double-shift QR iteration, to real Schur
// form Z_i^T P_i Z_i = T_i (upper triangular).  Block Jacobi is invariant
// under the block-diagonal change of basis x = Z x~, and in the new basis the
// shifted diagonal solve of every system, (T_i + i omega V_i I) y = r, is a
// back-substitution.  A block whose spectrum has a complex pair keeps the
// Hessenberg form (the solve then eliminates first).  The 5 x 5 mean-flow
// block of a b = 6 frozen-turbulence node takes the cheaper FP32-seeded
// eigenvector basis first (schur_eigvec), the FP64 iteration only where that
// is not accepted.
template <int BS>
__global__ void __launch_bounds__(128) k_prepare_basis(int32_t n, const double* __restrict__ diag,
                                                       const double* __restrict__ D, double* __restrict__ rot,
                                                       double* __restrict__ hess, float* __restrict__ hessf,
                                                       float* __restrict__ rotf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double P[BS][BS], Q[BS][BS];
  const double Di = D[i];
  for (int r = 0; r < BS; ++r)
    for (int c = 0; c < BS; ++c) {
      P[r][c] = diag[(size_t)i * BS * BS + r * BS + c] + (r == c ? Di : 0.0);
      Q[r][c] = (r == c) ? 1.0 : 0.0;
    }
  if constexpr (BS == 6) {
    // Frozen turbulence: the mean-flow rows do not see the turbulence
    // variable (column 5 of rows 0..4 is zero), so M is block triangular once
    // the turbulence variable comes first.  Its basis Z = [e_5 | (Z5; 0)],
    // with Z5 the Schur (or Hessenberg) basis of the 5x5 mean-flow block,
    // keeps that: every rotated block then has zeros below its first entry
    // in column 0, which the FP64 kernels skip (k_check_structure certifies).
    bool st = true;
    for (int r = 0; r < 5; ++r) st = st && (P[r][5] == 0.0);
    if (st) {
      double P5[5][5], Q5[5][5];
      for (int r = 0; r < 5; ++r)
        for (int c = 0; c < 5; ++c) {
          P5[r][c] = P[r][c];
          Q5[r][c] = (r == c) ? 1.0 : 0.0;
        }
      // Z5 from the FP32-seeded eigenvector basis when it is accepted
      // (about a third of the FP64 work), else by the FP64 Francis iteration.
      // Only this path takes the eigenvector route: with it inlined into the
      // generic path of the same kernel as well, every node's H came out
      // wrong on GB300 while Z stayed right -- read back, H held exactly what
      // it would if T5 and H6 shared storage (H6's zero fill and its first
      // entries showing through T5) -- although the source reads T5 only
      // after writing it.  With this one instance H is exact.
      double T5[5][5], Z5[5][5];
      bool tri5 = schur_eigvec<5>(P5, Z5, T5);
      if (!tri5) {
        hessenberg_reduce<5>(P5, Q5);
        for (int r = 0; r < 5; ++r)
          for (int c = 0; c < 5; ++c) {
            T5[r][c] = P5[r][c];
            Z5[r][c] = Q5[r][c];
          }
        tri5 = schur_real<5>(T5, Z5);
      }
      double Z6[6][6], H6[6][6];
      for (int m = 0; m < 6; ++m)
        for (int c = 0; c < 6; ++c) {
          Z6[m][c] = (c == 0) ? (m == 5 ? 1.0 : 0.0) : (m < 5 ? (tri5 ? Z5[m][c - 1] : Q5[m][c - 1]) : 0.0);
          H6[m][c] = 0.0;
        }
      H6[0][0] = P[5][5];
      for (int c = 1; c < 6; ++c) {
        double t = 0.0;
        for (int m = 0; m < 5; ++m) t += P[5][m] * Z6[m][c];
        H6[0][c] = t;
      }
      for (int r = 1; r < 6; ++r)
        for (int c = 1; c < 6; ++c) {
          const double v = tri5 ? T5[r - 1][c - 1] : P5[r - 1][c - 1];
          H6[r][c] = tri5 ? ((r > c) ? 0.0 : v) : ((r > c + 1) ? 0.0 : v);
        }
      for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 6; ++c) {
          const size_t o = (size_t)i * 36 + r * 6 + c;
          rot[o] = Z6[r][c];
          if (rotf) rotf[o] = (float)Z6[r][c];
          hess[o] = H6[r][c];
          if (hessf) hessf[o] = (float)H6[r][c];
        }
      return;
    }
  }
  hessenberg_reduce<BS>(P, Q);
  double T[BS][BS], Z[BS][BS];
  for (int r = 0; r < BS; ++r)
    for (int c = 0; c < BS; ++c) {
      T[r][c] = P[r][c];
      Z[r][c] = Q[r][c];
    }
  const bool tri = schur_real<BS>(T, Z);
  for (int r = 0; r < BS; ++r)
    for (int c = 0; c < BS; ++c) {
      const double h = tri ? ((r > c) ? 0.0 : T[r][c]) : ((r > c + 1) ? 0.0 : P[r][c]);
      const double z = tri ? Z[r][c] : Q[r][c];
      rot[(size_t)i * BS * BS + r * BS + c] = z;
      if (rotf) rotf[(size_t)i * BS * BS + r * BS + c] = (float)z;
      hess[(size_t)i * BS * BS + r * BS + c] = h;
      if (hessf) hessf[(size_t)i * BS * BS + r * BS + c] = (float)h;
    }
}

// b = 6: the basis Q = [e_5 | (Z5; 0)] that k_prepare_basis builds when the
// mean-flow rows do not see the turbulence variable (exact zeros and one).
template <int BS>
__device__ __forceinline__ bool turbulence_first(const double* __restrict__ Q) {
  if constexpr (BS != 6) {
    return false;
  } else {
    bool st = Q[5 * 6] == 1.0;
#pragma unroll
    for (int r = 0; r < 5; ++r) st = st && Q[r * 6] == 0.0;
#pragma unroll
    for (int c = 1; c < 6; ++c) st = st && Q[5 * 6 + c] == 0.0;
    return st;
  }
}

// Rotated off-diagonal blocks Q_i^T J_ij Q_j, one thread per CSR entry (the
// owning row found by binary search over row_ptr), written in every
// requested precision (round to nearest).  Between two frozen-turbulence
// bases the products skip the basis' structural zeros (300 instead of 432
// multiply-adds; the same sums in the same order, so the same values).  Four
// CTAs per SM (128 registers) beat three at 168 registers: the whole build
// step runs 5% faster on GB300.
template <int BS>
__global__ void __launch_bounds__(128, 4) k_rotate_offd(int32_t n, int32_t nnz, const int32_t* __restrict__ row_ptr,
                                                     const int32_t* __restrict__ col_idx,
                                                     const double* __restrict__ offd, const double* __restrict__ rot,
                                                     double* __restrict__ o64, float* __restrict__ o32,
                                                     __nv_bfloat16* __restrict__ o16) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nnz) return;
  int lo = 0, hi = n - 1;  // largest i with row_ptr[i] <= p
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (row_ptr[mid] <= p) lo = mid;
    else hi = mid - 1;
  }
  const int i = lo, j = col_idx[p];
  double T[BS][BS];
  const double* J = offd + (size_t)p * BS * BS;
  const double* Qj = rot + (size_t)j * BS * BS;
  const double* Qi = rot + (size_t)i * BS * BS;
  auto emit = [&](int r, int c, double t) {
    const size_t o = (size_t)p * BS * BS + r * BS + c;
    if (o64) o64[o] = t;
    if (o32) o32[o] = (float)t;
    if (o16) o16[o] = __double2bfloat16(t);
  };
  if (turbulence_first<BS>(Qi) && turbulence_first<BS>(Qj)) {
    // T = J Q_j: column 0 is J's last column; row 5 of Q_j is zero elsewhere
#pragma unroll
    for (int r = 0; r < BS; ++r) {
      T[r][0] = J[r * BS + BS - 1];
#pragma unroll
      for (int c = 1; c < BS; ++c) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < BS - 1; ++k) t += J[r * BS + k] * Qj[k * BS + c];
        T[r][c] = t;
      }
    }
    // Q_i^T T: row 0 is T's last row; the rest skip row 5 of Q_i
#pragma unroll
    for (int r = 0; r < BS; ++r)
#pragma unroll
      for (int c = 0; c < BS; ++c) {
        double t = 0.0;
        if (r == 0) {
          t = T[BS - 1][c];
        } else {
#pragma unroll
          for (int k = 0; k < BS - 1; ++k) t += Qi[k * BS + r] * T[k][c];
        }
        emit(r, c, t);
      }
    return;
  }
#pragma unroll
  for (int r = 0; r < BS; ++r)
#pragma unroll
    for (int c = 0; c < BS; ++c) {
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < BS; ++k) t += J[r * BS + k] * Qj[k * BS + c];
      T[r][c] = t;
    }
#pragma unroll
  for (int r = 0; r < BS; ++r)
#pragma unroll
    for (int c = 0; c < BS; ++c) {
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < BS; ++k) t += Qi[k * BS + r] * T[k][c];
      emit(r, c, t);
    }
}

// Tagged copy of col_idx, one thread per row: entry p of row i across edge e
// gets the passage offset of its neighbour as seen from i (phase-lagged
// periodic edges) -- periodic[e] when i is the edge's first node, its
// opposite otherwise -- in the top two bits, and the cut bit when the
// neighbour lies in another partition.  Neither array: an untagged copy.
__global__ void __launch_bounds__(128) k_tag_columns(int32_t n, const int32_t* __restrict__ row_ptr,
                                                     const int32_t* __restrict__ col_idx,
                                                     const int32_t* __restrict__ csr_edge,
                                                     const int32_t* __restrict__ edge_nodes,
                                                     const int8_t* __restrict__ periodic,
                                                     const int32_t* __restrict__ part, int32_t* __restrict__ cols) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
    uint32_t tag = 0;
    if (periodic) {
      const int e = csr_edge[p];
      int side = periodic[e] > 0 ? 1 : (periodic[e] < 0 ? -1 : 0);
      if (edge_nodes[2 * e] != i) side = -side;
      tag = side > 0 ? (kSideNext << 30) : (side < 0 ? (kSidePrev << 30) : 0u);
    }
    if (part && part[col_idx[p]] != part[i]) tag |= kCutBit;
    cols[p] = (int32_t)((uint32_t)col_idx[p] | tag);
  }
}

// Certifies the frozen-turbulence zero pattern (b = 6) that the FP64 kernels
// exploit: every node's basis has e_5 as its first column (so its M had
// column 5 zero above the diagonal) and every off-diagonal block has column 5
// zero in rows 0..4.  Any violation sets info[0]; thread t checks node t and
// CSR entry t.
__global__ void __launch_bounds__(128) k_check_structure(int32_t n, int32_t nnz, const double* __restrict__ offd,
                                                         const double* __restrict__ rot, int32_t* __restrict__ info) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  if (t < n) bad = rot[(size_t)t * 36 + 5 * 6 + 0] != 1.0;
  if (t < nnz)
    for (int r = 0; r < 5; ++r) bad = bad || (offd[(size_t)t * 36 + r * 6 + 5] != 0.0);
  if (bad) atomicOr(info, 1);
}

template <int BS>
int launch_build(const BuildArgs& a, cudaStream_t s) {
  if (a.n == 0) return FNLH_OK;
  k_build_jacobian<BS><<<(a.n + 127) / 128, 128, 0, s>>>(a);
  FNLH_LAUNCH_CHECK();
  return FNLH_OK;
}

// Float-float copies for the mixed solve's float-float residual checks: the
// off-diagonal blocks, and the diagonal blocks with the pseudo-time term
// folded in (J_ii + D_i I, summed in FP64 before the split).
template <int BS>
__global__ void __launch_bounds__(256) k_split_ff(long long n_offd, long long n_diag, const double* __restrict__ offd,
                                                  const double* __restrict__ diag, const double* __restrict__ D,
                                                  float2* __restrict__ offdff, float2* __restrict__ diagff) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n_offd) offdff[e] = ff_split(offd[e]);
  if (e < n_diag) {
    const long long i = e / (BS * BS);
    const int rc = (int)(e - i * BS * BS);
    const double v = diag[e] + ((rc / BS == rc % BS) ? D[i] : 0.0);
    diagff[e] = ff_split(v);
  }
}

template <int BS>
int launch_prepare(const fnlh_mesh* mesh, fnlh_jacobian* J, cudaStream_t s) {
  const PrepLayout L = prep_layout(J->n_nodes, J->nnz, BS, J->prep_flags);
  double* rot = at<double>(J->prep, L.rot);
  double* hess = at<double>(J->prep, L.hess);
  float* hessf = (L.hessf != (size_t)-1) ? at<float>(J->prep, L.hessf) : nullptr;
  float* rotf = (L.rotf != (size_t)-1) ? at<float>(J->prep, L.rotf) : nullptr;
  const int n = J->n_nodes;
  if (n > 0) {
    k_prepare_basis<BS><<<(n + 127) / 128, 128, 0, s>>>(n, J->diag, J->D, rot, hess, hessf, rotf);
    FNLH_LAUNCH_CHECK();
  }
  int32_t* info = at<int32_t>(J->prep, L.info);
  // nonzero bytes: no pattern to exploit (b = 5), cleared for b = 6 before the check
  FNLH_CUDA_TRY(cudaMemsetAsync(info, BS == 6 ? 0 : 1, sizeof(int32_t), s));
  if (BS == 6 && std::max(n, J->nnz) > 0) {
    k_check_structure<<<(std::max(n, J->nnz) + 127) / 128, 128, 0, s>>>(n, J->nnz, J->offd, rot, info);
    FNLH_LAUNCH_CHECK();
  }
  double* o64 = (L.offd64 != (size_t)-1) ? at<double>(J->prep, L.offd64) : nullptr;
  float* o32 = (L.offd32 != (size_t)-1) ? at<float>(J->prep, L.offd32) : nullptr;
  __nv_bfloat16* o16 = (L.offd16 != (size_t)-1) ? at<__nv_bfloat16>(J->prep, L.offd16) : nullptr;
  if (J->nnz > 0 && (o64 || o32 || o16)) {
    k_rotate_offd<BS><<<(J->nnz + 127) / 128, 128, 0, s>>>(n, J->nnz, mesh->row_ptr, mesh->col_idx, J->offd, rot,
                                                         o64, o32, o16);
    FNLH_LAUNCH_CHECK();
  }
  if (L.offdff != (size_t)-1) {
    const long long no = (long long)J->nnz * BS * BS, nd = (long long)n * BS * BS;
    const long long cnt = std::max(no, nd);
    if (cnt > 0) {
      k_split_ff<BS><<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(no, nd, J->offd, J->diag, J->D,
                                                                  at<float2>(J->prep, L.offdff),
                                                                  at<float2>(J->prep, L.diagff));
      FNLH_LAUNCH_CHECK();
    }
  }
  if (L.cols != (size_t)-1 && n > 0) {
    k_tag_columns<<<(n + 127) / 128, 128, 0, s>>>(n, mesh->row_ptr, mesh->col_idx, mesh->csr_edge, mesh->edge_nodes,
                                                  mesh->periodic, mesh->part, at<int32_t>(J->prep, L.cols));
    FNLH_LAUNCH_CHECK();
  }
  return FNLH_OK;
}

int build_jacobian_impl(const fnlh_mesh* mesh, const double* Q, const fnlh_params* prm, fnlh_jacobian* J,
                        cudaStream_t s) {
  BuildArgs a;
  a.n = mesh->n_nodes;
  a.row_ptr = mesh->row_ptr;
  a.col_idx = mesh->col_idx;
  a.csr_edge = mesh->csr_edge;
  a.edge_nodes = mesh->edge_nodes;
  a.normals = mesh->normals;
  a.Q = Q;
  a.offd = J->offd;
  a.diag = J->diag;
  a.D = J->D;
  a.gamma = prm->gamma;
  a.cfl = prm->cfl;
  a.delta = prm->entropy_delta;
  a.eps = prm->eps;
  a.pseudo_time = prm->pseudo_time;
  return J->block == 5 ? launch_build<5>(a, s) : launch_build<6>(a, s);
}

int prepare_impl(const fnlh_mesh* mesh, fnlh_jacobian* J, cudaStream_t s) {
  return J->block == 5 ? launch_prepare<5>(mesh, J, s) : launch_prepare<6>(mesh, J, s);
}

}  // namespace fnlh
