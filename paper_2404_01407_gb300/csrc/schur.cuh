// Real Schur form of the small per-node diagonal blocks (host and device).
//
// Implicit double-shift QR (Francis) with deflation: H <- Z^T H Z with Z
// accumulating every reflection, until H is upper triangular.  2 x 2 blocks
// with real eigenvalues are split by one rotation; a block with a complex
// pair makes the routine report failure (the caller then keeps the
// Hessenberg form).  The reduction and the iteration are templated on the
// element type: FP64 for the basis itself, FP32 for the estimates that
// schur_eigvec refines.
#pragma once

#include <math.h>

namespace fnlh {

// Householder reduction to upper Hessenberg form: P <- Q^T P Q, Q <- Q Q_k.
template <int BS, typename R>
__host__ __device__ inline void hessenberg_reduce(R (&P)[BS][BS], R (&Q)[BS][BS]) {
  for (int k = 0; k < BS - 2; ++k) {
    R v[BS];
    R alpha2 = R(0);
    for (int r = 0; r < BS; ++r) {
      v[r] = (r > k) ? P[r][k] : R(0);
      alpha2 += v[r] * v[r];
    }
    if (alpha2 == R(0)) continue;
    const R alpha = sqrt(alpha2);
    v[k + 1] += (v[k + 1] >= R(0)) ? alpha : -alpha;
    R vn2 = R(0);
    for (int r = 0; r < BS; ++r) vn2 += v[r] * v[r];
    if (vn2 == R(0)) continue;
    const R beta = R(2) / vn2;
    for (int c = 0; c < BS; ++c) {  // P <- (I - beta v v^T) P
      R t = R(0);
      for (int r = 0; r < BS; ++r) t += v[r] * P[r][c];
      t *= beta;
      for (int r = 0; r < BS; ++r) P[r][c] -= t * v[r];
    }
    for (int r = 0; r < BS; ++r) {  // P <- P (I - beta v v^T),  Q <- Q (I - beta v v^T)
      R t = R(0), u = R(0);
      for (int c = 0; c < BS; ++c) {
        t += P[r][c] * v[c];
        u += Q[r][c] * v[c];
      }
      t *= beta;
      u *= beta;
      for (int c = 0; c < BS; ++c) {
        P[r][c] -= t * v[c];
        Q[r][c] -= u * v[c];
      }
    }
    for (int r = k + 2; r < BS; ++r) P[r][k] = R(0);
  }
}

template <int BS, typename R>
__host__ __device__ inline void schur_rotate(R (&H)[BS][BS], R (&Z)[BS][BS], int r, R cs, R sn, int col_lo,
                                             int row_hi) {
  // rows r, r+1 (from the left, G^T) over columns col_lo..BS-1
  for (int c = col_lo; c < BS; ++c) {
    const R a = H[r][c], b = H[r + 1][c];
    H[r][c] = cs * a + sn * b;
    H[r + 1][c] = -sn * a + cs * b;
  }
  // columns r, r+1 (from the right, G) over rows 0..row_hi, and Z
  for (int q = 0; q <= row_hi; ++q) {
    const R a = H[q][r], b = H[q][r + 1];
    H[q][r] = cs * a + sn * b;
    H[q][r + 1] = -sn * a + cs * b;
  }
  for (int q = 0; q < BS; ++q) {
    const R a = Z[q][r], b = Z[q][r + 1];
    Z[q][r] = cs * a + sn * b;
    Z[q][r + 1] = -sn * a + cs * b;
  }
}

// Returns true when H was brought to upper triangular form (all eigenvalues
// real); on false, H and Z hold a partially reduced (still valid) similarity.
template <int BS, typename R>
__host__ __device__ inline bool schur_real(R (&H)[BS][BS], R (&Z)[BS][BS]) {
  const R eps = sizeof(R) == 8 ? R(2.220446049250313e-16) : R(1.1920929e-07);  // machine epsilon
  R anorm = R(0);
  for (int r = 0; r < BS; ++r)
    for (int c = 0; c < BS; ++c) anorm += fabs(H[r][c]);
  if (anorm == R(0)) return true;
  int hi = BS - 1, its = 0, total = 0;
  while (hi >= 1) {
    if (++total > 40 * BS) return false;
    int l = hi;
    for (; l > 0; --l) {
      R s = fabs(H[l - 1][l - 1]) + fabs(H[l][l]);
      if (s == R(0)) s = anorm;
      if (fabs(H[l][l - 1]) <= eps * s) {
        H[l][l - 1] = R(0);
        break;
      }
    }
    if (l == hi) {  // one eigenvalue converged
      --hi;
      its = 0;
      continue;
    }
    if (l == hi - 1) {  // trailing 2 x 2 block
      const R a = H[hi - 1][hi - 1], b = H[hi - 1][hi], c = H[hi][hi - 1], d = H[hi][hi];
      const R p = R(0.5) * (a - d);
      const R disc = p * p + b * c;
      if (disc < R(0)) return false;  // complex conjugate pair
      const R lam = d + p + copysign(sqrt(disc), p);
      // eigenvector of the block for lam, from its better-scaled row
      R u0, u1;
      if (fabs(lam - d) + fabs(c) >= fabs(b) + fabs(lam - a)) {
        u0 = lam - d;
        u1 = c;
      } else {
        u0 = b;
        u1 = lam - a;
      }
      const R un = sqrt(u0 * u0 + u1 * u1);
      if (un > R(0)) {
        schur_rotate<BS>(H, Z, hi - 1, u0 / un, u1 / un, hi - 1, hi);
      }
      H[hi][hi - 1] = R(0);
      hi -= 2;
      its = 0;
      continue;
    }
    // double-shift QR sweep on the active window l..hi
    ++its;
    R s, t;
    if (its % 10 == 0) {  // exceptional shift
      const R x = fabs(H[hi][hi - 1]) + fabs(H[hi - 1][hi - 2]);
      s = R(1.5) * x;
      t = x * x;
    } else {
      s = H[hi - 1][hi - 1] + H[hi][hi];
      t = H[hi - 1][hi - 1] * H[hi][hi] - H[hi - 1][hi] * H[hi][hi - 1];
    }
    R x = H[l][l] * H[l][l] + H[l][l + 1] * H[l + 1][l] - s * H[l][l] + t;
    R y = H[l + 1][l] * (H[l][l] + H[l + 1][l + 1] - s);
    R z = H[l + 1][l] * H[l + 2][l + 1];
    for (int k = l; k <= hi - 2; ++k) {
      // reflector (I - beta v v^T) taking (x, y, z) onto the first axis
      const R alpha = sqrt(x * x + y * y + z * z);
      if (alpha != R(0)) {
        const R v0 = x + copysign(alpha, x), v1 = y, v2 = z;
        const R beta = R(2) / (v0 * v0 + v1 * v1 + v2 * v2);
        const int c_lo = (k == l) ? l : k - 1;
        for (int c = c_lo; c < BS; ++c) {
          const R w = beta * (v0 * H[k][c] + v1 * H[k + 1][c] + v2 * H[k + 2][c]);
          H[k][c] -= w * v0;
          H[k + 1][c] -= w * v1;
          H[k + 2][c] -= w * v2;
        }
        const int r_hi = (k + 3 < hi) ? k + 3 : hi;
        for (int q = 0; q <= r_hi; ++q) {
          const R w = beta * (H[q][k] * v0 + H[q][k + 1] * v1 + H[q][k + 2] * v2);
          H[q][k] -= w * v0;
          H[q][k + 1] -= w * v1;
          H[q][k + 2] -= w * v2;
        }
        for (int q = 0; q < BS; ++q) {
          const R w = beta * (Z[q][k] * v0 + Z[q][k + 1] * v1 + Z[q][k + 2] * v2);
          Z[q][k] -= w * v0;
          Z[q][k + 1] -= w * v1;
          Z[q][k + 2] -= w * v2;
        }
        if (k > l) {
          H[k + 1][k - 1] = R(0);
          H[k + 2][k - 1] = R(0);
        }
      }
      x = H[k + 1][k];
      y = H[k + 2][k];
      z = (k < hi - 2) ? H[k + 3][k] : R(0);
    }
    // closing rotation on rows / columns hi-1, hi
    {
      const R r = sqrt(x * x + y * y);
      if (r != R(0)) {
        schur_rotate<BS>(H, Z, hi - 1, x / r, y / r, hi - 2, hi);
        H[hi][hi - 2] = R(0);
      }
    }
  }
  for (int r = 1; r < BS; ++r)
    for (int c = 0; c < r; ++c) H[r][c] = R(0);
  return true;
}


// Real Schur basis of a block with a real spectrum, mostly on the FP32 units
// (GB300 runs FP32 at 63x its FP64 rate):
//   1. the Francis iteration above in FP32 gives the eigenvalues in Schur
//      order (the diagonal of the FP32 triangle) and approximate Schur
//      vectors;
//   2. two steps of FP64 inverse iteration per eigenvalue (one LU with
//      partial pivoting of A - lambda_k I, started from the k-th FP32 Schur
//      vector) refine each vector to an eigenvector;
//   3. Gram-Schmidt, applied twice, orthonormalises them in Schur order, so
//      that span(q_1..q_k) is invariant under A for every k and
//      T = Q^T A Q is upper triangular up to rounding.
// The result is accepted only when every entry of T below the diagonal is at
// most 64 eps ||A||_F and everything is finite; those entries are then set
// to zero (the triangular solves of the sweeps test for exact zeros).  On
// false (a complex pair, close or defective eigenvalues, no FP32
// convergence) the caller runs the FP64 Francis iteration instead.
template <int BS>
__host__ __device__ inline bool schur_eigvec(const double (&A)[BS][BS], double (&Q)[BS][BS], double (&T)[BS][BS]) {
  float Hf[BS][BS], Zf[BS][BS];
  double anorm2 = 0.0;
  for (int r = 0; r < BS; ++r)
    for (int c = 0; c < BS; ++c) {
      Hf[r][c] = (float)A[r][c];
      Zf[r][c] = (r == c) ? 1.0f : 0.0f;
      anorm2 += A[r][c] * A[r][c];
    }
  hessenberg_reduce<BS>(Hf, Zf);
  if (!schur_real<BS>(Hf, Zf)) return false;
  const double eps = 2.220446049250313e-16;
  const double anorm = sqrt(anorm2);
  for (int k = 0; k < BS; ++k) {
    // LU of M = A - lambda_k I with partial pivoting (row order in perm)
    const double lam = (double)Hf[k][k];
    double M[BS][BS], inv[BS];
    int perm[BS];
    for (int r = 0; r < BS; ++r) {
      perm[r] = r;
      for (int c = 0; c < BS; ++c) M[r][c] = A[r][c] - ((r == c) ? lam : 0.0);
    }
    for (int j = 0; j < BS; ++j) {
      int piv = j;
      for (int r = j + 1; r < BS; ++r)
        if (fabs(M[r][j]) > fabs(M[piv][j])) piv = r;
      if (piv != j) {
        for (int c = 0; c < BS; ++c) {
          const double t = M[j][c];
          M[j][c] = M[piv][c];
          M[piv][c] = t;
        }
        const int t = perm[j];
        perm[j] = perm[piv];
        perm[piv] = t;
      }
      const double d = (M[j][j] != 0.0) ? M[j][j] : eps * anorm;  // an exact eigenvalue: a tiny pivot
      inv[j] = 1.0 / d;
      for (int r = j + 1; r < BS; ++r) {
        const double f = M[r][j] * inv[j];
        M[r][j] = f;
        for (int c = j + 1; c < BS; ++c) M[r][c] -= f * M[j][c];
      }
    }
    // x <- M^{-1} x / ||M^{-1} x||, twice
    double x[BS];
    for (int r = 0; r < BS; ++r) x[r] = (double)Zf[r][k];
    for (int it = 0; it < 2; ++it) {
      double y[BS];
      for (int r = 0; r < BS; ++r) {
        double t = x[perm[r]];
        for (int c = 0; c < r; ++c) t -= M[r][c] * y[c];
        y[r] = t;
      }
      for (int r = BS - 1; r >= 0; --r) {
        double t = y[r];
        for (int c = r + 1; c < BS; ++c) t -= M[r][c] * y[c];
        y[r] = t * inv[r];
      }
      double nn = 0.0;
      for (int r = 0; r < BS; ++r) nn += y[r] * y[r];
      nn = 1.0 / sqrt(nn);
      for (int r = 0; r < BS; ++r) x[r] = y[r] * nn;
    }
    for (int r = 0; r < BS; ++r) Q[r][k] = x[r];
  }
  for (int pass = 0; pass < 2; ++pass)
    for (int c = 0; c < BS; ++c) {
      for (int d = 0; d < c; ++d) {
        double t = 0.0;
        for (int r = 0; r < BS; ++r) t += Q[r][d] * Q[r][c];
        for (int r = 0; r < BS; ++r) Q[r][c] -= t * Q[r][d];
      }
      double nn = 0.0;
      for (int r = 0; r < BS; ++r) nn += Q[r][c] * Q[r][c];
      nn = 1.0 / sqrt(nn);
      for (int r = 0; r < BS; ++r) Q[r][c] *= nn;
    }
  // T = Q^T (A Q) and the acceptance test
  double AQ[BS][BS];
  for (int r = 0; r < BS; ++r)
    for (int c = 0; c < BS; ++c) {
      double t = 0.0;
      for (int m = 0; m < BS; ++m) t += A[r][m] * Q[m][c];
      AQ[r][c] = t;
    }
  const double lim = 64.0 * eps * anorm;
  bool ok = true;
  for (int r = 0; r < BS; ++r)
    for (int c = 0; c < BS; ++c) {
      double t = 0.0;
      for (int m = 0; m < BS; ++m) t += Q[m][r] * AQ[m][c];
      T[r][c] = t;
      ok = ok && (fabs(t) <= 1e300) && (fabs(Q[r][c]) <= 2.0) && (r <= c || fabs(t) <= lim);
    }
  if (!ok) return false;
  for (int r = 1; r < BS; ++r)
    for (int c = 0; c < r; ++c) T[r][c] = 0.0;
  return true;
}

}  // namespace fnlh
