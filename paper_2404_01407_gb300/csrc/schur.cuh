// Real Schur form of a small upper Hessenberg matrix (FP64, host and device).
//
// Implicit double-shift QR (Francis) with deflation, written for the
// per-node diagonal blocks of the sweeps: H <- Z^T H Z with Z accumulating
// every reflection, until H is upper triangular.  2 x 2 blocks with real
// eigenvalues are split by one rotation; a block with a complex pair makes
// the routine report failure (the caller then keeps the Hessenberg form).
#pragma once

#include <math.h>

namespace fnlh {

// Householder reduction to upper Hessenberg form: P <- Q^T P Q, Q <- Q Q_k.
template <int BS>
__host__ __device__ inline void hessenberg_reduce(double (&P)[BS][BS], double (&Q)[BS][BS]) {
  for (int k = 0; k < BS - 2; ++k) {
    double v[BS];
    double alpha2 = 0.0;
    for (int r = 0; r < BS; ++r) {
      v[r] = (r > k) ? P[r][k] : 0.0;
      alpha2 += v[r] * v[r];
    }
    if (alpha2 == 0.0) continue;
    const double alpha = sqrt(alpha2);
    v[k + 1] += (v[k + 1] >= 0.0) ? alpha : -alpha;
    double vn2 = 0.0;
    for (int r = 0; r < BS; ++r) vn2 += v[r] * v[r];
    if (vn2 == 0.0) continue;
    const double beta = 2.0 / vn2;
    for (int c = 0; c < BS; ++c) {  // P <- (I - beta v v^T) P
      double t = 0.0;
      for (int r = 0; r < BS; ++r) t += v[r] * P[r][c];
      t *= beta;
      for (int r = 0; r < BS; ++r) P[r][c] -= t * v[r];
    }
    for (int r = 0; r < BS; ++r) {  // P <- P (I - beta v v^T),  Q <- Q (I - beta v v^T)
      double t = 0.0, u = 0.0;
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
    for (int r = k + 2; r < BS; ++r) P[r][k] = 0.0;
  }
}

template <int BS>
__host__ __device__ inline void schur_rotate(double (&H)[BS][BS], double (&Z)[BS][BS], int r, double cs, double sn,
                                             int col_lo, int row_hi) {
  // rows r, r+1 (from the left, G^T) over columns col_lo..BS-1
  for (int c = col_lo; c < BS; ++c) {
    const double a = H[r][c], b = H[r + 1][c];
    H[r][c] = cs * a + sn * b;
    H[r + 1][c] = -sn * a + cs * b;
  }
  // columns r, r+1 (from the right, G) over rows 0..row_hi, and Z
  for (int q = 0; q <= row_hi; ++q) {
    const double a = H[q][r], b = H[q][r + 1];
    H[q][r] = cs * a + sn * b;
    H[q][r + 1] = -sn * a + cs * b;
  }
  for (int q = 0; q < BS; ++q) {
    const double a = Z[q][r], b = Z[q][r + 1];
    Z[q][r] = cs * a + sn * b;
    Z[q][r + 1] = -sn * a + cs * b;
  }
}

// Returns true when H was brought to upper triangular form (all eigenvalues
// real); on false, H and Z hold a partially reduced (still valid) similarity.
template <int BS>
__host__ __device__ inline bool schur_real(double (&H)[BS][BS], double (&Z)[BS][BS]) {
  const double eps = 2.220446049250313e-16;
  double anorm = 0.0;
  for (int r = 0; r < BS; ++r)
    for (int c = 0; c < BS; ++c) anorm += fabs(H[r][c]);
  if (anorm == 0.0) return true;
  int hi = BS - 1, its = 0, total = 0;
  while (hi >= 1) {
    if (++total > 40 * BS) return false;
    int l = hi;
    for (; l > 0; --l) {
      double s = fabs(H[l - 1][l - 1]) + fabs(H[l][l]);
      if (s == 0.0) s = anorm;
      if (fabs(H[l][l - 1]) <= eps * s) {
        H[l][l - 1] = 0.0;
        break;
      }
    }
    if (l == hi) {  // one eigenvalue converged
      --hi;
      its = 0;
      continue;
    }
    if (l == hi - 1) {  // trailing 2 x 2 block
      const double a = H[hi - 1][hi - 1], b = H[hi - 1][hi], c = H[hi][hi - 1], d = H[hi][hi];
      const double p = 0.5 * (a - d);
      const double disc = p * p + b * c;
      if (disc < 0.0) return false;  // complex conjugate pair
      const double lam = d + p + copysign(sqrt(disc), p);
      // eigenvector of the block for lam, from its better-scaled row
      double u0, u1;
      if (fabs(lam - d) + fabs(c) >= fabs(b) + fabs(lam - a)) {
        u0 = lam - d;
        u1 = c;
      } else {
        u0 = b;
        u1 = lam - a;
      }
      const double un = sqrt(u0 * u0 + u1 * u1);
      if (un > 0.0) {
        schur_rotate<BS>(H, Z, hi - 1, u0 / un, u1 / un, hi - 1, hi);
      }
      H[hi][hi - 1] = 0.0;
      hi -= 2;
      its = 0;
      continue;
    }
    // double-shift QR sweep on the active window l..hi
    ++its;
    double s, t;
    if (its % 10 == 0) {  // exceptional shift
      const double x = fabs(H[hi][hi - 1]) + fabs(H[hi - 1][hi - 2]);
      s = 1.5 * x;
      t = x * x;
    } else {
      s = H[hi - 1][hi - 1] + H[hi][hi];
      t = H[hi - 1][hi - 1] * H[hi][hi] - H[hi - 1][hi] * H[hi][hi - 1];
    }
    double x = H[l][l] * H[l][l] + H[l][l + 1] * H[l + 1][l] - s * H[l][l] + t;
    double y = H[l + 1][l] * (H[l][l] + H[l + 1][l + 1] - s);
    double z = H[l + 1][l] * H[l + 2][l + 1];
    for (int k = l; k <= hi - 2; ++k) {
      // reflector (I - beta v v^T) taking (x, y, z) onto the first axis
      const double alpha = sqrt(x * x + y * y + z * z);
      if (alpha != 0.0) {
        const double v0 = x + copysign(alpha, x), v1 = y, v2 = z;
        const double beta = 2.0 / (v0 * v0 + v1 * v1 + v2 * v2);
        const int c_lo = (k == l) ? l : k - 1;
        for (int c = c_lo; c < BS; ++c) {
          const double w = beta * (v0 * H[k][c] + v1 * H[k + 1][c] + v2 * H[k + 2][c]);
          H[k][c] -= w * v0;
          H[k + 1][c] -= w * v1;
          H[k + 2][c] -= w * v2;
        }
        const int r_hi = (k + 3 < hi) ? k + 3 : hi;
        for (int q = 0; q <= r_hi; ++q) {
          const double w = beta * (H[q][k] * v0 + H[q][k + 1] * v1 + H[q][k + 2] * v2);
          H[q][k] -= w * v0;
          H[q][k + 1] -= w * v1;
          H[q][k + 2] -= w * v2;
        }
        for (int q = 0; q < BS; ++q) {
          const double w = beta * (Z[q][k] * v0 + Z[q][k + 1] * v1 + Z[q][k + 2] * v2);
          Z[q][k] -= w * v0;
          Z[q][k + 1] -= w * v1;
          Z[q][k + 2] -= w * v2;
        }
        if (k > l) {
          H[k + 1][k - 1] = 0.0;
          H[k + 2][k - 1] = 0.0;
        }
      }
      x = H[k + 1][k];
      y = H[k + 2][k];
      z = (k < hi - 2) ? H[k + 3][k] : 0.0;
    }
    // closing rotation on rows / columns hi-1, hi
    {
      const double r = sqrt(x * x + y * y);
      if (r != 0.0) {
        schur_rotate<BS>(H, Z, hi - 1, x / r, y / r, hi - 2, hi);
        H[hi][hi - 2] = 0.0;
      }
    }
  }
  for (int r = 1; r < BS; ++r)
    for (int c = 0; c < r; ++c) H[r][c] = 0.0;
  return true;
}

}  // namespace fnlh
