// Per-(node, system) body of the block-Jacobi sweep, shared by the single-row
// and the batched multi-row kernels.
#pragma once

#include "common.cuh"

namespace fnlh {

// x_i <- (H_i + i omega_k V_i I)^-1 (B~_i - sum_j J~_ij x_j) for the columns of
// system k (column 0 for the mean flow, 2k-1 / 2k for harmonic k), all in the
// per-node Hessenberg basis.  The mean flow goes through the same complex
// code with a zero imaginary part, so every lane of a warp runs the same
// instructions.
template <int BS, typename TJ, typename T>
__device__ __forceinline__ void sweep_pair(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                                           const TJ* __restrict__ offd, const T* __restrict__ hess,
                                           const double* __restrict__ vol, const T* __restrict__ Bt,
                                           const T* __restrict__ Xin, T* __restrict__ Xout, int C, int i, int k,
                                           double omega_k, bool x_zero) {
  const int c0 = (k == 0) ? 0 : 2 * k - 1;
  const bool cplx = k > 0;
  T sr[BS], si[BS];
  const T* bi = Bt + ((size_t)i * C + c0) * BS;
#pragma unroll
  for (int r = 0; r < BS; ++r) {
    sr[r] = bi[r];
    si[r] = cplx ? bi[BS + r] : T(0);
  }
  if (!x_zero) {
    const int p0 = __ldg(row_ptr + i), p1 = __ldg(row_ptr + i + 1);
    for (int p = p0; p < p1; ++p) {
      const int j = __ldg(col_idx + p);
      const T* xj = Xin + ((size_t)j * C + c0) * BS;
      T xr[BS], xi[BS];
#pragma unroll
      for (int t = 0; t < BS; ++t) {
        xr[t] = xj[t];
        xi[t] = cplx ? xj[BS + t] : T(0);
      }
      const TJ* J = offd + (size_t)p * BS * BS;
#pragma unroll
      for (int r = 0; r < BS; ++r)
#pragma unroll
        for (int t = 0; t < BS; ++t) {
          const T jv = ld<T>(J + r * BS + t);
          sr[r] -= jv * xr[t];
          si[r] -= jv * xi[t];
        }
    }
  }
  const T s = (T)(omega_k * __ldg(vol + i));
  hess_solve<BS, T>(hess + (size_t)i * BS * BS, s, sr, si);
  T* xo = Xout + ((size_t)i * C + c0) * BS;
#pragma unroll
  for (int r = 0; r < BS; ++r) {
    xo[r] = sr[r];
    if (cplx) xo[BS + r] = si[r];
  }
}

}  // namespace fnlh
