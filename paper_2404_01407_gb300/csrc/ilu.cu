// Block ILU(0) smoother in multicolour order.
//
// Paper: arXiv 2404.01407, "Generalized RK Scheme" -- the implicit LHS of
// every RK stage (mean flow and each harmonic, Eq. lhs_mean / Eq. lhs_lin) is
// inverted approximately by ILU(0) iterations, stopped by the linear-residual
// rule of Table fnlh_para; on a parallel run each partition is factored on its
// own (the couplings between partitions are ignored).
//
// Design (GB300): the nodes are ordered by colour (no two neighbours share a
// colour), so every triangular solve is a short sequence of fully parallel
// colour passes.  On a pattern without triangles (three pairwise adjacent
// nodes -- none in a hexahedral edge graph) block ILU(0) changes only the
// pivot blocks: with P_i = A_ii - sum_{j earlier} A_ij P_j^-1 A_ji the factors
// are L_ij = A_ij P_j^-1 and U_ij = A_ij, so the library stores just P_i^-1
// per node and system, and the shared J supplies every off-diagonal block.
// One iteration x <- x + (LU)^-1 r, r = B - A x (FP64, every coupling):
//   forward, colours ascending:   z_i = P_i^-1 (r_i - sum_{j earlier} A_ij z_j)
//   backward, colours descending: y_i = z_i - P_i^-1 sum_{j later} A_ij y_j,
//                                 x_i += y_i
// with A_ij carrying the phase-lag factor of periodic entries.  An edge's two
// couplings carry opposite phases, so the pivots do not depend on them.
//
// Precision: the FP64 smoother works in the original basis on J's FP64
// blocks.  The FP32 smoother works in the per-node Schur basis of the sweeps
// (x = Q x~), on the prep blob's FP32 rotated blocks: ILU(0) in pivot form is
// invariant under that block-diagonal orthogonal change of basis (by
// induction P~_i = Q_i^T P_i Q_i), so it is the same smoother, while every
// block is read in FP32 without conversions; the FP64 residual is rotated to
// FP32 on the fly and the correction is added back as x += Q e (product in
// FP32, sum in FP64) -- the defect-correction pattern of the mixed sweeps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace fnlh {

constexpr int kIluThreads = 128;
constexpr int kPivotThreads = 32;

int residual_launch(const fnlh_mesh* m, const fnlh_jacobian* J, const Systems& sys, const double* B,
                    const double* X, double* r, float* r32rot, const float* rotf, int x_zero, double* norms, void* ws,
                    cudaStream_t s);
Systems make_systems(int n_harm, const double* omega, const double* sigma);
int mark_sweeps_begin(cudaStream_t s);
int mark_sweeps_end(cudaStream_t s);
int update_f32(int n, int K, int BS, const float* rotf, const float* e, double* X, cudaStream_t s,
               float2* xff = nullptr);
int residual_ff_launch(const fnlh_mesh* m, const fnlh_jacobian* J, const Systems& sys, const float2* bff,
                       const float2* xff, float* r32rot, const float* rotf, double* norms, void* ws, cudaStream_t s);
int split_ff(long long count, const double* v, float2* out, cudaStream_t s);

// ------------------------------------------------------------- validation

// Bit 0: two neighbours share a colour or a colour is out of range; bit 1: the
// (truncated) pattern has a triangle; bit 2: `order` is not a permutation
// grouped by colour.
__global__ void k_ilu_check_graph(int32_t n, int32_t n_colors, const int32_t* __restrict__ row_ptr,
                                  const int32_t* __restrict__ cols, const int32_t* __restrict__ color,
                                  int32_t* __restrict__ flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int ci = color[i];
  int f = (ci < 0 || ci >= n_colors) ? 1 : 0;
  const int p0 = row_ptr[i], p1 = row_ptr[i + 1];
  for (int p = p0; p < p1; ++p) {
    const int c = cols[p];
    if (cut_of(c)) continue;
    const int j = col_of(c);
    if (color[j] == ci) f |= 1;
    if (j < i) continue;  // each edge once
    for (int q = row_ptr[j]; q < row_ptr[j + 1]; ++q) {
      const int d = cols[q];
      if (cut_of(d)) continue;
      const int k = col_of(d);
      if (k == i) continue;
      for (int t = p0; t < p1; ++t)
        if (!cut_of(cols[t]) && col_of(cols[t]) == k) f |= 2;
    }
  }
  if (f) atomicOr(flags, f);
}

// Counts the appearances of every node in order[begin, end) and checks their colour.
__global__ void k_ilu_check_order(int32_t n, int32_t begin, int32_t end, int32_t c, const int32_t* __restrict__ order,
                                  const int32_t* __restrict__ color, int32_t* __restrict__ seen,
                                  int32_t* __restrict__ flags) {
  const int t = begin + blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= end) return;
  const int i = order[t];
  if (i < 0 || i >= n || color[i] != c) {
    atomicOr(flags, 4);
    return;
  }
  atomicAdd(seen + i, 1);
}

__global__ void k_ilu_check_seen(int32_t n, const int32_t* __restrict__ seen, int32_t* __restrict__ flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && seen[i] != 1) atomicOr(flags, 4);
}

// -------------------------------------------------------------- factor

struct IluArgs {
  int32_t n, K, begin, end;
  const int32_t* order;
  const int32_t* color;
  const int32_t* row_ptr;
  const int32_t* cols;  // tagged column indices (col_of / side_of / cut_of)
  const double* offd;   // J_ij, original basis (FP64 smoother)
  const int32_t* info;  // prep info word, nullable: 0 = the b = 6 frozen-turbulence pattern holds
  const double* diag;
  const double* D;
  const double* vol;
  const float* offd32;  // Q_i^T J_ij Q_j in FP32 (FP32 smoother)
  const double* hess;   // Q_i^T (J_ii + D_i I) Q_i (FP32 smoother)
  const float* r32;     // Q^T r in FP32, internal FP32 layout (FP32 smoother)
  void* factor;         // [n][b*b][K] complex inverse pivots (T), systems innermost
  const double* r;      // [n][C][b] residual, caller layout
  void* E;              // work vector (T), internal layout of T (common.cuh, node_stride)
  double* X;            // [n][C][b] iterate, caller layout
  int32_t* status;      // bit 1: a zero pivot
  int32_t masked;
  int32_t last;         // forward pass over the top colour: y = z there, so it also updates x (FP64)
  uint64_t active[2];
  Systems sys;
};

__device__ __forceinline__ bool ilu_active(const IluArgs& a, int k) {
  return !a.masked || ((a.active[k >> 6] >> (k & 63)) & 1ull);
}

// Position of column i in row j (the transposed coupling), -1 if absent.
__device__ __forceinline__ int find_in_row(const int32_t* row_ptr, const int32_t* cols, int j, int i) {
  for (int q = row_ptr[j]; q < row_ptr[j + 1]; ++q)
    if (col_of(cols[q]) == i) return q;
  return -1;
}

// Factor entry e (row-major in the block) of node i, system k: the systems of
// one entry are adjacent, so the K threads of a node read them coalesced.
__host__ __device__ __forceinline__ size_t pivot_at(int i, int e, int k, int K, int BS) {
  return (((size_t)i * BS * BS + e) * K + k) * 2;
}

// Pivot blocks of the nodes of one colour, thread per (node, system): P in
// shared memory (complex, row-major), updated by every earlier-coloured
// neighbour j with  P -= A_ij P_j^-1 A_ji  one row at a time, then inverted by
// Gauss-Jordan elimination with partial pivoting.
template <int BS, typename T>
__global__ void __launch_bounds__(kPivotThreads) k_ilu_pivots(const __grid_constant__ IluArgs a) {
  __shared__ double sP[kPivotThreads][2 * BS * BS];
  __shared__ double sV[kPivotThreads][2 * BS * BS];
  const int t = a.begin + blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (t >= a.end) return;
  const int i = a.order[t];
  double* P = sP[threadIdx.x];
  double* V = sV[threadIdx.x];
  constexpr bool kRot = sizeof(T) == 4;  // FP32 smoother: Schur basis, D inside hess
  const double shift_re = kRot ? 0.0 : a.D[i], shift_im = a.sys.omega[k] * a.vol[i];
  for (int e = 0; e < BS * BS; ++e) {
    P[2 * e] = kRot ? a.hess[(size_t)i * BS * BS + e] : a.diag[(size_t)i * BS * BS + e];
    P[2 * e + 1] = 0.0;
  }
  for (int r = 0; r < BS; ++r) {
    P[2 * (r * BS + r)] += shift_re;
    P[2 * (r * BS + r) + 1] += shift_im;
  }
  const int ci = a.color[i];
  for (int p = a.row_ptr[i]; p < a.row_ptr[i + 1]; ++p) {
    const int c = a.cols[p];
    if (cut_of(c)) continue;
    const int j = col_of(c);
    if (a.color[j] >= ci) continue;
    const int q = find_in_row(a.row_ptr, a.cols, j, i);
    if (q < 0) continue;  // not reached on a symmetric pattern
    const size_t oij = (size_t)p * BS * BS, oji = (size_t)q * BS * BS;
    const T* F = (const T*)a.factor;
    for (int r = 0; r < BS; ++r) {
      double wr[BS], wi[BS];  // row r of A_ij P_j^-1
      for (int cc = 0; cc < BS; ++cc) {
        double sr = 0.0, si = 0.0;
        for (int u = 0; u < BS; ++u) {
          const size_t e = oij + r * BS + u;
          const double av = kRot ? (double)a.offd32[e] : a.offd[e];
          const size_t o = pivot_at(j, u * BS + cc, k, a.K, BS);
          sr += av * (double)F[o];
          si += av * (double)F[o + 1];
        }
        wr[cc] = sr;
        wi[cc] = si;
      }
      for (int cc = 0; cc < BS; ++cc) {
        double sr = 0.0, si = 0.0;
        for (int u = 0; u < BS; ++u) {
          const size_t e = oji + u * BS + cc;
          const double av = kRot ? (double)a.offd32[e] : a.offd[e];
          sr += wr[u] * av;
          si += wi[u] * av;
        }
        P[2 * (r * BS + cc)] -= sr;
        P[2 * (r * BS + cc) + 1] -= si;
      }
    }
  }
  // V = P^-1 by Gauss-Jordan elimination with partial pivoting (|.|^2 compare)
  for (int e = 0; e < BS * BS; ++e) {
    V[2 * e] = (e / BS == e % BS) ? 1.0 : 0.0;
    V[2 * e + 1] = 0.0;
  }
  bool ok = true;
  for (int col = 0; col < BS; ++col) {
    int piv = col;
    double best = P[2 * (col * BS + col)] * P[2 * (col * BS + col)] +
                  P[2 * (col * BS + col) + 1] * P[2 * (col * BS + col) + 1];
    for (int r = col + 1; r < BS; ++r) {
      const double m2 = P[2 * (r * BS + col)] * P[2 * (r * BS + col)] + P[2 * (r * BS + col) + 1] * P[2 * (r * BS + col) + 1];
      if (m2 > best) {
        best = m2;
        piv = r;
      }
    }
    if (!(best > 0.0)) {
      ok = false;
      break;
    }
    if (piv != col)
      for (int cc = 0; cc < BS; ++cc)
        for (int h = 0; h < 2; ++h) {
          double tp = P[2 * (col * BS + cc) + h];
          P[2 * (col * BS + cc) + h] = P[2 * (piv * BS + cc) + h];
          P[2 * (piv * BS + cc) + h] = tp;
          tp = V[2 * (col * BS + cc) + h];
          V[2 * (col * BS + cc) + h] = V[2 * (piv * BS + cc) + h];
          V[2 * (piv * BS + cc) + h] = tp;
        }
    // scale the pivot row by 1 / p
    const double pr = P[2 * (col * BS + col)], pi = P[2 * (col * BS + col) + 1];
    const double inv = 1.0 / (pr * pr + pi * pi);
    const double qr = pr * inv, qi = -pi * inv;
    for (int cc = 0; cc < BS; ++cc) {
      double xr = P[2 * (col * BS + cc)], xi = P[2 * (col * BS + cc) + 1];
      P[2 * (col * BS + cc)] = xr * qr - xi * qi;
      P[2 * (col * BS + cc) + 1] = xr * qi + xi * qr;
      xr = V[2 * (col * BS + cc)];
      xi = V[2 * (col * BS + cc) + 1];
      V[2 * (col * BS + cc)] = xr * qr - xi * qi;
      V[2 * (col * BS + cc) + 1] = xr * qi + xi * qr;
    }
    for (int r = 0; r < BS; ++r) {
      if (r == col) continue;
      const double fr = P[2 * (r * BS + col)], fi = P[2 * (r * BS + col) + 1];
      for (int cc = 0; cc < BS; ++cc) {
        P[2 * (r * BS + cc)] -= fr * P[2 * (col * BS + cc)] - fi * P[2 * (col * BS + cc) + 1];
        P[2 * (r * BS + cc) + 1] -= fr * P[2 * (col * BS + cc) + 1] + fi * P[2 * (col * BS + cc)];
        V[2 * (r * BS + cc)] -= fr * V[2 * (col * BS + cc)] - fi * V[2 * (col * BS + cc) + 1];
        V[2 * (r * BS + cc) + 1] -= fr * V[2 * (col * BS + cc) + 1] + fi * V[2 * (col * BS + cc)];
      }
    }
  }
  if (!ok) atomicOr(a.status, 2);
  T* F = (T*)a.factor;
  for (int e = 0; e < BS * BS; ++e) {
    const size_t o = pivot_at(i, e, k, a.K, BS);
    F[o] = ok ? (T)V[2 * e] : T(0);
    F[o + 1] = ok ? (T)V[2 * e + 1] : T(0);
  }
}

// --------------------------------------------------------------- apply

// s -= A_ij e^{i side sigma} y_j (kSubtract) or s += ... for one neighbour
// slice (complex, T), accumulated straight into s.
template <int BS, typename T, bool kSubtract>
__device__ __forceinline__ void ilu_gather(const IluArgs& a, int p, int cj, int k, T (&sr)[BS], T (&si)[BS]) {
  const int j = col_of(cj);
  const T* yj = (const T*)a.E + slice_at<BS, T>(j, a.K, k);
  const bool real = real_mean<T>(a.K) && k == 0;  // a real mean flow
  T xr[BS], xi[BS];
#pragma unroll
  for (int t = 0; t < BS; ++t) {
    xr[t] = real ? yj[mean_pos<BS>(t)] : yj[2 * t];
    xi[t] = real ? T(0) : yj[2 * t + 1];
  }
  if (side_of(cj)) phase_shift<BS, T>(xr, xi, side_of(cj), a.sys.phase[k]);
  // FP64, b = 6 with frozen turbulence: rows 0..4 of the original-basis
  // block skip their structurally zero column 5
  bool pattern = false;
  if constexpr (BS == 6 && sizeof(T) == 8) pattern = a.info != nullptr && __ldg(a.info) == 0;
  if (pattern) {
#pragma unroll
    for (int r = 0; r < BS; ++r)
#pragma unroll
      for (int t = 0; t < ((r < BS - 1) ? BS - 1 : BS); ++t) {
        const T av = __ldg(a.offd + (size_t)p * BS * BS + r * BS + t);
        if constexpr (kSubtract) {
          sr[r] -= av * xr[t];
          si[r] -= av * xi[t];
        } else {
          sr[r] += av * xr[t];
          si[r] += av * xi[t];
        }
      }
    return;
  }
#pragma unroll
  for (int r = 0; r < BS; ++r)
#pragma unroll
    for (int t = 0; t < BS; ++t) {
      T av;
      if constexpr (sizeof(T) == 4) av = __ldg(a.offd32 + (size_t)p * BS * BS + r * BS + t);
      else av = __ldg(a.offd + (size_t)p * BS * BS + r * BS + t);
      if constexpr (kSubtract) {
        sr[r] -= av * xr[t];
        si[r] -= av * xi[t];
      } else {
        sr[r] += av * xr[t];
        si[r] += av * xi[t];
      }
    }
}

template <typename T> struct Cplx2;
template <> struct Cplx2<double> { using type = double2; };
template <> struct Cplx2<float> { using type = float2; };

// (yr, yi) = P_i^-1 (sr, si), complex; F points at the factor of node i,
// system k (entry stride 2K values).
template <int BS, typename T>
__device__ __forceinline__ void ilu_pivot_apply(const T* __restrict__ F, int K, const T (&sr)[BS], const T (&si)[BS],
                                                T (&yr)[BS], T (&yi)[BS]) {
  using V2 = typename Cplx2<T>::type;
#pragma unroll
  for (int r = 0; r < BS; ++r) {
    T ar = 0, ai = 0;
#pragma unroll
    for (int t = 0; t < BS; ++t) {
      const V2 p = __ldg(reinterpret_cast<const V2*>(F + (size_t)(r * BS + t) * 2 * K));
      ar += p.x * sr[t] - p.y * si[t];
      ai += p.x * si[t] + p.y * sr[t];
    }
    yr[r] = ar;
    yi[r] = ai;
  }
}

// One system's slice of the work vector in the internal layout (common.cuh,
// node_stride): complex pairs, or for a real mean flow its values (the pivot
// of the real system gives a zero imaginary part) and the pad.
template <int BS, typename T>
__device__ __forceinline__ void store_e(T* __restrict__ e, bool real, const T (&yr)[BS], const T (&yi)[BS]) {
  if (real) {
#pragma unroll
    for (int q = 0; q < BS; ++q) e[mean_pos<BS>(q)] = yr[q];
    for (int t = 0; t < kMeanSlot<BS>; ++t)
      if (mean_pad<BS>(t)) e[t] = T(0);
    return;
  }
#pragma unroll
  for (int q = 0; q < BS; ++q) {
    e[2 * q] = yr[q];
    e[2 * q + 1] = yi[q];
  }
}

// Forward pass over one colour: z_i = P_i^-1 (r_i - sum_{j earlier} A_ij z_j).
// The top colour has no later neighbours, so its backward pass would only
// copy y_i = z_i: in FP64 this pass adds it to x_i instead, and the
// backward passes start one colour lower.
template <int BS, typename T>
__global__ void __launch_bounds__(kIluThreads) k_ilu_forward(const __grid_constant__ IluArgs a) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long t = a.begin + g / a.K;
  const int k = (int)(g % a.K);
  if (t >= a.end) return;
  const int i = a.order[t];
  if (!ilu_active(a, k)) {  // a frozen system: no correction
    T* e = (T*)a.E + slice_at<BS, T>(i, a.K, k);
    const int len = slice_len<BS, T>(a.K, k);
#pragma unroll
    for (int q = 0; q < 2 * BS; ++q)
      if (q < len) e[q] = T(0);
    return;
  }
  T sr[BS], si[BS];
  if constexpr (sizeof(T) == 4) {
    const float* rp = a.r32 + slice_at<BS, float>(i, a.K, k);
#pragma unroll
    for (int q = 0; q < BS; ++q) {
      sr[q] = real_mean<float>(a.K) && k == 0 ? rp[mean_pos<BS>(q)] : rp[2 * q];
      si[q] = real_mean<float>(a.K) && k == 0 ? 0.0f : rp[2 * q + 1];
    }
  } else {
    const int c0 = (k == 0) ? 0 : 2 * k - 1;
    const double* rp = a.r + ((size_t)i * a.sys.C + c0) * BS;
#pragma unroll
    for (int q = 0; q < BS; ++q) {
      sr[q] = rp[q];
      si[q] = (k == 0) ? 0.0 : rp[BS + q];
    }
  }
  const int ci = a.color[i];
  for (int p = a.row_ptr[i]; p < a.row_ptr[i + 1]; ++p) {
    const int cj = a.cols[p];
    if (cut_of(cj) || a.color[col_of(cj)] >= ci) continue;
    ilu_gather<BS, T, true>(a, p, cj, k, sr, si);
  }
  T yr[BS], yi[BS];
  ilu_pivot_apply<BS, T>((const T*)a.factor + pivot_at(i, 0, k, a.K, BS), a.K, sr, si, yr, yi);
  store_e<BS, T>((T*)a.E + slice_at<BS, T>(i, a.K, k), real_mean<T>(a.K) && k == 0, yr, yi);
  if constexpr (sizeof(T) == 8) {  // FP32: x += Q e after the passes
    if (a.last) {
      double* xp = a.X + ((size_t)i * a.sys.C + ((k == 0) ? 0 : 2 * k - 1)) * BS;
#pragma unroll
      for (int q = 0; q < BS; ++q) {
        xp[q] += yr[q];
        if (k > 0) xp[BS + q] += yi[q];
      }
    }
  }
}

// Backward pass over one colour: y_i = z_i - P_i^-1 sum_{j later} A_ij y_j,
// then x_i += y_i (the update, in FP64, in the caller's layout).
template <int BS, typename T>
__global__ void __launch_bounds__(kIluThreads) k_ilu_backward(const __grid_constant__ IluArgs a) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long t = a.begin + g / a.K;
  const int k = (int)(g % a.K);
  if (t >= a.end || !ilu_active(a, k)) return;
  const int i = a.order[t];
  const int ci = a.color[i];
  T sr[BS], si[BS];
#pragma unroll
  for (int q = 0; q < BS; ++q) {
    sr[q] = 0;
    si[q] = 0;
  }
  bool any = false;
  for (int p = a.row_ptr[i]; p < a.row_ptr[i + 1]; ++p) {
    const int cj = a.cols[p];
    if (cut_of(cj) || a.color[col_of(cj)] <= ci) continue;
    ilu_gather<BS, T, false>(a, p, cj, k, sr, si);
    any = true;
  }
  T* e = (T*)a.E + slice_at<BS, T>(i, a.K, k);
  const bool real = real_mean<T>(a.K) && k == 0;  // a real mean flow
  T yr[BS], yi[BS];
#pragma unroll
  for (int q = 0; q < BS; ++q) {
    yr[q] = real ? e[mean_pos<BS>(q)] : e[2 * q];
    yi[q] = real ? T(0) : e[2 * q + 1];
  }
  if (any) {
    T dr[BS], di[BS];
    ilu_pivot_apply<BS, T>((const T*)a.factor + pivot_at(i, 0, k, a.K, BS), a.K, sr, si, dr, di);
#pragma unroll
    for (int q = 0; q < BS; ++q) {
      yr[q] -= dr[q];
      yi[q] -= di[q];
    }
    store_e<BS, T>(e, real, yr, yi);
  }
  if constexpr (sizeof(T) == 8) {  // FP32: x += Q e after the passes
    double* xp = a.X + ((size_t)i * a.sys.C + ((k == 0) ? 0 : 2 * k - 1)) * BS;
#pragma unroll
    for (int q = 0; q < BS; ++q) {
      xp[q] += yr[q];
      if (k > 0) xp[BS + q] += yi[q];
    }
  }
}

// ----------------------------------------------------------------- host

static inline unsigned grid_for(long long count, int threads) { return (unsigned)((count + threads - 1) / threads); }

static IluArgs ilu_args(const fnlh_mesh* m, const fnlh_jacobian* J, const fnlh_ilu* ilu, const Systems& sys) {
  IluArgs a;
  std::memset(&a, 0, sizeof(a));
  if (ilu->precision == FNLH_F32) {  // rotated FP32 blocks and the FP64 Schur factor
    const PrepLayout L = prep_layout(J->n_nodes, J->nnz, J->block, J->prep_flags);
    a.offd32 = at<float>(J->prep, L.offd32);
    a.hess = at<double>(J->prep, L.hess);
  }
  a.n = m->n_nodes;
  a.K = sys.K;
  a.order = ilu->order;
  a.color = ilu->color;
  a.row_ptr = m->row_ptr;
  a.cols = csr_columns(m, J);
  a.offd = J->offd;
  a.info = prep_info(J);
  a.diag = J->diag;
  a.D = J->D;
  a.vol = m->vol;
  a.factor = ilu->factor;
  a.sys = sys;
  a.active[0] = a.active[1] = ~0ull;
  return a;
}

template <int BS, typename T>
static int factor_typed(const fnlh_mesh* m, const fnlh_jacobian* J, const Systems& sys, fnlh_ilu* ilu, void* ws,
                        cudaStream_t s) {
  const int n = m->n_nodes;
  const WsLayout W = ws_layout(n, BS, sys.K - 1, FNLH_F64);
  int32_t* flags = at<int32_t>(ws, W.status);
  int32_t* seen = at<int32_t>(ws, W.vec[0]);
  FNLH_CUDA_TRY(cudaMemsetAsync(flags, 0, 2 * sizeof(int32_t), s));
  FNLH_CUDA_TRY(cudaMemsetAsync(seen, 0, sizeof(int32_t) * (size_t)std::max(n, 1), s));
  IluArgs a = ilu_args(m, J, ilu, sys);
  a.status = flags + 1;
  if (n > 0) {
    k_ilu_check_graph<<<grid_for(n, 128), 128, 0, s>>>(n, ilu->n_colors, m->row_ptr, a.cols, ilu->color, flags);
    FNLH_LAUNCH_CHECK();
    for (int c = 0; c < ilu->n_colors; ++c) {
      const int b = ilu->color_ptr[c], e = ilu->color_ptr[c + 1];
      if (e > b) {
        k_ilu_check_order<<<grid_for(e - b, 128), 128, 0, s>>>(n, b, e, c, ilu->order, ilu->color, seen, flags);
        FNLH_LAUNCH_CHECK();
      }
    }
    k_ilu_check_seen<<<grid_for(n, 128), 128, 0, s>>>(n, seen, flags);
    FNLH_LAUNCH_CHECK();
  }
  int32_t hflags = 0;
  FNLH_CUDA_TRY(cudaMemcpyAsync(&hflags, flags, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FNLH_CUDA_TRY(cudaStreamSynchronize(s));
  if (hflags & (1 | 4)) return FNLH_ERR_BAD_MESH;
  if (hflags & 2) return FNLH_ERR_UNSUPPORTED;
  for (int c = 0; c < ilu->n_colors; ++c) {
    a.begin = ilu->color_ptr[c];
    a.end = ilu->color_ptr[c + 1];
    if (a.end <= a.begin) continue;
    dim3 grid(grid_for(a.end - a.begin, kPivotThreads), sys.K);
    k_ilu_pivots<BS, T><<<grid, kPivotThreads, 0, s>>>(a);
    FNLH_LAUNCH_CHECK();
  }
  int32_t hstatus = 0;
  FNLH_CUDA_TRY(cudaMemcpyAsync(&hstatus, flags + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FNLH_CUDA_TRY(cudaStreamSynchronize(s));
  if (hstatus) return FNLH_ERR_NONFINITE;
  ilu->n_harm = sys.K - 1;
  ilu->ready = 1;
  return FNLH_OK;
}

int ilu_factor_impl(const fnlh_mesh* m, const fnlh_jacobian* J, int n_harm, const double* omega, fnlh_ilu* ilu,
                    void* ws, cudaStream_t s) {
  const Systems sys = make_systems(n_harm, omega, nullptr);
  if (J->block == 5)
    return ilu->precision == FNLH_F64 ? factor_typed<5, double>(m, J, sys, ilu, ws, s)
                                      : factor_typed<5, float>(m, J, sys, ilu, ws, s);
  return ilu->precision == FNLH_F64 ? factor_typed<6, double>(m, J, sys, ilu, ws, s)
                                    : factor_typed<6, float>(m, J, sys, ilu, ws, s);
}

struct IluCheck {
  double rel[kMaxSys];
  double first_max;
};

template <int BS, typename T>
static int solve_ilu_typed(const fnlh_mesh* m, const fnlh_jacobian* J, const fnlh_ilu* ilu, const Systems& sys,
                           const double* B, double* X, double tol, int max_iterations, int flags, void* ws,
                           int* iterations_done, double* rel_res, cudaStream_t s) {
  const int n = m->n_nodes, K = sys.K;
  const WsLayout W = ws_layout(n, BS, K - 1, FNLH_F64);
  double* norms = at<double>(ws, W.norms);
  double* r = at<double>(ws, W.vec[0]);
  constexpr bool kRot = sizeof(T) == 4;
  const float* rotf = nullptr;
  if (kRot) {
    const PrepLayout L = prep_layout(J->n_nodes, J->nnz, J->block, J->prep_flags);
    rotf = at<float>(J->prep, L.rotf);
  }
  IluArgs a = ilu_args(m, J, ilu, sys);
  a.r = r;
  a.r32 = (const float*)r;
  a.E = at<T>(ws, W.vec[1]);
  a.X = X;
  a.status = at<int32_t>(ws, W.status);
  const bool masking = (flags & FNLH_SOLVE_MASK_CONVERGED) != 0;
  bool x_zero = (flags & FNLH_SOLVE_ZERO_GUESS) != 0;
  if (x_zero) FNLH_CUDA_TRY(cudaMemsetAsync(X, 0, sizeof(double) * (size_t)n * sys.C * BS, s));
  // Float-float checks (FP32 smoother, prep blob with FNLH_PREP_FF), as in
  // fnlh_solve: every residual after the first on the FP32 units
  // from float-float shadows of B and x, a passing one confirmed at once in
  // FP64, and one that the decay predicts at or below 2 tol made in FP64
  // directly.  The shadows take the workspace's third vector and pivot-table
  // slots, which this solve does not use otherwise (each holds n C b float2).
  const PrepLayout PL = prep_layout(J->n_nodes, J->nnz, J->block, J->prep_flags);
  const bool ff = kRot && n > 0 && PL.offdff != (size_t)-1;
  float2* bff = ff ? at<float2>(ws, W.vec[2]) : nullptr;
  float2* xff = ff ? at<float2>(ws, W.pivinv) : nullptr;
  int it = 0, rc = FNLH_OK;
  if (ff) {
    const long long nv = (long long)n * sys.C * BS;
    if ((rc = split_ff(nv, B, bff, s))) return rc;
    if (x_zero) FNLH_CUDA_TRY(cudaMemsetAsync(xff, 0, sizeof(float2) * (size_t)nv, s));
    else if ((rc = split_ff(nv, X, xff, s))) return rc;
  }
  double hn[2 * kMaxSys], bnorm[kMaxSys] = {};
  IluCheck ck;
  ck.first_max = 0.0;
  bool conv = false, fp64_next = false;
  double prev_worst = -1.0;
  // the relative residuals of hn into ck.rel; returns the worst, or -1 on a non-finite value
  auto evaluate = [&]() -> double {
    double worst = 0.0;
    for (int k = 0; k < K; ++k) {
      const double rr = hn[2 * k], bb = hn[2 * k + 1];
      if (!(rr == rr) || !(bb == bb) || rr > 1e300 || bb > 1e300) return -1.0;
      ck.rel[k] = (bb > 0.0) ? std::sqrt(rr / bb) : std::sqrt(rr);
      worst = std::max(worst, ck.rel[k]);
    }
    return worst;
  };
  for (;;) {
    bool need64 = true;
    if (ff && it > 0 && !fp64_next) {
      if ((rc = residual_ff_launch(m, J, sys, bff, xff, (float*)r, rotf, norms, ws, s))) return rc;
      FNLH_CUDA_TRY(cudaMemcpyAsync(hn, norms, sizeof(double) * 2 * K, cudaMemcpyDeviceToHost, s));
      FNLH_CUDA_TRY(cudaStreamSynchronize(s));
      for (int k = 0; k < K; ++k) hn[2 * k + 1] = bnorm[k];
      const double w = evaluate();
      need64 = !(w >= 0.0) || w <= tol;
    }
    if (need64) {
      // FP64: r in the caller's layout; FP32: Q^T r in FP32 straight from the residual kernel
      if ((rc = residual_launch(m, J, sys, B, X, kRot ? nullptr : r, kRot ? (float*)r : nullptr, rotf,
                                x_zero ? 1 : 0, norms, ws, s)))
        return rc;
      x_zero = false;
      FNLH_CUDA_TRY(cudaMemcpyAsync(hn, norms, sizeof(double) * 2 * K, cudaMemcpyDeviceToHost, s));
      FNLH_CUDA_TRY(cudaStreamSynchronize(s));
      if (it == 0)
        for (int k = 0; k < K; ++k) bnorm[k] = hn[2 * k + 1];
    }
    const double worst = evaluate();
    if (!(worst >= 0.0)) {
      rc = FNLH_ERR_NONFINITE;
      break;
    }
    if (it == 0) ck.first_max = worst;
    else if (worst > 1e3 * std::max(ck.first_max, 1e-300)) {
      rc = FNLH_ERR_DIVERGED;
      break;
    }
    conv = worst <= tol;
    if (conv || it >= max_iterations) break;
    if (ff) {  // does the decay predict the next check at or below 2 tol?  Then make it in FP64.
      fp64_next = prev_worst > 0.0 && worst * worst / prev_worst <= 2.0 * tol;
      prev_worst = worst;
    }
    if (masking) {
      a.masked = 1;
      for (int k = 0; k < K; ++k)
        if (ck.rel[k] <= tol) a.active[k >> 6] &= ~(1ull << (k & 63));
    }
    if ((rc = mark_sweeps_begin(s))) return rc;
    for (int c = 0; c < ilu->n_colors; ++c) {
      a.begin = ilu->color_ptr[c];
      a.end = ilu->color_ptr[c + 1];
      a.last = (c == ilu->n_colors - 1) ? 1 : 0;
      if (a.end <= a.begin) continue;
      k_ilu_forward<BS, T><<<grid_for((long long)(a.end - a.begin) * K, kIluThreads), kIluThreads, 0, s>>>(a);
      FNLH_LAUNCH_CHECK();
    }
    a.last = 0;
    for (int c = ilu->n_colors - 2; c >= 0; --c) {  // the top colour's y = z is final
      a.begin = ilu->color_ptr[c];
      a.end = ilu->color_ptr[c + 1];
      if (a.end <= a.begin) continue;
      k_ilu_backward<BS, T><<<grid_for((long long)(a.end - a.begin) * K, kIluThreads), kIluThreads, 0, s>>>(a);
      FNLH_LAUNCH_CHECK();
    }
    if ((rc = mark_sweeps_end(s))) return rc;
    if (kRot && (rc = update_f32(n, K, BS, rotf, (const float*)a.E, X, s, xff))) return rc;
    ++it;
  }
  if (iterations_done) *iterations_done = it;
  if (rel_res)
    for (int k = 0; k < K; ++k) rel_res[k] = ck.rel[k];
  if (rc) return rc;
  return conv ? FNLH_OK : FNLH_ERR_NOT_CONVERGED;
}

int solve_ilu_impl(const fnlh_mesh* m, const fnlh_jacobian* J, const fnlh_ilu* ilu, int n_harm, const double* omega,
                   const double* sigma, const double* B, double* X, double tol, int max_iterations, int flags,
                   void* ws, int* iterations_done, double* rel_res, cudaStream_t s) {
  const Systems sys = make_systems(n_harm, omega, sigma);
#define FNLH_ILU_SOLVE(BS, T) \
  solve_ilu_typed<BS, T>(m, J, ilu, sys, B, X, tol, max_iterations, flags, ws, iterations_done, rel_res, s)
  if (J->block == 5) return ilu->precision == FNLH_F64 ? FNLH_ILU_SOLVE(5, double) : FNLH_ILU_SOLVE(5, float);
  return ilu->precision == FNLH_F64 ? FNLH_ILU_SOLVE(6, double) : FNLH_ILU_SOLVE(6, float);
#undef FNLH_ILU_SOLVE
}

}  // namespace fnlh
