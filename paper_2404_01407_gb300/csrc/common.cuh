// Internal helpers of the FNLH CUDA library (sm_103a).  Not part of the ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fnlh.h"

namespace fnlh {

constexpr int kMaxSys = FNLH_MAX_HARMONICS + 1;  // mean + harmonics
constexpr int kResidualGrid = 1216;               // fixed grid of the residual kernels (deterministic sums)
constexpr int kResidualThreads = 256;

// Per-launch system description passed by value (omega baked into the launch).
struct Systems {
  int32_t K;             // systems = 1 + N
  int32_t C;             // real columns = 1 + 2N
  double omega[kMaxSys]; // omega[0] = 0 (mean), omega[l] harmonic l
  double2 phase[kMaxSys];  // (cos, sin) of the inter-blade phase angle; phase[0] = (1, 0)
};

// Column entries of a tagged mesh (the prep blob's copy of col_idx) carry the
// neighbour's blade passage in their top two bits -- 1 = the next passage
// (factor e^{+i sigma_k} on x_j), 2 = the previous one (e^{-i sigma_k}) -- and
// in bit 29 whether the neighbour lies in another partition (a coupling the
// sweeps drop and the residual keeps).
constexpr uint32_t kColMask = 0x1fffffffu;
constexpr uint32_t kSideNext = 1u, kSidePrev = 2u;
constexpr uint32_t kCutBit = 1u << 29;
__host__ __device__ __forceinline__ int col_of(int c) { return (int)((uint32_t)c & kColMask); }
__host__ __device__ __forceinline__ uint32_t side_of(int c) { return (uint32_t)c >> 30; }
__host__ __device__ __forceinline__ bool cut_of(int c) { return ((uint32_t)c & kCutBit) != 0; }

// x <- e^{+-i sigma} x for a neighbour across the periodic boundary (side
// kSideNext: +, kSidePrev: -), ph = (cos sigma, sin sigma).
template <int BS, typename T>
__device__ __forceinline__ void phase_shift(T (&re)[BS], T (&im)[BS], uint32_t side, double2 ph) {
  const T c = (T)ph.x, s = (side == kSideNext) ? (T)ph.y : -(T)ph.y;
#pragma unroll
  for (int t = 0; t < BS; ++t) {
    const T a = re[t], b = im[t];
    re[t] = c * a - s * b;
    im[t] = s * a + c * b;
  }
}

// ------------------------------------------------ internal vector layout
//
// Iterates and right-hand sides of the sweeps, in the rotated basis, per node
// the systems' slices one after another: complex (re, im) pairs, the mean
// flow (k = 0) with a zero imaginary part -- except for FP32 vectors of few
// systems per node (K <= kRealMeanMaxSystems), where the mean flow keeps its
// b real values alone (order: mean_pos), padded to kMeanSlot<BS> floats.
// There the zero imaginary part would be a large share of the bytes (a
// quarter at K = 2), and one thread carries all of a node's systems
// (k_sweep_f32_node); with more systems the stored zeros cost less than the
// selects the thread-per-(node, system) kernels would need.  The pad keeps
// every slice on the alignment of its vector loads: 16 bytes for b = 6, 8
// bytes for b = 5.
constexpr int kRealMeanMaxSystems = 2;

template <int BS>
constexpr int kMeanSlot = ((2 * BS) % 4 == 0) ? (BS + 3) / 4 * 4 : (BS + 1) / 2 * 2;

// Position of the mean flow's real value t in its FP32 slot: the first
// kMeanSlot/2 values on the even positions, where a harmonic's slice keeps
// its real parts, the rest on the odd positions from 1; the slot's other
// positions hold zeros.
template <int BS>
__host__ __device__ constexpr int mean_pos(int t) {
  return t < kMeanSlot<BS> / 2 ? 2 * t : 2 * (t - kMeanSlot<BS> / 2) + 1;
}

// Is slot position e of the FP32 mean flow a pad (zero)?
template <int BS>
__host__ __device__ constexpr bool mean_pad(int e) {
  return (e & 1) ? (e >> 1) >= BS - kMeanSlot<BS> / 2 : false;
}

// Does a vector of type T with K systems per node keep the mean flow real?
template <typename T>
__host__ __device__ __forceinline__ bool real_mean(int K) {
  return sizeof(T) == 4 && K <= kRealMeanMaxSystems;
}

template <int BS, typename T>
__host__ __device__ __forceinline__ size_t node_stride(int K) {
  return real_mean<T>(K) ? (size_t)kMeanSlot<BS> + (size_t)(K - 1) * 2 * BS : (size_t)K * 2 * BS;
}

template <int BS, typename T>
__host__ __device__ __forceinline__ size_t sys_offset(int K, int k) {
  if (!real_mean<T>(K)) return (size_t)k * 2 * BS;
  return k == 0 ? 0 : (size_t)kMeanSlot<BS> + (size_t)(k - 1) * 2 * BS;
}

// element offset of system k's slice of node i
template <int BS, typename T>
__host__ __device__ __forceinline__ size_t slice_at(size_t i, int K, int k) {
  return i * node_stride<BS, T>(K) + sys_offset<BS, T>(K, k);
}

// values stored for system k's slice: kMeanSlot for a real mean flow, else 2b
template <int BS, typename T>
__host__ __device__ __forceinline__ int slice_len(int K, int k) {
  return (real_mean<T>(K) && k == 0) ? kMeanSlot<BS> : 2 * BS;
}

// ------------------------------------------------------------------ loads

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ double to_d(double x) { return x; }
template <typename T> __device__ __forceinline__ T cvt(double x);
template <> __device__ __forceinline__ double cvt<double>(double x) { return x; }
template <> __device__ __forceinline__ float cvt<float>(double x) { return (float)x; }

template <typename TACC, typename T> __device__ __forceinline__ TACC ld(const T* p);
template <> __device__ __forceinline__ double ld<double, double>(const double* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld<float, float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld<float, __nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}
template <> __device__ __forceinline__ float ld<float, double>(const double* p) { return (float)__ldg(p); }

// Reciprocal: exact IEEE division in FP64; in FP32 (the inner sweeps of the
// defect correction, whose result is corrected in FP64 anyway) the
// hardware approximation, within 2 ulp.
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }

// Division by a small runtime constant d without an integer divide:
// q = (n * m) >> s with m = ceil(2^s / d), s = 31 + ceil(log2 d); exact for
// every n < 2^31 (the rounding error of m is below 2^-l <= 1/d per unit of n/2^31).
struct FastDiv {
  uint32_t d, m, s;
};
inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  uint32_t l = 0;
  while ((1u << l) < d) ++l;
  f.d = d;
  f.s = 31 + l;
  f.m = (uint32_t)(((1ull << f.s) + d - 1) / d);
  return f;
}
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
  return (uint32_t)(((uint64_t)n * f.m) >> f.s);
}

// 1 / m_q for q = 0..BS-1 with a single division: prefix products, one
// reciprocal of the full product, then one multiply-back per entry
// (simultaneous inversion, Montgomery 1987).  In FP64 a division is a
// multi-instruction sequence on the scarce FP64 units, so BS of them per
// solve are worth folding into one.  The m_q are pivots of a nonsingular
// block (|m_q| well inside 1e+-50, so the product stays in range).
template <int BS>
__device__ __forceinline__ void batch_recip(const double (&m)[BS], double (&inv)[BS]) {
  double pre[BS];
  pre[0] = m[0];
#pragma unroll
  for (int q = 1; q < BS; ++q) pre[q] = pre[q - 1] * m[q];
  double r = 1.0 / pre[BS - 1];
#pragma unroll
  for (int q = BS - 1; q > 0; --q) {
    inv[q] = r * pre[q - 1];
    r *= m[q];
  }
  inv[0] = r;
}

// ----------------------------------------------- shifted Hessenberg solve
//
// Solve (H + i s I) y = b for an upper Hessenberg H (row-major BS x BS,
// entries below the subdiagonal are not read) and a real shift s, by
// Gaussian elimination with partial pivoting between the two candidate rows
// of each step (the only rows with a nonzero entry in the pivot column).
// (yr, yi) holds b on entry and y on return.  Cost O(BS^2) complex
// operations instead of the O(BS^3) of a general block LU.  H may point to
// global or shared memory (plain loads).
// pivinv (nullable, FP64): per row k the precomputed pair
// (d_k, s) / (d_k^2 + s^2) of this block and shift, so that
// y_k = (a_r alpha_k + a_i beta_k) + i (a_i alpha_k - a_r beta_k) needs no
// division and two fewer multiplies.
template <int BS, typename T, typename TH>
__device__ __forceinline__ void hess_solve(const TH* __restrict__ H, T s, T (&yr)[BS], T (&yi)[BS],
                                           const T* __restrict__ pivinv = nullptr) {
  // Triangular factor (real Schur form, every subdiagonal exactly zero):
  // plain back-substitution, y_k = (b_k - sum_{c>k} T_kc y_c) / (T_kk + i s).
  bool tri = true;
#pragma unroll
  for (int k = 0; k < BS - 1; ++k) tri = tri && (H[(k + 1) * BS + k] == TH(0));
  if (tri && pivinv) {
#pragma unroll
    for (int k = BS - 1; k >= 0; --k) {
      T ar = yr[k], ai = yi[k];
#pragma unroll
      for (int c = k + 1; c < BS; ++c) {
        const T t = (T)H[k * BS + c];
        ar -= t * yr[c];
        ai -= t * yi[c];
      }
      T al, be;
      if constexpr (sizeof(T) == 8) {  // the table is 16-byte aligned: one vector load per row
        const double2 f = __ldg(reinterpret_cast<const double2*>(pivinv) + k);
        al = f.x;
        be = f.y;
      } else {
        al = pivinv[2 * k];
        be = pivinv[2 * k + 1];
      }
      yr[k] = ar * al + ai * be;
      yi[k] = ai * al - ar * be;
    }
    return;
  }
  if (tri) {
    // 1 / (d_k^2 + s^2): in FP64 one division for the whole block
    T invs[BS];
    if constexpr (sizeof(T) == 8) {
      double m[BS];
#pragma unroll
      for (int k = 0; k < BS; ++k) {
        const double d = (double)H[k * BS + k];
        m[k] = d * d + s * s;
      }
      batch_recip<BS>(m, invs);
    } else {
#pragma unroll
      for (int k = 0; k < BS; ++k) {
        const T d = (T)H[k * BS + k];
        invs[k] = recip(d * d + s * s);
      }
    }
#pragma unroll
    for (int k = BS - 1; k >= 0; --k) {
      T ar = yr[k], ai = yi[k];
#pragma unroll
      for (int c = k + 1; c < BS; ++c) {
        const T t = (T)H[k * BS + c];
        ar -= t * yr[c];
        ai -= t * yi[c];
      }
      const T d = (T)H[k * BS + k];
      yr[k] = (ar * d + ai * s) * invs[k];
      yi[k] = (ai * d - ar * s) * invs[k];
    }
    return;
  }
  // upper-triangular factor rows (complex); row k holds columns k..BS-1
  T ur[BS][BS], ui[BS][BS];
  T rr[BS], ri[BS];  // reciprocal of each pivot
  // current candidate row for position k (row 0 initially)
  T cr[BS], ci[BS], cbr, cbi;
#pragma unroll
  for (int c = 0; c < BS; ++c) {
    cr[c] = (T)H[c];
    ci[c] = (c == 0) ? s : T(0);
  }
  cbr = yr[0];
  cbi = yi[0];
#pragma unroll
  for (int k = 0; k < BS - 1; ++k) {
    // next original row k+1: columns k..BS-1
    T nr[BS], ni[BS];
#pragma unroll
    for (int c = k; c < BS; ++c) {
      nr[c] = (T)H[(k + 1) * BS + c];
      ni[c] = (c == k + 1) ? s : T(0);
    }
    T nbr = yr[k + 1], nbi = yi[k + 1];
    // pivot choice (1-norm magnitude); on the matrices of this method the
    // swap is rare, so a branch (uniform over a warp when nobody swaps) is
    // cheaper than selecting every entry
    if ((fabs(nr[k]) + fabs(ni[k])) > (fabs(cr[k]) + fabs(ci[k]))) {
#pragma unroll
      for (int c = k; c < BS; ++c) {
        const T tr = nr[c], ti = ni[c];
        nr[c] = cr[c];
        ni[c] = ci[c];
        cr[c] = tr;
        ci[c] = ti;
      }
      const T tr = nbr, ti = nbi;
      nbr = cbr;
      nbi = cbi;
      cbr = tr;
      cbi = ti;
    }
    // pivot reciprocal
    const T m2 = cr[k] * cr[k] + ci[k] * ci[k];
    const T inv = recip(m2);
    rr[k] = cr[k] * inv;
    ri[k] = -ci[k] * inv;
    // store pivot row
#pragma unroll
    for (int c = k; c < BS; ++c) {
      ur[k][c] = cr[c];
      ui[k][c] = ci[c];
    }
    yr[k] = cbr;
    yi[k] = cbi;
    // multiplier l = n_k / p
    const T lr = nr[k] * rr[k] - ni[k] * ri[k];
    const T li = nr[k] * ri[k] + ni[k] * rr[k];
    // eliminate: new candidate = n - l * c  (columns k+1..)
#pragma unroll
    for (int c = k + 1; c < BS; ++c) {
      const T ar = nr[c] - (lr * cr[c] - li * ci[c]);
      const T ai = ni[c] - (lr * ci[c] + li * cr[c]);
      cr[c] = ar;
      ci[c] = ai;
    }
    const T br = nbr - (lr * cbr - li * cbi);
    const T bi = nbi - (lr * cbi + li * cbr);
    cbr = br;
    cbi = bi;
  }
  {
    const int k = BS - 1;
    const T m2 = cr[k] * cr[k] + ci[k] * ci[k];
    const T inv = recip(m2);
    rr[k] = cr[k] * inv;
    ri[k] = -ci[k] * inv;
    yr[k] = cbr;
    yi[k] = cbi;
  }
  // back substitution
#pragma unroll
  for (int k = BS - 1; k >= 0; --k) {
    T ar = yr[k], ai = yi[k];
#pragma unroll
    for (int c = k + 1; c < BS; ++c) {
      ar -= ur[k][c] * yr[c] - ui[k][c] * yi[c];
      ai -= ur[k][c] * yi[c] + ui[k][c] * yr[c];
    }
    yr[k] = ar * rr[k] - ai * ri[k];
    yi[k] = ar * ri[k] + ai * rr[k];
  }
}

// --------------------------------------------------------- float-float
//
// A value as an unevaluated sum of two FP32 numbers, hi + lo with |lo| <=
// ulp(hi) / 2 (Dekker 1971): products and sums below are exact up to
// O(2^-44) of the magnitudes involved.  Every operation is spelled with an
// explicit rounding intrinsic so that the compiler neither fuses nor
// reassociates it.

// FP64 -> (hi, lo): hi the nearest FP32, lo the nearest FP32 to the rest.
__device__ __forceinline__ float2 ff_split(double d) {
  const float h = __double2float_rn(d);
  return make_float2(h, __double2float_rn(d - (double)h));
}

// (h, l) -= a * b for float-float a and b: the product of the high parts
// exactly (TwoProduct with one FMA), the cross terms in FP32, and the
// subtraction from the high part exactly (TwoSum, 6 additions).
__device__ __forceinline__ void ff_sub_prod(float& h, float& l, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  const float pe = __fmaf_rn(a.x, b.x, -p);                            // a.x b.x - p, exact
  const float pl = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, pe));       // the rest of the product
  const float t = __fsub_rn(h, p);
  const float z = __fsub_rn(t, h);
  const float e = __fsub_rn(__fsub_rn(h, __fsub_rn(t, z)), __fadd_rn(p, z));  // (h - p) - t, exact
  h = t;
  l = __fadd_rn(l, __fsub_rn(e, pl));
}

// (h, l) += e for an FP32 e: exact sum of the high parts (TwoSum), then
// renormalised so that |l| stays below half an ulp of h.
__device__ __forceinline__ float2 ff_add_f(float2 a, float e) {
  const float t = __fadd_rn(a.x, e);
  const float z = __fsub_rn(t, a.x);
  const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(t, z)), __fsub_rn(e, z));
  const float l = __fadd_rn(a.y, err);
  const float h = __fadd_rn(t, l);
  return make_float2(h, __fsub_rn(l, __fsub_rn(h, t)));
}

// ---------------------------------------------------------- workspace map
//
// [0, 256)                      status words (int32)
// [256, +partials)              residual partial sums  kResidualGrid x 2K doubles
// norms                         final 2K doubles of the last residual
// vec0, vec1, vec2              three vectors in the internal layout (node_stride) of the precision's type
// pivinv                        FP64 only: [n][K][b] pairs (d, s) / (d^2 + s^2) of the shifted triangular solves
struct WsLayout {
  size_t status, partials, norms, vec[3], pivinv, total, vec_bytes;
  // fnlh_solve's float-float shadows after `total` ([n][C][b] float2 each, FP32 / BF16 only):
  size_t bff, xff, total_ff;
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

inline WsLayout ws_layout(int32_t n, int32_t block, int32_t n_harm, int32_t precision) {
  WsLayout w;
  const size_t K = 1 + (size_t)n_harm;
  const size_t elem = (precision == FNLH_F64) ? 8 : 4;
  w.status = 0;
  w.partials = 256;
  w.norms = w.partials + (size_t)kResidualGrid * 2 * K * sizeof(double);
  size_t off = align256(w.norms + 2 * K * sizeof(double));
  w.vec_bytes = (size_t)n * K * 2 * block * elem;
  for (int v = 0; v < 3; ++v) {
    w.vec[v] = off;
    off = align256(off + w.vec_bytes);
  }
  w.pivinv = (size_t)-1;
  if (precision == FNLH_F64) {
    w.pivinv = off;
    off = align256(off + (size_t)n * K * block * 2 * sizeof(double));
  }
  w.total = off;
  w.bff = w.xff = (size_t)-1;
  if (precision != FNLH_F64) {
    const size_t shadow = (size_t)n * (2 * K - 1) * block * 2 * sizeof(float);
    w.bff = off;
    off = align256(off + shadow);
    w.xff = off;
    off = align256(off + shadow);
  }
  w.total_ff = off;
  return w;
}

// ----------------------------------------------------------- prep blob map
//
// rot   [n][b][b] f64   Q_i
// hess  [n][b][b] f64   Q_i^T (J_ii + D_i I) Q_i  (upper Hessenberg, zeros below)
// hessf [n][b][b] f32   (when an F32/BF16 copy is requested)
// rotf  [n][b][b] f32   Q_i in FP32 (same condition: the mixed solve's rotations)
// offd64 / offd32 / offd16 [nnz][b][b] rotated off-diagonal copies
// cols  [nnz] int32     col_idx with the passage and partition tags (FNLH_PREP_TAGS)
// info  int32 words: [0] nonzero when the blocks do NOT have the frozen-
//       turbulence zero pattern (see k_check_structure)
// offdff [nnz][b][b] float2, diagff [n][b][b] float2 (FNLH_PREP_FF): the
//       original-basis J_ij and J_ii + D_i I as float-float pairs (hi, lo)
struct PrepLayout {
  size_t info, rot, hess, hessf, rotf, offd64, offd32, offd16, cols, offdff, diagff, total;
};

inline PrepLayout prep_layout(int32_t n, int32_t nnz, int32_t b, int32_t flags) {
  PrepLayout p;
  const size_t bb = (size_t)b * b;
  size_t off = 0;
  p.info = off;
  off = 256;
  p.rot = off;
  off = align256(off + (size_t)n * bb * 8);
  p.hess = off;
  off = align256(off + (size_t)n * bb * 8);
  p.hessf = p.rotf = p.offd64 = p.offd32 = p.offd16 = p.cols = (size_t)-1;
  if (flags & (FNLH_PREP_F32 | FNLH_PREP_BF16)) {
    p.hessf = off;
    off = align256(off + (size_t)n * bb * 4);
    p.rotf = off;
    off = align256(off + (size_t)n * bb * 4);
  }
  if (flags & FNLH_PREP_F64) {
    p.offd64 = off;
    off = align256(off + (size_t)nnz * bb * 8);
  }
  if (flags & FNLH_PREP_F32) {
    p.offd32 = off;
    off = align256(off + (size_t)nnz * bb * 4);
  }
  if (flags & FNLH_PREP_BF16) {
    p.offd16 = off;
    off = align256(off + (size_t)nnz * bb * 2);
  }
  if (flags & FNLH_PREP_TAGS) {
    p.cols = off;
    off = align256(off + (size_t)nnz * 4);
  }
  p.offdff = p.diagff = (size_t)-1;
  if (flags & FNLH_PREP_FF) {
    p.offdff = off;
    off = align256(off + (size_t)nnz * bb * 8);
    p.diagff = off;
    off = align256(off + (size_t)n * bb * 8);
  }
  p.total = off;
  return p;
}

template <typename T> inline T* at(void* base, size_t off) { return reinterpret_cast<T*>((char*)base + off); }

// The prepared blob's info word, or null (no prepared blob: nothing certified).
inline const int32_t* prep_info(const fnlh_jacobian* J) {
  if (!J->prep || !J->prep_ready) return nullptr;
  return at<int32_t>(J->prep, prep_layout(J->n_nodes, J->nnz, J->block, J->prep_flags).info);
}

// The column array the sweeps and the residual read: the mesh's own, or on a
// mesh with periodic edges or partitions the tagged copy in the prep blob (the
// entry points check that it exists before anything launches).
inline bool tagged_mesh(const fnlh_mesh* m) { return m->periodic != nullptr || m->part != nullptr; }
inline const int32_t* csr_columns(const fnlh_mesh* m, const fnlh_jacobian* J) {
  if (!tagged_mesh(m)) return m->col_idx;
  const PrepLayout L = prep_layout(J->n_nodes, J->nnz, J->block, J->prep_flags);
  return at<int32_t>(J->prep, L.cols);
}

}  // namespace fnlh

#define FNLH_CUDA_TRY(expr)                       \
  do {                                            \
    cudaError_t _e = (expr);                      \
    if (_e != cudaSuccess) return FNLH_ERR_CUDA;  \
  } while (0)

#define FNLH_LAUNCH_CHECK() FNLH_CUDA_TRY(cudaGetLastError())
