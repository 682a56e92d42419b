// Fused block-Jacobi sweep over the mean flow and every harmonic.
//
// Paper: arXiv 2404.01407, "Solution Update" -- the block-diagonal inversion,
// node by node (block Jacobi), of Eq. lhs_mean / Eq. lhs_lin with
// the harmonic LHS of Eq. precon_linear, K_l = K + i omega_l V I, sharing one
// J across all systems:
//   x_i <- (J_ii + (D_i + i omega_k V_i) I)^-1 (B_i - sum_j J_ij x_j).
//
// Design (GB300): one thread per (node, system); the off-diagonal product is
// accumulated in registers and the shifted diagonal system solved in
// registers.  FP64: a CTA owns 32 nodes and each warp whole systems for them
// (the mean flow's warp runs a real-only path).  FP32/BF16: 64-pair tiles
// whose blocks are staged in shared memory when a node serves enough systems;
// with one or two systems per node, one thread per node instead
// (k_sweep_f32_node), each block loaded once for all of them.
// The sweeps run in the per-node Hessenberg basis prepared by
// fnlh_prepare (x = Q x~), where the diagonal block of system k is
// H_i + i omega_k V_i I and its solve costs O(b^2).  Iterates live in the
// internal layout (common.cuh, node_stride: complex pairs per system, the
// mean flow real in FP32 vectors of K <= 2 systems); the rotate kernels move
// between it and the caller's [n][C][b] layout.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "sweep_kernel.cuh"

namespace fnlh {

constexpr int kSweepThreads = 256;      // FP64 sweep CTA (32 nodes x up to 8 system warps)
constexpr int kSweepThreadsF32 = 64;    // FP32 sweep tile: 64 (node, system) pairs

struct SweepArgs {
  TileRow row;
  const void* Xin;
  void* Xout;
  int32_t x_zero;
  int32_t smem_floats;
  int32_t masked;   // 0: every system is swept; 1: only the systems set in `active`
  uint64_t active[2];
  double omega[kMaxSys];
  double2 phase[kMaxSys];
};

// FP64: a CTA per 32 consecutive nodes, each warp taking whole systems for
// them (system-major), so that the mean flow's warp runs the real-only path.
template <int BS>
__global__ void __launch_bounds__(kSweepThreads, 2) k_sweep_f64(const __grid_constant__ SweepArgs a) {
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  if (i >= a.row.n) return;
  const SweepIO io{a.Xin, a.Xout, a.omega, a.masked ? a.active : nullptr, a.phase};
  const int nwarps = blockDim.x >> 5;
  for (int k = threadIdx.x >> 5; k < a.row.K; k += nwarps) {
    if (sys_active(io, k)) sweep_node_f64<BS>(a.row, io, i, k, a.x_zero != 0);
    else freeze_pair<BS, double>(a.row, io, i, k, a.x_zero != 0);
  }
}

// FP32 arithmetic on FP32 or BF16 blocks, staged per CTA tile.  64 registers:
// sixteen 64-thread CTAs per SM (measured on GB300: 0.5-1.3% faster than eight
// 128-thread CTAs, and those 15% faster than 256-thread tiles at three or four
// CTAs per SM on the 2.1M-node, 9-system workload).
template <int BS, typename TJ>
__global__ void __launch_bounds__(kSweepThreadsF32, 16) k_sweep_f32(const __grid_constant__ SweepArgs a) {
  extern __shared__ __align__(16) float smem[];
  const SweepIO io{a.Xin, a.Xout, a.omega, a.masked ? a.active : nullptr, a.phase};
  sweep_tile_f32<BS, TJ>(a.row, io, (long long)blockIdx.x * blockDim.x, a.x_zero != 0, smem, a.smem_floats);
}

// ------------------------------------------- FP32, few systems per node

constexpr int kNodeThreads = 128;
constexpr int kNodeMaxSystems = kRealMeanMaxSystems;  // K up to this: one thread per node

// `COUNT` floats from a 16- (COUNT % 4 == 0) or 8-byte aligned (COUNT even) address.
template <int COUNT>
__device__ __forceinline__ void load_floats(const float* __restrict__ p, float (&v)[COUNT]) {
  if constexpr (COUNT % 4 == 0) {
#pragma unroll
    for (int q = 0; q < COUNT / 4; ++q) {
      const float4 f = __ldg(reinterpret_cast<const float4*>(p) + q);
      v[4 * q] = f.x;
      v[4 * q + 1] = f.y;
      v[4 * q + 2] = f.z;
      v[4 * q + 3] = f.w;
    }
  } else {
    static_assert(COUNT % 2 == 0, "node slices are padded to an even length");
#pragma unroll
    for (int q = 0; q < COUNT / 2; ++q) {
      const float2 f = __ldg(reinterpret_cast<const float2*>(p) + q);
      v[2 * q] = f.x;
      v[2 * q + 1] = f.y;
    }
  }
}

template <int COUNT>
__device__ __forceinline__ void store_floats(float* __restrict__ p, const float (&v)[COUNT]) {
  if constexpr (COUNT % 4 == 0) {
#pragma unroll
    for (int q = 0; q < COUNT / 4; ++q)
      reinterpret_cast<float4*>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else {
#pragma unroll
    for (int q = 0; q < COUNT / 2; ++q) reinterpret_cast<float2*>(p)[q] = make_float2(v[2 * q], v[2 * q + 1]);
  }
}

// One whole BS x BS block as raw words, issued as one batch of the widest
// loads its alignment allows (block p starts at p * BS^2 * sizeof(TJ) bytes).
template <int BS, typename TJ>
struct RawBlock {
  static constexpr int kBytes = BS * BS * (int)sizeof(TJ);
  static constexpr int kWords = (kBytes + 3) / 4;
  uint32_t w[kWords];
  __device__ __forceinline__ void load(const TJ* __restrict__ blk) {
    if constexpr (kBytes % 16 == 0) {
#pragma unroll
      for (int q = 0; q < kBytes / 16; ++q) {
        const uint4 f = __ldg(reinterpret_cast<const uint4*>(blk) + q);
        w[4 * q] = f.x;
        w[4 * q + 1] = f.y;
        w[4 * q + 2] = f.z;
        w[4 * q + 3] = f.w;
      }
    } else if constexpr (kBytes % 8 == 0) {
#pragma unroll
      for (int q = 0; q < kBytes / 8; ++q) {
        const uint2 f = __ldg(reinterpret_cast<const uint2*>(blk) + q);
        w[2 * q] = f.x;
        w[2 * q + 1] = f.y;
      }
    } else if constexpr (kBytes % 4 == 0) {
#pragma unroll
      for (int q = 0; q < kWords; ++q) w[q] = __ldg(reinterpret_cast<const uint32_t*>(blk) + q);
    } else {  // BF16 with odd BS: 2-byte alignment only
      const uint16_t* h = reinterpret_cast<const uint16_t*>(blk);
#pragma unroll
      for (int q = 0; q < kWords; ++q) {
        const uint32_t lo = __ldg(h + 2 * q);
        const uint32_t hi = (2 * q + 1 < BS * BS) ? (uint32_t)__ldg(h + 2 * q + 1) : 0u;
        w[q] = lo | (hi << 16);
      }
    }
  }
  // entry e of the row-major block, as FP32
  __device__ __forceinline__ float at(int e) const {
    if constexpr (sizeof(TJ) == 2) return (e & 1) ? bf16_hi(w[e >> 1]) : bf16_lo(w[e >> 1]);
    else return __uint_as_float(w[e]);
  }
};

// A node's FP32 slices (the mean flow's padded reals, then (re, im) pairs)
// into one complex vector per system, the mean flow's imaginary part zero.
template <int BS, int KS, int V>
__device__ __forceinline__ void unpack_node(const float (&v)[V], Cvec<BS, float> (&c)[KS]) {
#pragma unroll
  for (int t = 0; t < BS; ++t) {
    c[0].re[t] = v[mean_pos<BS>(t)];
    c[0].im[t] = 0.0f;
  }
#pragma unroll
  for (int k = 1; k < KS; ++k)
#pragma unroll
    for (int t = 0; t < BS; ++t) {
      c[k].re[t] = v[kMeanSlot<BS> + (k - 1) * 2 * BS + 2 * t];
      c[k].im[t] = v[kMeanSlot<BS> + (k - 1) * 2 * BS + 2 * t + 1];
    }
}

// FP32 arithmetic for few systems per node (K <= kNodeMaxSystems, vectors
// with a real mean flow: common.cuh, real_mean): one
// thread per node carries every system, so each off-diagonal block is loaded
// once, whole, and applied from registers to the mean flow's real column and
// to every harmonic's (re, im) pair -- instead of each of the node's K
// threads loading it row by row.  Per system the operations and their order
// are those of the thread-per-(node, system) tile (sweep_tile_f32), so the
// two kernels give the same values.
template <int BS, typename TJ, int KS>
__global__ void __launch_bounds__(kNodeThreads) k_sweep_f32_node(const __grid_constant__ SweepArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const TileRow& R = a.row;
  if (i >= R.n) return;
  constexpr int M = kMeanSlot<BS>;
  constexpr int V = M + (KS - 1) * 2 * BS;  // floats of one node's slices
  const SweepIO io{a.Xin, a.Xout, a.omega, a.masked ? a.active : nullptr, a.phase};
  const bool x_zero = a.x_zero != 0;
  Cvec<BS, float> s[KS];
  {
    float v[V];
    load_floats<V>((const float*)R.Bt + (size_t)i * V, v);
    unpack_node<BS, KS>(v, s);
  }
  if (!x_zero) {
    const float* __restrict__ X = (const float*)io.Xin;
    const int p0 = __ldg(R.row_ptr + i), p1 = __ldg(R.row_ptr + i + 1);
    for (int p = p0; p < p1; ++p) {
      const int cj = __ldg(R.col_idx + p);
      if (cut_of(cj)) continue;  // coupling to another partition: dropped
      float v[V];
      load_floats<V>(X + (size_t)col_of(cj) * V, v);
      RawBlock<BS, TJ> J;
      J.load((const TJ*)R.offd + (size_t)p * BS * BS);
      Cvec<BS, float> x[KS];
      unpack_node<BS, KS>(v, x);
      if (side_of(cj)) {
#pragma unroll
        for (int k = 0; k < KS; ++k) phase_shift<BS, float>(x[k].re, x[k].im, side_of(cj), io.phase[k]);
      }
#pragma unroll
      for (int r = 0; r < BS; ++r)
#pragma unroll
        for (int t = 0; t < BS; ++t) {
          const float jv = J.at(r * BS + t);
#pragma unroll
          for (int k = 0; k < KS; ++k) {
            s[k].re[r] -= jv * x[k].re[t];
            if (k > 0) s[k].im[r] -= jv * x[k].im[t];  // the mean flow's stays zero
          }
        }
    }
  }
  const float* H = (const float*)R.hess + (size_t)i * BS * BS;
  const double vol = __ldg(R.vol + i);
  const float* xin = (const float*)io.Xin + (size_t)i * V;
  float out[V];
#pragma unroll
  for (int k = 0; k < KS; ++k) {
    const int o = (k == 0) ? 0 : M + (k - 1) * 2 * BS;
    if (sys_active(io, k)) {
      hess_solve<BS, float>(H, (float)(io.omega[k] * vol), s[k].re, s[k].im);
#pragma unroll
      for (int t = 0; t < BS; ++t) {
        if (k == 0) {
          out[mean_pos<BS>(t)] = s[0].re[t];
        } else {
          out[o + 2 * t] = s[k].re[t];
          out[o + 2 * t + 1] = s[k].im[t];
        }
      }
      if (k == 0) {
#pragma unroll
        for (int e = 0; e < M; ++e)
          if (mean_pad<BS>(e)) out[e] = 0.0f;
      }
    } else {  // a frozen (converged) system keeps its iterate
      const int len = (k == 0) ? M : 2 * BS;
#pragma unroll
      for (int t = 0; t < 2 * BS; ++t)
        if (t < len) out[o + t] = x_zero ? 0.0f : xin[o + t];
    }
  }
  store_floats<V>((float*)io.Xout + (size_t)i * V, out);
}

// Caller layout [n][C][b] (FP64) -> internal layout, y = Q_i^T x,
// one thread per (node, system).
template <int BS, typename TO>
__global__ void __launch_bounds__(256) k_rotate_in(long long count, int K, const double* __restrict__ rot,
                                                   const double* __restrict__ x, TO* __restrict__ y) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= count) return;
  const long long i = g / K;
  const int k = (int)(g - i * K);
  const int C = 2 * K - 1;
  const double* Q = rot + i * BS * BS;
  const double* xr = x + (i * C + (k == 0 ? 0 : 2 * k - 1)) * BS;
  double vr[BS], vi[BS];
#pragma unroll
  for (int t = 0; t < BS; ++t) {
    vr[t] = xr[t];
    vi[t] = (k == 0) ? 0.0 : xr[BS + t];
  }
  TO* out = y + slice_at<BS, TO>(i, K, k);
  const bool real = real_mean<TO>(K) && k == 0;  // a real mean flow: its values, then the pad
#pragma unroll
  for (int r = 0; r < BS; ++r) {
    double ar = 0.0, ai = 0.0;
#pragma unroll
    for (int t = 0; t < BS; ++t) {
      const double q = __ldg(Q + t * BS + r);
      ar += q * vr[t];
      ai += q * vi[t];
    }
    if (real) {
      out[mean_pos<BS>(r)] = (TO)ar;
    } else {
      out[2 * r] = (TO)ar;
      out[2 * r + 1] = (TO)ai;
    }
  }
  if (real)
    for (int e = 0; e < kMeanSlot<BS>; ++e)
      if (mean_pad<BS>(e)) out[e] = TO(0);
}

// Internal layout -> caller layout (FP64), x (+)= Q_i y.
template <int BS, typename TI>
__global__ void __launch_bounds__(256) k_rotate_out(long long count, int K, const double* __restrict__ rot,
                                                    const TI* __restrict__ y, double* __restrict__ x, int accumulate) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= count) return;
  const long long i = g / K;
  const int k = (int)(g - i * K);
  const int C = 2 * K - 1;
  const double* Q = rot + i * BS * BS;
  const TI* in = y + slice_at<BS, TI>(i, K, k);
  const bool real = real_mean<TI>(K) && k == 0;  // a real mean flow
  double vr[BS], vi[BS];
#pragma unroll
  for (int t = 0; t < BS; ++t) {
    vr[t] = (double)(real ? in[mean_pos<BS>(t)] : in[2 * t]);
    vi[t] = real ? 0.0 : (double)in[2 * t + 1];
  }
  double* xr = x + (i * C + (k == 0 ? 0 : 2 * k - 1)) * BS;
#pragma unroll
  for (int r = 0; r < BS; ++r) {
    double ar = accumulate ? xr[r] : 0.0, ai = 0.0;
    if (k > 0 && accumulate) ai = xr[BS + r];
#pragma unroll
    for (int t = 0; t < BS; ++t) {
      const double q = __ldg(Q + r * BS + t);
      ar += q * vr[t];
      ai += q * vi[t];
    }
    xr[r] = ar;
    if (k > 0) xr[BS + r] = ai;
  }
}

// x_i[c] += Q_i y_i[c] with the product in FP32 and the sum in FP64: the
// defect-correction update, whose correction only needs FP32 accuracy.
// xff (nullable): the float-float shadow of x, advanced by the same FP32
// correction in float-float arithmetic (no FP64 conversion per value).
template <int BS>
__global__ void __launch_bounds__(256) k_update_f32(long long count, int K, const float* __restrict__ rotf,
                                                    const float* __restrict__ y, double* __restrict__ x,
                                                    float2* __restrict__ xff = nullptr) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= count) return;
  const long long i = g / K;
  const int k = (int)(g - i * K);
  const int C = 2 * K - 1;
  const float* Q = rotf + i * BS * BS;
  const float* in = y + slice_at<BS, float>(i, K, k);
  const bool real = real_mean<float>(K) && k == 0;  // a real mean flow
  float vr[BS], vi[BS];
#pragma unroll
  for (int t = 0; t < BS; ++t) {
    vr[t] = real ? in[mean_pos<BS>(t)] : in[2 * t];
    vi[t] = real ? 0.0f : in[2 * t + 1];
  }
  // All loads of the read-modify-write are issued before any store, so one
  // memory round trip covers the whole update of this (node, system).
  const long long row0 = i * C + (k == 0 ? 0 : 2 * k - 1);
  double* xr = x + row0 * BS;
  const int nrow = k == 0 ? BS : 2 * BS;
  double xo[2 * BS];
  float2 fo[2 * BS];
#pragma unroll
  for (int t = 0; t < 2 * BS; ++t) {
    if (t < nrow) {
      xo[t] = xr[t];
      if (xff) fo[t] = xff[row0 * BS + t];
    }
  }
#pragma unroll
  for (int r = 0; r < BS; ++r) {
    float ar = 0.0f, ai = 0.0f;
#pragma unroll
    for (int t = 0; t < BS; ++t) {
      const float q = __ldg(Q + r * BS + t);
      ar += q * vr[t];
      ai += q * vi[t];
    }
    xr[r] = xo[r] + (double)ar;
    if (xff) xff[row0 * BS + r] = ff_add_f(fo[r], ar);
    if (k > 0) {
      xr[BS + r] = xo[BS + r] + (double)ai;
      if (xff) xff[row0 * BS + BS + r] = ff_add_f(fo[BS + r], ai);
    }
  }
}

// v -> (hi, lo) FP32 pairs: the float-float shadows of B and x.
__global__ void __launch_bounds__(256) k_split_vec(long long count, const double* __restrict__ v,
                                                   float2* __restrict__ out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) out[e] = ff_split(v[e]);
}

// Host side of k_split_vec (csrc/ilu.cu: the FP32 ILU(0) solve's float-float checks).
int split_ff(long long count, const double* v, float2* out, cudaStream_t s) {
  if (count <= 0) return FNLH_OK;
  k_split_vec<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(count, v, out);
  FNLH_LAUNCH_CHECK();
  return FNLH_OK;
}

static inline unsigned blocks_for(long long count, int threads) {
  return (unsigned)((count + threads - 1) / threads);
}

struct PivotArgs {
  long long count;  // n K
  int32_t K;
  const double* hess;
  const double* vol;
  double* out;      // [n][K][b] pairs
  double omega[kMaxSys];
};

// Pivot factors of every (node, system) triangular solve, once per call: the
// sweeps then divide nowhere (an FP64 division is a multi-instruction
// sequence on GB300's scarce FP64 units).  Mean flow: (1 / d_q, 0); harmonic
// k: (d_q, s) / (d_q^2 + s^2), s = omega_k V_i, d_q the diagonal of the
// Schur factor, so that 1 / (d_q + i s) = alpha - i beta.
template <int BS>
__global__ void __launch_bounds__(256) k_pivot_inverses(const __grid_constant__ PivotArgs a) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.count) return;
  const long long i = g / a.K;
  const int k = (int)(g - i * a.K);
  const double s = a.omega[k] * a.vol[i];
#pragma unroll
  for (int q = 0; q < BS; ++q) {
    const double d = a.hess[(size_t)i * BS * BS + q * BS + q];
    double al, be;
    if (k == 0) {
      al = 1.0 / d;
      be = 0.0;
    } else {
      const double inv = 1.0 / (d * d + s * s);
      al = d * inv;
      be = s * inv;
    }
    reinterpret_cast<double2*>(a.out)[(size_t)g * BS + q] = make_double2(al, be);
  }
}

template <int BS>
static int pivot_inverses(const fnlh_mesh* m, const double* hess, const Systems& sys, double* out, cudaStream_t s) {
  PivotArgs a;
  a.count = (long long)m->n_nodes * sys.K;
  if (a.count == 0) return FNLH_OK;
  a.K = sys.K;
  a.hess = hess;
  a.vol = m->vol;
  a.out = out;
  for (int k = 0; k < kMaxSys; ++k) a.omega[k] = sys.omega[k];
  k_pivot_inverses<BS><<<blocks_for(a.count, 256), 256, 0, s>>>(a);
  FNLH_LAUNCH_CHECK();
  return FNLH_OK;
}

template <int BS, typename TO>
int rotate_in(int n, int K, const double* rot, const double* x, TO* y, cudaStream_t s) {
  const long long count = (long long)n * K;
  if (count == 0) return FNLH_OK;
  k_rotate_in<BS, TO><<<blocks_for(count, 256), 256, 0, s>>>(count, K, rot, x, y);
  FNLH_LAUNCH_CHECK();
  return FNLH_OK;
}

template <int BS, typename TI>
int rotate_out(int n, int K, const double* rot, const TI* y, double* x, int accumulate, cudaStream_t s) {
  const long long count = (long long)n * K;
  if (count == 0) return FNLH_OK;
  k_rotate_out<BS, TI><<<blocks_for(count, 256), 256, 0, s>>>(count, K, rot, y, x, accumulate);
  FNLH_LAUNCH_CHECK();
  return FNLH_OK;
}

// Everything a sweep needs, resolved from the prep blob for one precision.
struct SweepOperands {
  const void* offd;
  const void* hess;
  const double* rot;
  const float* rotf;    // FP32 basis (low-precision sweeps only)
  const int32_t* cols;  // column indices (passage-tagged on a periodic mesh)
  const int32_t* info;  // prep info word (frozen-turbulence pattern)
};

int sweep_operands(const fnlh_mesh* m, const fnlh_jacobian* J, int precision, SweepOperands* o) {
  const PrepLayout L = prep_layout(J->n_nodes, J->nnz, J->block, J->prep_flags);
  o->cols = csr_columns(m, J);
  o->info = at<int32_t>(J->prep, L.info);
  o->rot = at<double>(J->prep, L.rot);
  o->rotf = (L.rotf != (size_t)-1) ? at<float>(J->prep, L.rotf) : nullptr;
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

Systems make_systems(int n_harm, const double* omega, const double* sigma) {
  Systems s;
  s.K = 1 + n_harm;
  s.C = 1 + 2 * n_harm;
  for (int k = 0; k < kMaxSys; ++k) {
    s.omega[k] = 0.0;
    s.phase[k] = make_double2(1.0, 0.0);
  }
  for (int k = 1; k <= n_harm; ++k) {
    s.omega[k] = omega[k - 1];
    if (sigma) s.phase[k] = make_double2(std::cos(sigma[k - 1]), std::sin(sigma[k - 1]));
  }
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

// x += Q e with the product in FP32 and the sum in FP64 (csrc/ilu.cu).
int update_f32(int n, int K, int BS, const float* rotf, const float* e, double* X, cudaStream_t s,
               float2* xff = nullptr);

// xff (nullable): the float-float shadow of X, advanced by the same correction.
int update_f32(int n, int K, int BS, const float* rotf, const float* e, double* X, cudaStream_t s, float2* xff) {
  const long long count = (long long)n * K;
  if (count == 0) return FNLH_OK;
  if (BS == 5) k_update_f32<5><<<blocks_for(count, 256), 256, 0, s>>>(count, K, rotf, e, X, xff);
  else k_update_f32<6><<<blocks_for(count, 256), 256, 0, s>>>(count, K, rotf, e, X, xff);
  FNLH_LAUNCH_CHECK();
  return FNLH_OK;
}

// The same hook for the ILU(0) passes (csrc/ilu.cu).
int mark_sweeps_begin(cudaStream_t s) { return mark(g_ev_begin, s); }
int mark_sweeps_end(cudaStream_t s) { return mark(g_ev_end, s); }

constexpr size_t kMaxStageBytes = 200 * 1024;

// Dynamic shared memory of a staged launch; tiles that need more than this
// fall back to unstaged loads inside the kernel.
template <typename KernelT>
int stage_setup(KernelT kernel, int threads, int K, int BS, int* floats, size_t* bytes) {
  size_t b = (size_t)stage_floats(threads, K, BS) * sizeof(float);
  b = std::min(b, kMaxStageBytes);
  *floats = (int)(b / sizeof(float));
  *bytes = b;
  if (b > 48 * 1024) FNLH_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b));
  return FNLH_OK;
}

template <int BS, typename TJ, typename T>
int sweep_launch(const SweepArgs& a, size_t smem_bytes, cudaStream_t s) {
  const long long count = (long long)a.row.n * a.row.K;
  if (count == 0) return FNLH_OK;
  if constexpr (sizeof(T) == 8) {
    const int warps = std::min(a.row.K, kSweepThreads / 32);
    k_sweep_f64<BS><<<(unsigned)((a.row.n + 31) / 32), 32 * warps, 0, s>>>(a);
  } else if (a.row.K <= kNodeMaxSystems) {
    const unsigned grid = blocks_for(a.row.n, kNodeThreads);
    if (a.row.K == 1) k_sweep_f32_node<BS, TJ, 1><<<grid, kNodeThreads, 0, s>>>(a);
    else k_sweep_f32_node<BS, TJ, 2><<<grid, kNodeThreads, 0, s>>>(a);
  } else {
    k_sweep_f32<BS, TJ><<<blocks_for(count, kSweepThreadsF32), kSweepThreadsF32, smem_bytes, s>>>(a);
  }
  FNLH_LAUNCH_CHECK();
  return FNLH_OK;
}

// Runs `sweeps` sweeps between the ping-pong buffers x0/x1 starting from x0
// (or from zero when x_zero), returns the buffer holding the result.
template <int BS, typename TJ, typename T>
int run_sweeps(const fnlh_mesh* m, const SweepOperands& op, const Systems& sys, const T* Bt, T* x0, T* x1,
               int sweeps, int x_zero, cudaStream_t s, T** result,
               const uint64_t* active = nullptr, const double* pivinv = nullptr) {
  SweepArgs a;
  std::memset(&a, 0, sizeof(a));
  a.row.n = m->n_nodes;
  a.row.K = sys.K;
  a.row.divK = make_fastdiv((uint32_t)sys.K);
  a.row.stage = sys.K >= kStageMinSystems ? 1 : 0;
  a.row.row_ptr = m->row_ptr;
  a.row.col_idx = op.cols;
  a.row.offd = op.offd;
  a.row.hess = op.hess;
  a.row.vol = m->vol;
  a.row.Bt = Bt;
  a.row.info = op.info;
  a.row.pivinv = pivinv;
  a.masked = active ? 1 : 0;
  a.active[0] = active ? active[0] : ~0ull;
  a.active[1] = active ? active[1] : ~0ull;
  for (int k = 0; k < kMaxSys; ++k) {
    a.omega[k] = sys.omega[k];
    a.phase[k] = sys.phase[k];
  }
  size_t smem = 0;
  int rc = FNLH_OK;
  if constexpr (sizeof(T) == 4) {
    if (a.row.stage && (rc = stage_setup(k_sweep_f32<BS, TJ>, kSweepThreadsF32, sys.K, BS, &a.smem_floats, &smem)))
      return rc;
  }
  T* cur = x0;
  T* nxt = x1;
  if ((rc = mark(g_ev_begin, s))) return rc;
  for (int it = 0; it < sweeps; ++it) {
    a.Xin = cur;
    a.Xout = nxt;
    a.x_zero = (it == 0) ? x_zero : 0;
    if ((rc = sweep_launch<BS, TJ, T>(a, smem, s))) return rc;
    T* t = cur;
    cur = nxt;
    nxt = t;
  }
  *result = cur;
  return mark(g_ev_end, s);
}

template <int BS, typename TJ, typename T>
int relax_typed(const fnlh_mesh* m, const fnlh_jacobian* J, int n_harm, const double* omega, const double* sigma,
                const double* B, double* X, int sweeps, int precision, void* ws, cudaStream_t s) {
  SweepOperands op;
  int rc = sweep_operands(m, J, precision, &op);
  if (rc) return rc;
  const Systems sys = make_systems(n_harm, omega, sigma);
  const WsLayout W = ws_layout(J->n_nodes, BS, n_harm, precision);
  T* bt = at<T>(ws, W.vec[0]);
  T* x0 = at<T>(ws, W.vec[1]);
  T* x1 = at<T>(ws, W.vec[2]);
  const int n = J->n_nodes;
  if ((rc = rotate_in<BS, T>(n, sys.K, op.rot, B, bt, s))) return rc;
  if ((rc = rotate_in<BS, T>(n, sys.K, op.rot, X, x0, s))) return rc;
  T* res = x0;
  double* pivinv = nullptr;
  if constexpr (sizeof(T) == 8) {
    pivinv = at<double>(ws, W.pivinv);
    if ((rc = pivot_inverses<BS>(m, (const double*)op.hess, sys, pivinv, s))) return rc;
  }
  if ((rc = run_sweeps<BS, TJ, T>(m, op, sys, bt, x0, x1, sweeps, 0, s, &res, nullptr,
                                  pivinv)))
    return rc;
  return rotate_out<BS, T>(n, sys.K, op.rot, res, X, 0, s);
}

int relax_impl(const fnlh_mesh* m, const fnlh_jacobian* J, int n_harm, const double* omega, const double* sigma,
               const double* B, double* X, int sweeps, int precision, void* ws, cudaStream_t s) {
#define FNLH_RELAX(BS, TJ, T) relax_typed<BS, TJ, T>(m, J, n_harm, omega, sigma, B, X, sweeps, precision, ws, s)
  if (J->block == 5) {
    if (precision == FNLH_F64) return FNLH_RELAX(5, double, double);
    if (precision == FNLH_F32) return FNLH_RELAX(5, float, float);
    return FNLH_RELAX(5, __nv_bfloat16, float);
  }
  if (precision == FNLH_F64) return FNLH_RELAX(6, double, double);
  if (precision == FNLH_F32) return FNLH_RELAX(6, float, float);
  return FNLH_RELAX(6, __nv_bfloat16, float);
#undef FNLH_RELAX
}

// ------------------------------------------------------------------ solve

int residual_launch(const fnlh_mesh* m, const fnlh_jacobian* J, const Systems& sys, const double* B,
                    const double* X, double* r, float* r32rot, const float* rotf, int x_zero, double* norms, void* ws,
                    cudaStream_t s);
int residual_ff_launch(const fnlh_mesh* m, const fnlh_jacobian* J, const Systems& sys, const float2* bff,
                       const float2* xff, float* r32rot, const float* rotf, double* norms, void* ws, cudaStream_t s);

struct Check {
  double rel[kMaxSys];
  double first_max;
};

// Classifies the residual norms copied to the host.
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
int solve_typed(const fnlh_mesh* m, const fnlh_jacobian* J, int n_harm, const double* omega, const double* sigma,
                const double* B, double* X, int precision, double tol, int inner, int max_checks, int flags, void* ws,
                size_t ws_bytes, int* checks_done, int* sweeps_done, double* rel_res, cudaStream_t s) {
  SweepOperands op;
  int rc = sweep_operands(m, J, precision, &op);
  if (rc) return rc;
  const Systems sys = make_systems(n_harm, omega, sigma);
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
  const bool masking = (flags & FNLH_SOLVE_MASK_CONVERGED) != 0;
  // On a partitioned mesh the sweeps drop the cross-partition couplings, so
  // plain FP64 Jacobi would converge to the truncated system: there the FP64
  // solve is a defect correction too, against the full FP64 residual.
  const bool defect = mixed || m->part != nullptr;
  uint64_t active[2] = {~0ull, ~0ull};
  bool x_zero = (flags & FNLH_SOLVE_ZERO_GUESS) != 0;
  if (x_zero) FNLH_CUDA_TRY(cudaMemsetAsync(X, 0, sizeof(double) * (size_t)n * sys.C * BS, s));
  if (!defect) {
    // plain FP64 Jacobi: iterate in the rotated basis, check every `inner` sweeps
    if ((rc = rotate_in<BS, T>(n, K, op.rot, B, v0, s))) return rc;
    if ((rc = rotate_in<BS, T>(n, K, op.rot, X, v1, s))) return rc;
  }
  T* cur = v1;
  double* pivinv = nullptr;
  if constexpr (sizeof(T) == 8) {
    pivinv = at<double>(ws, W.pivinv);
    if ((rc = pivot_inverses<BS>(m, (const double*)op.hess, sys, pivinv, s))) return rc;
  }
  // Float-float checks (mixed solves whose prep blob has FNLH_PREP_FF and whose
  // workspace holds the shadows): every check after the first evaluates B - A x
  // on the FP32 units from float-float shadows of B and x (x's is rewritten
  // by every update); a passing one is confirmed at once by the FP64 residual,
  // and a check that the residual's decay predicts at or below 2 tol is made
  // in FP64 directly, so that convergence is always certified in FP64.
  const PrepLayout PL = prep_layout(J->n_nodes, J->nnz, BS, J->prep_flags);
  const bool ff = mixed && n > 0 && PL.offdff != (size_t)-1 && ws_bytes >= W.total_ff;
  float2* bff = ff ? at<float2>(ws, W.bff) : nullptr;
  float2* xff = ff ? at<float2>(ws, W.xff) : nullptr;
  if (ff) {
    const long long nv = (long long)n * sys.C * BS;
    k_split_vec<<<blocks_for(nv, 256), 256, 0, s>>>(nv, B, bff);
    FNLH_LAUNCH_CHECK();
    if (x_zero) {
      FNLH_CUDA_TRY(cudaMemsetAsync(xff, 0, sizeof(float2) * (size_t)nv, s));
    } else {
      k_split_vec<<<blocks_for(nv, 256), 256, 0, s>>>(nv, X, xff);
      FNLH_LAUNCH_CHECK();
    }
  }
  double bnorm[kMaxSys];  // ||B_k||^2 from the first (FP64) check
  double prev_worst = -1.0;
  bool fp64_next = false;
  auto fetch = [&]() -> int {
    FNLH_CUDA_TRY(cudaMemcpyAsync(hn, norms, sizeof(double) * 2 * K, cudaMemcpyDeviceToHost, s));
    FNLH_CUDA_TRY(cudaStreamSynchronize(s));
    return FNLH_OK;
  };
  for (;;) {
    const bool use_ff = ff && checks > 0 && !fp64_next;
    if (use_ff) {
      rc = residual_ff_launch(m, J, sys, bff, xff, (float*)v0, op.rotf, norms, ws, s);
      if (rc || (rc = fetch())) return rc;
      for (int k = 0; k < K; ++k) hn[2 * k + 1] = bnorm[k];
      rc = check_norms(hn, K, tol, &ck, false, &conv);
    }
    if (!use_ff || (rc == FNLH_OK && conv)) {
      // mixed: Q^T r in FP32 straight into v0; FP64 defect correction: r into v2
      double* r64 = (defect && !mixed) ? (double*)v2 : nullptr;
      rc = residual_launch(m, J, sys, B, X, r64, mixed ? (float*)v0 : nullptr, op.rotf, x_zero ? 1 : 0, norms, ws,
                           s);
      x_zero = false;
      if (rc || (rc = fetch())) return rc;
      if (checks == 0)
        for (int k = 0; k < K; ++k) bnorm[k] = hn[2 * k + 1];
      rc = check_norms(hn, K, tol, &ck, checks == 0, &conv);
    }
    ++checks;
    if (rc || conv || checks >= max_checks) break;
    if (ff) {  // does the decay predict the next check at or below 2 tol?  Then make it in FP64.
      double worst = 0.0;
      for (int k = 0; k < K; ++k) worst = fmax(worst, ck.rel[k]);
      fp64_next = prev_worst > 0.0 && worst * worst / prev_worst <= 2.0 * tol;
      prev_worst = worst;
    }
    if (masking)  // converged systems are frozen for the following sweeps
      for (int k = 0; k < K; ++k)
        if (ck.rel[k] <= tol) active[k >> 6] &= ~(1ull << (k & 63));
    const uint64_t* act = masking ? active : nullptr;
    T* res = nullptr;
    if (defect) {
      // inner: A~ e = r~ from e = 0 (v1/v2 ping-pong), then x += Q e in FP64
      if constexpr (sizeof(T) == 8) {
        if ((rc = rotate_in<BS, T>(n, K, op.rot, (const double*)v2, v0, s))) return rc;
      }
      if ((rc = run_sweeps<BS, TJ, T>(m, op, sys, v0, v1, v2, inner, 1, s, &res, act, pivinv))) return rc;
      const long long count = (long long)n * K;
      if constexpr (sizeof(T) == 4) {
        if (count > 0) {
          k_update_f32<BS><<<blocks_for(count, 256), 256, 0, s>>>(count, K, op.rotf, (const float*)res, X, xff);
          FNLH_LAUNCH_CHECK();
        }
      } else {
        if ((rc = rotate_out<BS, T>(n, K, op.rot, res, X, 1, s))) return rc;
      }
    } else {
      T* other = (cur == v1) ? v2 : v1;
      if ((rc = run_sweeps<BS, TJ, T>(m, op, sys, v0, cur, other, inner, 0, s, &res, act, pivinv))) return rc;
      cur = res;
      if ((rc = rotate_out<BS, T>(n, K, op.rot, res, X, 0, s))) return rc;
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

int solve_impl(const fnlh_mesh* m, const fnlh_jacobian* J, int n_harm, const double* omega, const double* sigma,
               const double* B, double* X, int precision, double tol, int inner, int max_checks, int flags, void* ws,
               size_t ws_bytes, int* checks_done, int* sweeps_done, double* rel_res, cudaStream_t s) {
#define FNLH_SOLVE(BS, TJ, T)                                                                                   \
  solve_typed<BS, TJ, T>(m, J, n_harm, omega, sigma, B, X, precision, tol, inner, max_checks, flags, ws,       \
                         ws_bytes, checks_done, sweeps_done, rel_res, s)
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
// Several blade rows (different meshes and harmonic counts) in one launch per
// sweep (two when rows that stage their blocks are mixed with rows that do
// not).  The (node, system) pairs of every row are cut into tiles of
// blockDim.x consecutive pairs; the grid walks the global tile list -- one
// CTA per tile, or a persistent grid of SMs x ctas_per_sm CTAs striding over
// it -- so the rows share one launch and one tail instead of each paying its
// own.  The row descriptors travel as
// a __grid_constant__ kernel parameter (no device memory, capturable in a
// CUDA graph).

constexpr int kMaxBatchRows = 8;

struct BatchRow {
  TileRow row;
  void* x[2];        // ping-pong iterate buffers
  long long tile0;   // first global tile of this row
  int32_t masked;    // 0: every system is swept; 1: only the systems set in `active`
  int32_t pad;
  uint64_t active[2];
  double omega[kMaxSys];
  double2 phase[kMaxSys];
};

struct BatchArgs {
  int32_t n_rows, parity, smem_floats, x_zero;  // x_zero: the iterate is zero (first sweep of a correction)
  long long tile_base, tile_end;  // the tiles [tile_base, tile_end) of this launch
  int32_t order[kMaxBatchRows];   // row indices in tile order (rows that stage their blocks first)
  BatchRow row[kMaxBatchRows];
};

// One tile t of the global tile list.
template <int BS, typename TJ, typename T>
__device__ __forceinline__ void batched_tile(const BatchArgs& a, long long t, float* smem) {
  int q = 0;
  while (q + 1 < a.n_rows && t >= a.row[a.order[q + 1]].tile0) ++q;
  const BatchRow& D = a.row[a.order[q]];
  const SweepIO io{D.x[a.parity], D.x[a.parity ^ 1], D.omega, D.masked ? D.active : nullptr, D.phase};
  const long long g0 = (t - D.tile0) * blockDim.x;
  if constexpr (sizeof(T) == 8) {
    const long long g = g0 + threadIdx.x;
    if (g < (long long)D.row.n * D.row.K) {
      const int i = (int)fdiv((uint32_t)g, D.row.divK);
      const int k = (int)g - i * D.row.K;
      if (sys_active(io, k)) sweep_pair_f64<BS>(D.row, io, g, a.x_zero != 0);
      else freeze_pair<BS, double>(D.row, io, i, k, a.x_zero != 0);
    }
  } else {
    sweep_tile_f32<BS, TJ>(D.row, io, g0, a.x_zero != 0, smem, a.smem_floats);
  }
}

// One CTA per tile.  FP32: 64 registers (up to 256 threads, four CTAs per SM;
// 64 threads, sixteen); FP64 thread-per-pair needs 128.
template <int BS, typename TJ, typename T>
__global__ void __launch_bounds__(kSweepThreads, (sizeof(T) == 8) ? 2 : 4)
    k_sweep_batched(const __grid_constant__ BatchArgs a) {
  extern __shared__ __align__(16) float smem[];
  batched_tile<BS, TJ, T>(a, a.tile_base + blockIdx.x, smem);
}

// Persistent form: a grid of SMs x ctas_per_sm CTAs striding over the tile
// list.  The loop around the tile body costs registers, so it keeps two CTAs
// of 256 threads per SM; the autotuner weighs it against one CTA per tile.
template <int BS, typename TJ, typename T>
__global__ void __launch_bounds__(kSweepThreads, 2) k_sweep_batched_persistent(const __grid_constant__ BatchArgs a) {
  extern __shared__ __align__(16) float smem[];
  for (long long t = a.tile_base + blockIdx.x; t < a.tile_end; t += gridDim.x) batched_tile<BS, TJ, T>(a, t, smem);
}

size_t batched_extra_bytes(int n_rows) { return n_rows > 0 ? 256 : 0; }

// Launch shape, operands and workspace slices of a batch.
struct BatchPlan {
  int threads;
  bool persistent;
  size_t smem;            // dynamic shared memory of the staged group's launches
  long long split, n_tiles;  // tiles [0, split) belong to rows that stage their blocks, [split, n_tiles) do not
  unsigned grid[2];       // grid of the staged group's and of the other group's launch
  SweepOperands ops[kMaxBatchRows];
  Systems sys[kMaxBatchRows];
  char* base[kMaxBatchRows];  // the row's workspace slice (ws_layout of its size and precision)
  const fnlh_mesh* mesh[kMaxBatchRows];
  // FP32 rows of K <= kRealMeanMaxSystems (vectors with a real mean flow):
  // swept by their own single-row launches (k_sweep_f32_node), not in the
  // shared tiles
  bool own[kMaxBatchRows];
  int n_rows;
};

// ff_layout: each row's workspace slice also holds the float-float shadows
// of B and x (ws_layout total_ff instead of total).
template <int BS, typename TJ, typename T>
int batch_setup(const fnlh_row* rows, int n_rows, int precision, const fnlh_tuning* tn, void* ws, BatchArgs& a,
                BatchPlan& P, bool ff_layout = false) {
  std::memset(&a, 0, sizeof(a));
  P.threads = (tn && tn->threads > 0) ? tn->threads : (sizeof(T) == 4 ? kSweepThreadsF32 : kSweepThreads);
  const int ctas_per_sm = tn ? tn->ctas_per_sm : 0;  // 0: one CTA per tile
  if (P.threads > kSweepThreads || P.threads % 32) return FNLH_ERR_ARG;
  int dev = 0, sms = 0;
  FNLH_CUDA_TRY(cudaGetDevice(&dev));
  FNLH_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  size_t off = 256;
  long long tiles = 0;
  int kmin = kMaxSys;
  P.n_rows = n_rows;
  for (int r = 0; r < n_rows; ++r) {
    const fnlh_row& R = rows[r];
    int rc = sweep_operands(R.mesh, R.J, precision, &P.ops[r]);
    if (rc) return rc;
    P.sys[r] = make_systems(R.n_harm, R.omega, R.sigma);
    const Systems& sys = P.sys[r];
    P.mesh[r] = R.mesh;
    P.own[r] = real_mean<T>(sys.K);
    const WsLayout W = ws_layout(R.mesh->n_nodes, BS, R.n_harm, precision);
    char* base = (char*)ws + off;
    P.base[r] = base;
    off += ff_layout ? W.total_ff : W.total;
    BatchRow& D = a.row[r];
    D.row.n = R.mesh->n_nodes;
    D.row.K = sys.K;
    D.row.divK = make_fastdiv((uint32_t)sys.K);
    D.row.stage = sys.K >= kStageMinSystems ? 1 : 0;
    D.row.row_ptr = R.mesh->row_ptr;
    D.row.col_idx = P.ops[r].cols;
    D.row.offd = P.ops[r].offd;
    D.row.hess = P.ops[r].hess;
    D.row.vol = R.mesh->vol;
    D.row.Bt = base + W.vec[0];
    D.row.info = P.ops[r].info;
    D.row.pivinv = nullptr;  // the batched FP64 tile divides in place
    D.x[0] = base + W.vec[1];
    D.x[1] = base + W.vec[2];
    D.active[0] = D.active[1] = ~0ull;
    if (sizeof(T) == 4 && D.row.stage) kmin = std::min(kmin, sys.K);
    for (int k = 0; k < kMaxSys; ++k) {
      D.omega[k] = sys.omega[k];
      D.phase[k] = sys.phase[k];
    }
  }
  // Tiles in two groups: the rows that stage their blocks in shared memory
  // (FP32 with K >= kStageMinSystems), then the rest.  Each group gets its
  // own launch per sweep, so that the rows that read their blocks through L1
  // do not run on SMs configured for the staged rows' shared memory (mixing
  // them in one launch cost 3% on three rows with K = 3, 9, 5).  Rows swept
  // by their own launches (P.own) take no tiles.
  int q = 0;
  P.split = 0;
  for (int pass = 0; pass < 2; ++pass)
    for (int r = 0; r < n_rows; ++r) {
      BatchRow& D = a.row[r];
      const bool staged = sizeof(T) == 4 && D.row.stage;
      if (P.own[r] || staged != (pass == 0)) continue;
      a.order[q++] = r;
      D.tile0 = tiles;
      tiles += ((long long)D.row.n * D.row.K + P.threads - 1) / P.threads;
      if (pass == 0) P.split = tiles;
    }
  P.n_tiles = tiles;
  a.n_rows = q;  // rows in the tile list
  P.smem = 0;
  P.persistent = ctas_per_sm > 0;
  if constexpr (sizeof(T) == 4) {
    // sized for the staged row with the fewest systems (the largest stage),
    // so that every staged row's tiles fit
    if (kmin < kMaxSys) {
      int rc = P.persistent ? stage_setup(k_sweep_batched_persistent<BS, TJ, T>, P.threads, kmin, BS,
                                          &a.smem_floats, &P.smem)
                            : stage_setup(k_sweep_batched<BS, TJ, T>, P.threads, kmin, BS, &a.smem_floats, &P.smem);
      if (rc) return rc;
    }
  }
  const long long group[2] = {P.split, P.n_tiles - P.split};
  for (int g = 0; g < 2; ++g) {
    const long long grid_ll = P.persistent ? std::min<long long>(group[g], (long long)sms * ctas_per_sm) : group[g];
    P.grid[g] = (unsigned)std::max<long long>(grid_ll, 1);
  }
  return FNLH_OK;
}

// `sweeps` launches starting at a.parity (the first from zero when x_zero);
// a.parity holds the buffer of the result on return.  The rows that sweep on
// their own (P.own) run all their sweeps first, between the same buffers.
template <int BS, typename TJ, typename T>
int batch_launch(BatchArgs& a, const BatchPlan& P, int sweeps, int x_zero, cudaStream_t s) {
  int rc = mark(g_ev_begin, s);
  if (rc) return rc;
  {
    cudaEvent_t b = g_ev_begin, e = g_ev_end;  // the hook brackets the whole batch
    g_ev_begin = g_ev_end = nullptr;
    for (int r = 0; r < P.n_rows && !rc; ++r) {
      if (!P.own[r]) continue;
      const BatchRow& D = a.row[r];
      T* res = nullptr;
      rc = run_sweeps<BS, TJ, T>(P.mesh[r], P.ops[r], P.sys[r], (const T*)D.row.Bt, (T*)D.x[a.parity],
                                 (T*)D.x[a.parity ^ 1], sweeps, x_zero, s, &res, D.masked ? D.active : nullptr);
    }
    g_ev_begin = b;
    g_ev_end = e;
    if (rc) return rc;
  }
  for (int it = 0; it < sweeps; ++it) {
    a.x_zero = (it == 0) ? x_zero : 0;
    for (int g = 0; g < 2; ++g) {  // the staged rows' tiles, then the others'
      a.tile_base = g ? P.split : 0;
      a.tile_end = g ? P.n_tiles : P.split;
      if (a.tile_end <= a.tile_base) continue;
      const size_t smem = g ? 0 : P.smem;
      if (P.persistent) k_sweep_batched_persistent<BS, TJ, T><<<P.grid[g], P.threads, smem, s>>>(a);
      else k_sweep_batched<BS, TJ, T><<<P.grid[g], P.threads, smem, s>>>(a);
      FNLH_LAUNCH_CHECK();
    }
    a.parity ^= 1;
  }
  a.x_zero = 0;
  return mark(g_ev_end, s);
}

static thread_local BatchArgs g_batch;  // large: kept off the stack (each launch copies it)

static bool per_row_mode(const fnlh_tuning* tn) { return tn && tn->ctas_per_sm == FNLH_TUNING_PER_ROW; }

// Per-row mode: the single-row sweep of every row in turn (each row's rows
// of the workspace as batch_setup lays them out), `sweeps` from its x.
template <int BS, typename TJ, typename T>
int batched_per_row(const fnlh_row* rows, int n_rows, int sweeps, const BatchArgs& a, const BatchPlan& P,
                    cudaStream_t s) {
  int rc = mark(g_ev_begin, s);
  if (rc) return rc;
  for (int r = 0; r < n_rows; ++r) {
    const BatchRow& D = a.row[r];
    double* pivinv = nullptr;
    if constexpr (sizeof(T) == 8) {
      pivinv = at<double>(P.base[r], ws_layout(D.row.n, BS, D.row.K - 1, FNLH_F64).pivinv);
      if ((rc = pivot_inverses<BS>(rows[r].mesh, (const double*)P.ops[r].hess, P.sys[r], pivinv, s))) return rc;
    }
    T* res = nullptr;
    // the timing hook brackets the whole batch, not each row's sweeps
    cudaEvent_t b = g_ev_begin, e = g_ev_end;
    g_ev_begin = g_ev_end = nullptr;
    rc = run_sweeps<BS, TJ, T>(rows[r].mesh, P.ops[r], P.sys[r], (const T*)D.row.Bt, (T*)D.x[0], (T*)D.x[1], sweeps,
                               0, s, &res, D.masked ? D.active : nullptr, pivinv);
    g_ev_begin = b;
    g_ev_end = e;
    if (rc) return rc;
    if ((rc = rotate_out<BS, T>(D.row.n, D.row.K, P.ops[r].rot, res, rows[r].X, 0, s))) return rc;
  }
  return mark(g_ev_end, s);
}

// Per-row mode of the batched solve: `sweeps` single-row sweeps of every row
// between its ping-pong buffers, from a.parity (from zero when x_zero); the
// result is in D.x[a.parity] on return, as after batch_launch.
template <int BS, typename TJ, typename T>
int sweep_rows_per_row(const fnlh_row* rows, int n_rows, int sweeps, int x_zero, BatchArgs& a, const BatchPlan& P,
                       double* const* pivinv, cudaStream_t s) {
  int rc = mark(g_ev_begin, s);
  if (rc) return rc;
  cudaEvent_t b = g_ev_begin, e = g_ev_end;
  g_ev_begin = g_ev_end = nullptr;
  for (int r = 0; r < n_rows && !rc; ++r) {
    const BatchRow& D = a.row[r];
    T* res = nullptr;
    rc = run_sweeps<BS, TJ, T>(rows[r].mesh, P.ops[r], P.sys[r], (const T*)D.row.Bt, (T*)D.x[a.parity],
                               (T*)D.x[a.parity ^ 1], sweeps, x_zero, s, &res, D.masked ? D.active : nullptr,
                               pivinv[r]);
  }
  g_ev_begin = b;
  g_ev_end = e;
  if (rc) return rc;
  a.parity ^= (sweeps & 1);
  return mark(g_ev_end, s);
}

template <int BS, typename TJ, typename T>
int batched_typed(const fnlh_row* rows, int n_rows, int sweeps, int precision, const fnlh_tuning* tn, void* ws,
                  cudaStream_t s) {
  BatchArgs& a = g_batch;
  BatchPlan P;
  int rc = batch_setup<BS, TJ, T>(rows, n_rows, precision, tn, ws, a, P);
  if (rc) return rc;
  if (per_row_mode(tn)) {
    for (int r = 0; r < n_rows; ++r) {
      const BatchRow& D = a.row[r];
      if ((rc = rotate_in<BS, T>(D.row.n, D.row.K, P.ops[r].rot, rows[r].B, (T*)D.row.Bt, s))) return rc;
      if ((rc = rotate_in<BS, T>(D.row.n, D.row.K, P.ops[r].rot, rows[r].X, (T*)D.x[0], s))) return rc;
    }
    return batched_per_row<BS, TJ, T>(rows, n_rows, sweeps, a, P, s);
  }
  for (int r = 0; r < n_rows; ++r) {
    const BatchRow& D = a.row[r];
    if ((rc = rotate_in<BS, T>(D.row.n, D.row.K, P.ops[r].rot, rows[r].B, (T*)D.row.Bt, s))) return rc;
    if ((rc = rotate_in<BS, T>(D.row.n, D.row.K, P.ops[r].rot, rows[r].X, (T*)D.x[0], s))) return rc;
  }
  a.parity = 0;
  if ((rc = batch_launch<BS, TJ, T>(a, P, sweeps, 0, s))) return rc;
  for (int r = 0; r < n_rows; ++r) {
    const BatchRow& D = a.row[r];
    if ((rc = rotate_out<BS, T>(D.row.n, D.row.K, P.ops[r].rot, (const T*)D.x[a.parity], rows[r].X, 0, s))) return rc;
  }
  return FNLH_OK;
}

// Batched solve: every row's systems to ||r|| <= tol ||B|| together.  FP64:
// plain Jacobi in the rotated basis with the FP64 residual every `inner`
// sweeps; FP32 / BF16: defect correction (FP64 residual of every row, one
// batched launch per inner sweep from e = 0 over all rows, x += Q e).
template <int BS, typename TJ, typename T>
int solve_batched_typed(const fnlh_row* rows, int n_rows, int precision, double tol, int inner, int max_checks,
                        int flags, const fnlh_tuning* tn, void* ws, size_t ws_bytes, int* checks_done,
                        int* sweeps_done, double* rel_res, cudaStream_t s) {
  BatchArgs& a = g_batch;
  BatchPlan P;
  const bool mixed = sizeof(T) == 4;
  // Float-float checks, as in fnlh_solve: every row's prep blob has the split
  // blocks (FNLH_PREP_FF) and the workspace holds every row's shadows of B and x.
  bool ff = mixed;
  {
    size_t need = batched_extra_bytes(n_rows);
    for (int r = 0; r < n_rows && ff; ++r) {
      const fnlh_jacobian* J = rows[r].J;
      const PrepLayout PL = prep_layout(J->n_nodes, J->nnz, BS, J->prep_flags);
      if (PL.offdff == (size_t)-1 || J->n_nodes == 0) ff = false;
      need += ws_layout(J->n_nodes, BS, rows[r].n_harm, precision).total_ff;
    }
    ff = ff && ws_bytes >= need;
  }
  int rc = batch_setup<BS, TJ, T>(rows, n_rows, precision, tn, ws, a, P, ff);
  if (rc) return rc;
  const bool masking = (flags & FNLH_SOLVE_MASK_CONVERGED) != 0;
  bool x_zero = (flags & FNLH_SOLVE_ZERO_GUESS) != 0;
  const bool per_row = per_row_mode(tn);
  double* pivinv[kMaxBatchRows] = {};
  if constexpr (sizeof(T) == 8) {
    if (per_row)  // the single-row FP64 sweep reads its pivot table (fnlh_workspace_bytes at FNLH_F64 holds it)
      for (int r = 0; r < n_rows; ++r) {
        const BatchRow& D = a.row[r];
        pivinv[r] = at<double>(P.base[r], ws_layout(D.row.n, BS, D.row.K - 1, FNLH_F64).pivinv);
        if ((rc = pivot_inverses<BS>(rows[r].mesh, (const double*)P.ops[r].hess, P.sys[r], pivinv[r], s))) return rc;
      }
  }
  for (int r = 0; r < n_rows; ++r) {
    const BatchRow& D = a.row[r];
    if (x_zero) FNLH_CUDA_TRY(cudaMemsetAsync(rows[r].X, 0, sizeof(double) * (size_t)D.row.n * P.sys[r].C * BS, s));
    if (!mixed) {
      if ((rc = rotate_in<BS, T>(D.row.n, D.row.K, P.ops[r].rot, rows[r].B, (T*)D.row.Bt, s))) return rc;
      if ((rc = rotate_in<BS, T>(D.row.n, D.row.K, P.ops[r].rot, rows[r].X, (T*)D.x[0], s))) return rc;
    }
  }
  float2* bff[kMaxBatchRows] = {};
  float2* xff[kMaxBatchRows] = {};
  if (ff)
    for (int r = 0; r < n_rows; ++r) {
      const WsLayout W = ws_layout(a.row[r].row.n, BS, a.row[r].row.K - 1, precision);
      bff[r] = at<float2>(P.base[r], W.bff);
      xff[r] = at<float2>(P.base[r], W.xff);
      const long long nv = (long long)a.row[r].row.n * P.sys[r].C * BS;
      k_split_vec<<<blocks_for(nv, 256), 256, 0, s>>>(nv, rows[r].B, bff[r]);
      FNLH_LAUNCH_CHECK();
      if (x_zero) {
        FNLH_CUDA_TRY(cudaMemsetAsync(xff[r], 0, sizeof(float2) * (size_t)nv, s));
      } else {
        k_split_vec<<<blocks_for(nv, 256), 256, 0, s>>>(nv, rows[r].X, xff[r]);
        FNLH_LAUNCH_CHECK();
      }
    }
  a.parity = 0;
  std::vector<double> hn(2 * kMaxSys * n_rows);
  std::vector<double> rel(kMaxSys * n_rows, 0.0);
  std::vector<double> bnorm(kMaxSys * n_rows, 0.0);  // ||B_k||^2 per row and system, from the first (FP64) check
  double first_max = 0.0, prev_worst = -1.0;
  bool fp64_next = false;
  int checks = 0, sweeps = 0;
  bool conv = false;
  // the relative residuals of hn into rel; returns the worst, or -1 on a non-finite value
  auto evaluate = [&]() -> double {
    double worst = 0.0;
    for (int r = 0; r < n_rows; ++r)
      for (int k = 0; k < a.row[r].row.K; ++k) {
        const double rr = hn[2 * kMaxSys * r + 2 * k], bb = hn[2 * kMaxSys * r + 2 * k + 1];
        if (!(rr == rr) || !(bb == bb) || rr > 1e300 || bb > 1e300) return -1.0;
        const double v = (bb > 0.0) ? std::sqrt(rr / bb) : std::sqrt(rr);
        rel[kMaxSys * r + k] = v;
        worst = std::max(worst, v);
      }
    return worst;
  };
  for (;;) {
    // float-float check of every row; a passing one is confirmed at once in FP64
    bool need64 = true;
    if (ff && checks > 0 && !fp64_next) {
      for (int r = 0; r < n_rows; ++r) {
        const BatchRow& D = a.row[r];
        const WsLayout W = ws_layout(D.row.n, BS, D.row.K - 1, precision);
        double* norms = at<double>(P.base[r], W.norms);
        rc = residual_ff_launch(rows[r].mesh, rows[r].J, P.sys[r], bff[r], xff[r], (float*)D.row.Bt,
                                P.ops[r].rotf, norms, P.base[r], s);
        if (rc) return rc;
        FNLH_CUDA_TRY(cudaMemcpyAsync(hn.data() + 2 * kMaxSys * r, norms, sizeof(double) * 2 * D.row.K,
                                      cudaMemcpyDeviceToHost, s));
      }
      FNLH_CUDA_TRY(cudaStreamSynchronize(s));
      for (int r = 0; r < n_rows; ++r)
        for (int k = 0; k < a.row[r].row.K; ++k) hn[2 * kMaxSys * r + 2 * k + 1] = bnorm[kMaxSys * r + k];
      const double w = evaluate();
      need64 = !(w >= 0.0) || w <= tol;
    }
    if (need64) {
      for (int r = 0; r < n_rows; ++r) {
        const BatchRow& D = a.row[r];
        const WsLayout W = ws_layout(D.row.n, BS, D.row.K - 1, precision);
        double* norms = at<double>(P.base[r], W.norms);
        rc = residual_launch(rows[r].mesh, rows[r].J, P.sys[r], rows[r].B, rows[r].X, nullptr,
                             mixed ? (float*)D.row.Bt : nullptr, P.ops[r].rotf, x_zero ? 1 : 0, norms, P.base[r],
                             s);
        if (rc) return rc;
        FNLH_CUDA_TRY(cudaMemcpyAsync(hn.data() + 2 * kMaxSys * r, norms, sizeof(double) * 2 * D.row.K,
                                      cudaMemcpyDeviceToHost, s));
      }
      x_zero = false;
      FNLH_CUDA_TRY(cudaStreamSynchronize(s));
      if (checks == 0)
        for (int r = 0; r < n_rows; ++r)
          for (int k = 0; k < a.row[r].row.K; ++k) bnorm[kMaxSys * r + k] = hn[2 * kMaxSys * r + 2 * k + 1];
    }
    const double worst = evaluate();
    if (!(worst >= 0.0)) {
      rc = FNLH_ERR_NONFINITE;
      break;
    }
    if (checks == 0) first_max = worst;
    else if (worst > 1e3 * std::max(first_max, 1e-300)) {
      rc = FNLH_ERR_DIVERGED;
      break;
    }
    ++checks;
    conv = worst <= tol;
    if (conv || checks >= max_checks) break;
    if (ff) {  // does the decay predict the next check at or below 2 tol?  Then make it in FP64.
      fp64_next = prev_worst > 0.0 && worst * worst / prev_worst <= 2.0 * tol;
      prev_worst = worst;
    }
    if (masking)  // converged systems are frozen for the following sweeps
      for (int r = 0; r < n_rows; ++r) {
        BatchRow& D = a.row[r];
        D.masked = 1;
        for (int k = 0; k < D.row.K; ++k)
          if (rel[kMaxSys * r + k] <= tol) D.active[k >> 6] &= ~(1ull << (k & 63));
      }
    if (mixed) {
      a.parity = 0;
      if (per_row) rc = sweep_rows_per_row<BS, TJ, T>(rows, n_rows, inner, 1, a, P, pivinv, s);
      else rc = batch_launch<BS, TJ, T>(a, P, inner, 1, s);
      if (rc) return rc;
      for (int r = 0; r < n_rows; ++r) {
        const BatchRow& D = a.row[r];
        if ((rc = update_f32(D.row.n, D.row.K, BS, P.ops[r].rotf, (const float*)D.x[a.parity], rows[r].X, s,
                             xff[r])))
          return rc;
      }
    } else {
      if (per_row) rc = sweep_rows_per_row<BS, TJ, T>(rows, n_rows, inner, 0, a, P, pivinv, s);
      else rc = batch_launch<BS, TJ, T>(a, P, inner, 0, s);
      if (rc) return rc;
      for (int r = 0; r < n_rows; ++r) {
        const BatchRow& D = a.row[r];
        if ((rc = rotate_out<BS, T>(D.row.n, D.row.K, P.ops[r].rot, (const T*)D.x[a.parity], rows[r].X, 0, s)))
          return rc;
      }
    }
    sweeps += inner;
  }
  if (checks_done) *checks_done = checks;
  if (sweeps_done) *sweeps_done = sweeps;
  if (rel_res) {
    int o = 0;
    for (int r = 0; r < n_rows; ++r)
      for (int k = 0; k < a.row[r].row.K; ++k) rel_res[o++] = rel[kMaxSys * r + k];
  }
  if (rc) return rc;
  return conv ? FNLH_OK : FNLH_ERR_NOT_CONVERGED;
}

int solve_batched_impl(const fnlh_row* rows, int n_rows, int precision, double tol, int inner, int max_checks,
                       int flags, const fnlh_tuning* tn, void* ws, size_t ws_bytes, int* checks_done,
                       int* sweeps_done, double* rel_res, cudaStream_t s) {
  if (n_rows > kMaxBatchRows) return FNLH_ERR_UNSUPPORTED;
  const int b = rows[0].J->block;
  for (int r = 1; r < n_rows; ++r)
    if (rows[r].J->block != b) return FNLH_ERR_UNSUPPORTED;
#define FNLH_SB(BS, TJ, T) \
  solve_batched_typed<BS, TJ, T>(rows, n_rows, precision, tol, inner, max_checks, flags, tn, ws, ws_bytes, \
                                 checks_done, sweeps_done, rel_res, s)
  if (b == 5) {
    if (precision == FNLH_F64) return FNLH_SB(5, double, double);
    if (precision == FNLH_F32) return FNLH_SB(5, float, float);
    return FNLH_SB(5, __nv_bfloat16, float);
  }
  if (precision == FNLH_F64) return FNLH_SB(6, double, double);
  if (precision == FNLH_F32) return FNLH_SB(6, float, float);
  return FNLH_SB(6, __nv_bfloat16, float);
#undef FNLH_SB
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
