// Body of the block-Jacobi sweep, shared by the single-row and the batched
// multi-row kernels.
//
// One thread per (node, system).  The iterate and right-hand side use the
// library's internal layout [n][K][b] of complex (re, im) pairs in the
// per-node Hessenberg basis (the mean flow, system 0, carries a zero
// imaginary part), so each thread's slice is one contiguous vector.  (FP32
// vectors of K <= kRealMeanMaxSystems systems keep the mean flow real
// instead, common.cuh; they are swept only by k_sweep_f32_node.)
//
// A CTA owns a tile of consecutive (node, system) pairs.  In the staged form
// (low-precision blocks, FP32 arithmetic) the CTA first copies the
// off-diagonal blocks and Hessenberg factors of its nodes into shared memory
// with coalesced vector loads, converting them to FP32 once, instead of each
// of a node's K threads loading every block entry itself.
#pragma once

#include "common.cuh"

namespace fnlh {

// ---------------------------------------------------------- vector access

template <int BS, typename T>
struct Cvec {
  T re[BS], im[BS];
};

// Load / store the (re, im) interleaved slice of BS complex values.
template <int BS>
__device__ __forceinline__ void load_slice(const float* __restrict__ p, Cvec<BS, float>& v) {
  if constexpr ((2 * BS) % 4 == 0) {
#pragma unroll
    for (int q = 0; q < BS / 2; ++q) {
      const float4 f = __ldg(reinterpret_cast<const float4*>(p) + q);
      v.re[2 * q] = f.x;
      v.im[2 * q] = f.y;
      v.re[2 * q + 1] = f.z;
      v.im[2 * q + 1] = f.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < BS; ++q) {
      const float2 f = __ldg(reinterpret_cast<const float2*>(p) + q);
      v.re[q] = f.x;
      v.im[q] = f.y;
    }
  }
}

template <int BS>
__device__ __forceinline__ void load_slice(const double* __restrict__ p, Cvec<BS, double>& v) {
#pragma unroll
  for (int q = 0; q < BS; ++q) {
    const double2 f = __ldg(reinterpret_cast<const double2*>(p) + q);
    v.re[q] = f.x;
    v.im[q] = f.y;
  }
}

template <int BS>
__device__ __forceinline__ void store_slice(float* __restrict__ p, const Cvec<BS, float>& v) {
  if constexpr ((2 * BS) % 4 == 0) {
#pragma unroll
    for (int q = 0; q < BS / 2; ++q)
      reinterpret_cast<float4*>(p)[q] = make_float4(v.re[2 * q], v.im[2 * q], v.re[2 * q + 1], v.im[2 * q + 1]);
  } else {
#pragma unroll
    for (int q = 0; q < BS; ++q) reinterpret_cast<float2*>(p)[q] = make_float2(v.re[q], v.im[q]);
  }
}

template <int BS>
__device__ __forceinline__ void store_slice(double* __restrict__ p, const Cvec<BS, double>& v) {
#pragma unroll
  for (int q = 0; q < BS; ++q) reinterpret_cast<double2*>(p)[q] = make_double2(v.re[q], v.im[q]);
}

// Load one BS x BS block into registers (row-major).
template <int BS>
__device__ __forceinline__ void load_block(const double* __restrict__ p, double (&J)[BS * BS]) {
  if constexpr ((BS * BS) % 2 == 0) {
#pragma unroll
    for (int q = 0; q < BS * BS / 2; ++q) {
      const double2 f = __ldg(reinterpret_cast<const double2*>(p) + q);
      J[2 * q] = f.x;
      J[2 * q + 1] = f.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < BS * BS; ++q) J[q] = __ldg(p + q);
  }
}

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// ------------------------------------------------------------ staging

// Staging copies global -> shared, all threads of the CTA.  Each thread
// first issues a batch of kStageBatch independent loads into registers and
// only then converts and stores them, so that a batch costs one memory
// latency instead of one per element.
constexpr int kStageBatch = 8;

// `count` FP32 values (16-byte chunks when vec4: both pointers 16-byte
// aligned and count a multiple of 4).
__device__ __forceinline__ void stage_f32(float* __restrict__ dst, const float* __restrict__ src, int count,
                                          bool vec4) {
  if (vec4) {
    const int n4 = count >> 2;
    for (int base = 0; base < n4; base += kStageBatch * blockDim.x) {
      float4 w[kStageBatch];
#pragma unroll
      for (int u = 0; u < kStageBatch; ++u) {
        const int q = base + u * blockDim.x + threadIdx.x;
        if (q < n4) w[u] = __ldg(reinterpret_cast<const float4*>(src) + q);
      }
#pragma unroll
      for (int u = 0; u < kStageBatch; ++u) {
        const int q = base + u * blockDim.x + threadIdx.x;
        if (q < n4) reinterpret_cast<float4*>(dst)[q] = w[u];
      }
    }
  } else {
    for (int base = 0; base < count; base += kStageBatch * blockDim.x) {
      float w[kStageBatch];
#pragma unroll
      for (int u = 0; u < kStageBatch; ++u) {
        const int q = base + u * blockDim.x + threadIdx.x;
        if (q < count) w[u] = __ldg(src + q);
      }
#pragma unroll
      for (int u = 0; u < kStageBatch; ++u) {
        const int q = base + u * blockDim.x + threadIdx.x;
        if (q < count) dst[q] = w[u];
      }
    }
  }
}

// `count` BF16 values to shared memory as FP32 (8-byte chunks when the
// source is 8-byte aligned and count a multiple of 4).
__device__ __forceinline__ void stage_bf16(float* __restrict__ dst, const __nv_bfloat16* __restrict__ src, int count,
                                           bool vec4) {
  if (vec4) {
    const int n4 = count >> 2;
    for (int base = 0; base < n4; base += kStageBatch * blockDim.x) {
      uint2 w[kStageBatch];
#pragma unroll
      for (int u = 0; u < kStageBatch; ++u) {
        const int q = base + u * blockDim.x + threadIdx.x;
        if (q < n4) w[u] = __ldg(reinterpret_cast<const uint2*>(src) + q);
      }
#pragma unroll
      for (int u = 0; u < kStageBatch; ++u) {
        const int q = base + u * blockDim.x + threadIdx.x;
        if (q < n4)
          reinterpret_cast<float4*>(dst)[q] =
              make_float4(bf16_lo(w[u].x), bf16_hi(w[u].x), bf16_lo(w[u].y), bf16_hi(w[u].y));
      }
    }
  } else {
    const uint16_t* s = reinterpret_cast<const uint16_t*>(src);
    for (int base = 0; base < count; base += kStageBatch * blockDim.x) {
      uint32_t w[kStageBatch];
#pragma unroll
      for (int u = 0; u < kStageBatch; ++u) {
        const int q = base + u * blockDim.x + threadIdx.x;
        if (q < count) w[u] = __ldg(s + q);
      }
#pragma unroll
      for (int u = 0; u < kStageBatch; ++u) {
        const int q = base + u * blockDim.x + threadIdx.x;
        if (q < count) dst[q] = __uint_as_float(w[u] << 16);
      }
    }
  }
}

// `count` int32 values.
__device__ __forceinline__ void stage_i32(int* __restrict__ dst, const int* __restrict__ src, int count) {
  for (int base = 0; base < count; base += kStageBatch * blockDim.x) {
    int w[kStageBatch];
#pragma unroll
    for (int u = 0; u < kStageBatch; ++u) {
      const int q = base + u * blockDim.x + threadIdx.x;
      if (q < count) w[u] = __ldg(src + q);
    }
#pragma unroll
    for (int u = 0; u < kStageBatch; ++u) {
      const int q = base + u * blockDim.x + threadIdx.x;
      if (q < count) dst[q] = w[u];
    }
  }
}

// Shared-memory floats needed by a staged tile of `threads` pairs: the
// tile's blocks, factors and neighbour indices.
__host__ __device__ inline int stage_cap_nodes(int threads, int K) { return (threads + K - 1) / K + 1; }
// Staging pays when a staged block serves enough threads: a node's blocks are
// read by its K threads, and below this K the stage's shared memory costs
// more occupancy than the reuse wins (measured on GB300: K = 3..5 run 5-27%
// faster unstaged, K = 7 and up 12-15% faster staged).
constexpr int kStageMinSystems = 6;
constexpr int kStageDegree = 7;  // blocks per node the stage buffer is sized for (hex meshes: <= 6)
__host__ __device__ inline int stage_floats(int threads, int K, int BS) {
  const int nodes = stage_cap_nodes(threads, K);
  return (nodes * kStageDegree + nodes) * BS * BS + nodes * kStageDegree;
}

// ------------------------------------------------------------ the tile

struct TileRow {
  int32_t n, K;
  FastDiv divK;      // division by K (pair index -> node), n K < 2^31
  int32_t stage;     // 1: stage the tile's blocks in shared memory when they fit
  const int32_t* row_ptr;
  const int32_t* col_idx;  // possibly tagged (col_of / side_of / cut_of)
  const void* offd;  // rotated off-diagonal blocks (TJ)
  const void* hess;  // [n][b][b] (double for FP64 sweeps, float otherwise)
  const double* vol;
  const void* Bt;    // [n][K][b] complex, right-hand side in the rotated basis
  const int32_t* info;  // prep info word: 0 = the b = 6 frozen-turbulence pattern holds (FP64 skips its zeros)
  // nullable, FP64: [n][K][b] pairs of the triangular solves (k = 0: (1 / d_q, 0);
  // k > 0: (d_q, s_k) / (d_q^2 + s_k^2)).  Set only for the single-row
  // kernel, whose mean flow takes the real path, so the complex solve reads
  // it for k > 0 alone.
  const double* pivinv;
};

// b = 6 with the frozen-turbulence pattern certified by fnlh_prepare: in the
// rotated basis column 0 of every off-diagonal block is zero below row 0.
template <int BS>
__device__ __forceinline__ bool frozen_turbulence(const TileRow& R) {
  if constexpr (BS == 6) return R.info != nullptr && __ldg(R.info) == 0;
  else return false;
}

// s -= J x for one FP64 block (complex slice); with the pattern, rows 1..5
// skip their structurally zero column 0.
template <int BS>
__device__ __forceinline__ void spmv_block_f64(const double (&J)[BS * BS], const Cvec<BS, double>& x,
                                               Cvec<BS, double>& s, bool pattern) {
  if (pattern) {
#pragma unroll
    for (int t = 0; t < BS; ++t) {
      s.re[0] -= J[t] * x.re[t];
      s.im[0] -= J[t] * x.im[t];
    }
#pragma unroll
    for (int r = 1; r < BS; ++r)
#pragma unroll
      for (int t = 1; t < BS; ++t) {
        s.re[r] -= J[r * BS + t] * x.re[t];
        s.im[r] -= J[r * BS + t] * x.im[t];
      }
  } else {
#pragma unroll
    for (int r = 0; r < BS; ++r)
#pragma unroll
      for (int t = 0; t < BS; ++t) {
        s.re[r] -= J[r * BS + t] * x.re[t];
        s.im[r] -= J[r * BS + t] * x.im[t];
      }
  }
}

// The iterate buffers and frequencies of one launch (the row descriptor
// itself is read in place from the kernel parameters).
struct SweepIO {
  const void* Xin;       // [n][K][b] complex (not read when x_zero)
  void* Xout;            // [n][K][b] complex
  const double* omega;   // [K], omega[0] = 0
  const uint64_t* active;  // bit k set: system k is swept; null: every system
  const double2* phase;  // [K] (cos, sin) of the inter-blade phase angles, phase[0] = (1, 0)
};

__device__ __forceinline__ bool sys_active(const SweepIO& io, int k) {
  return io.active == nullptr || ((io.active[k >> 6] >> (k & 63)) & 1ull);
}

// A frozen (converged) system keeps its iterate: copy the slice through the
// ping-pong, or write zeros on a sweep that starts from zero.
template <int BS, typename T>
__device__ __forceinline__ void freeze_pair(const TileRow& R, const SweepIO& io, int i, int k, bool x_zero) {
  const size_t off = ((size_t)i * R.K + k) * 2 * BS;
  T* out = (T*)io.Xout + off;
  const T* in = (const T*)io.Xin + off;
#pragma unroll
  for (int t = 0; t < 2 * BS; ++t) out[t] = x_zero ? T(0) : in[t];
}

// Shifted Hessenberg solve + store for one pair, shared by both forms.
template <int BS, typename T, typename TH>
__device__ __forceinline__ void finish_pair(const TileRow& R, const SweepIO& io, const TH* H, int i, int k,
                                            Cvec<BS, T>& s) {
  const T shift = (T)(io.omega[k] * __ldg(R.vol + i));
  if constexpr (sizeof(T) == 8)
    hess_solve<BS, T>(H, shift, s.re, s.im, R.pivinv ? R.pivinv + ((size_t)i * R.K + k) * BS * 2 : nullptr);
  else
    hess_solve<BS, T>(H, shift, s.re, s.im);
  store_slice<BS>((T*)io.Xout + ((size_t)i * R.K + k) * 2 * BS, s);
}

// FP64 (or unstaged) form: blocks and factors straight from global memory.
template <int BS, bool kPattern>
__device__ __forceinline__ void sweep_pair_f64_body(const TileRow& R, const SweepIO& io, long long g, bool x_zero) {
  const int i = (int)fdiv((uint32_t)g, R.divK);
  const int k = (int)g - i * R.K;
  Cvec<BS, double> s;
  load_slice<BS>((const double*)R.Bt + ((size_t)i * R.K + k) * 2 * BS, s);
  if (!x_zero) {
    const double* __restrict__ X = (const double*)io.Xin;
    const double* __restrict__ offd = (const double*)R.offd;
    const int p0 = __ldg(R.row_ptr + i), p1 = __ldg(R.row_ptr + i + 1);
    for (int p = p0; p < p1; ++p) {
      const int cj = __ldg(R.col_idx + p);
      if (cut_of(cj)) continue;  // coupling to another partition: dropped
      Cvec<BS, double> x;
      load_slice<BS>(X + ((size_t)col_of(cj) * R.K + k) * 2 * BS, x);
      if (side_of(cj)) phase_shift<BS, double>(x.re, x.im, side_of(cj), io.phase[k]);
      double J[BS * BS];
      load_block<BS>(offd + (size_t)p * BS * BS, J);
      spmv_block_f64<BS>(J, x, s, kPattern);
    }
  }
  finish_pair<BS, double>(R, io, (const double*)R.hess + (size_t)i * BS * BS, i, k, s);
}

template <int BS>
__device__ __forceinline__ void sweep_pair_f64(const TileRow& R, const SweepIO& io, long long g, bool x_zero) {
  if (frozen_turbulence<BS>(R)) sweep_pair_f64_body<BS, true>(R, io, g, x_zero);
  else sweep_pair_f64_body<BS, false>(R, io, g, x_zero);
}

// FP64, system-major tile: a CTA owns 32 consecutive nodes and each warp
// takes whole systems for those nodes (lane = node).  The mean flow's warp
// (system 0, omega = 0) runs a real-only path -- half the multiply-adds of the
// complex path and a real back-substitution -- instead of carrying a zero
// imaginary part through the complex code.
template <int BS>
__device__ __forceinline__ void sweep_node_f64(const TileRow& R, const SweepIO& io, int i, int k, bool x_zero) {
  if (k != 0) {
    sweep_pair_f64<BS>(R, io, (long long)i * R.K + k, x_zero);
    return;
  }
  const double* bt = (const double*)R.Bt + (size_t)i * R.K * 2 * BS;  // system 0 slice: (re, 0) pairs
  double sr[BS];
#pragma unroll
  for (int t = 0; t < BS; ++t) sr[t] = __ldg(bt + 2 * t);
  if (!x_zero) {
    const double* __restrict__ X = (const double*)io.Xin;
    const double* __restrict__ offd = (const double*)R.offd;
    const bool pattern = frozen_turbulence<BS>(R);
    const int p0 = __ldg(R.row_ptr + i), p1 = __ldg(R.row_ptr + i + 1);
    for (int p = p0; p < p1; ++p) {
      const int cj = __ldg(R.col_idx + p);
      if (cut_of(cj)) continue;
      const int j = col_of(cj);  // the mean flow carries no phase
      const double* xs = X + (size_t)j * R.K * 2 * BS;
      double xr[BS];
#pragma unroll
      for (int t = 0; t < BS; ++t) xr[t] = __ldg(xs + 2 * t);
      double J[BS * BS];
      load_block<BS>(offd + (size_t)p * BS * BS, J);
      if (pattern) {
#pragma unroll
        for (int t = 0; t < BS; ++t) sr[0] -= J[t] * xr[t];
#pragma unroll
        for (int r = 1; r < BS; ++r)
#pragma unroll
          for (int t = 1; t < BS; ++t) sr[r] -= J[r * BS + t] * xr[t];
      } else {
#pragma unroll
        for (int r = 0; r < BS; ++r)
#pragma unroll
          for (int t = 0; t < BS; ++t) sr[r] -= J[r * BS + t] * xr[t];
      }
    }
  }
  const double* H = (const double*)R.hess + (size_t)i * BS * BS;
  bool tri = true;
#pragma unroll
  for (int q = 0; q < BS - 1; ++q) tri = tri && (H[(q + 1) * BS + q] == 0.0);
  double* xo = (double*)io.Xout + (size_t)i * R.K * 2 * BS;
  if (tri) {
    double inv[BS];
    if (R.pivinv) {
#pragma unroll
      for (int q = 0; q < BS; ++q) inv[q] = __ldg(R.pivinv + (size_t)i * R.K * BS * 2 + 2 * q);
    } else {
      double dg[BS];
#pragma unroll
      for (int q = 0; q < BS; ++q) dg[q] = H[q * BS + q];
      batch_recip<BS>(dg, inv);  // one division for the block
    }
#pragma unroll
    for (int q = BS - 1; q >= 0; --q) {
      double acc = sr[q];
#pragma unroll
      for (int c = q + 1; c < BS; ++c) acc -= H[q * BS + c] * sr[c];
      sr[q] = acc * inv[q];
    }
#pragma unroll
    for (int t = 0; t < BS; ++t) reinterpret_cast<double2*>(xo)[t] = make_double2(sr[t], 0.0);
  } else {
    Cvec<BS, double> v;
#pragma unroll
    for (int t = 0; t < BS; ++t) {
      v.re[t] = sr[t];
      v.im[t] = 0.0;
    }
    hess_solve<BS, double>(H, 0.0, v.re, v.im);
    store_slice<BS>(xo, v);
  }
}

// s -= J x for one staged FP32 block, consumed row by row from shared
// memory: six live block entries instead of thirty-six keep the register
// count (64, sixteen 64-thread CTAs per SM) without spilling.
template <int BS>
__device__ __forceinline__ void spmv_rows_smem(const float* jb, const Cvec<BS, float>& x, Cvec<BS, float>& s) {
#pragma unroll
  for (int r = 0; r < BS; ++r) {
    float jr[BS];
    if constexpr (BS % 2 == 0) {
#pragma unroll
      for (int t = 0; t < BS; t += 2) {
        const float2 f = reinterpret_cast<const float2*>(jb + r * BS)[t / 2];
        jr[t] = f.x;
        jr[t + 1] = f.y;
      }
    } else {
#pragma unroll
      for (int t = 0; t < BS; ++t) jr[t] = jb[r * BS + t];
    }
#pragma unroll
    for (int t = 0; t < BS; ++t) {
      s.re[r] -= jr[t] * x.re[t];
      s.im[r] -= jr[t] * x.im[t];
    }
  }
}

// s -= J x for one block read straight from global memory, row by row with
// vector loads (a row of an FP32 block starts on 8 bytes, of a BF16 block on
// 4 bytes, for even BS); the node's K threads share the block through L1.
template <int BS, typename TJ>
__device__ __forceinline__ void spmv_rows_global(const TJ* __restrict__ jb, const Cvec<BS, float>& x,
                                                 Cvec<BS, float>& s) {
#pragma unroll
  for (int r = 0; r < BS; ++r) {
    float jr[BS];
    if constexpr (BS % 2 == 0 && sizeof(TJ) == 2) {
      const uint32_t* q = reinterpret_cast<const uint32_t*>(jb + r * BS);
#pragma unroll
      for (int t = 0; t < BS / 2; ++t) {
        const uint32_t w = __ldg(q + t);
        jr[2 * t] = bf16_lo(w);
        jr[2 * t + 1] = bf16_hi(w);
      }
    } else if constexpr (BS % 2 == 0) {
      const float2* q = reinterpret_cast<const float2*>(jb + r * BS);
#pragma unroll
      for (int t = 0; t < BS / 2; ++t) {
        const float2 f = __ldg(q + t);
        jr[2 * t] = f.x;
        jr[2 * t + 1] = f.y;
      }
    } else {
#pragma unroll
      for (int t = 0; t < BS; ++t) jr[t] = ld<float, TJ>(jb + r * BS + t);
    }
#pragma unroll
    for (int t = 0; t < BS; ++t) {
      s.re[r] -= jr[t] * x.re[t];
      s.im[r] -= jr[t] * x.im[t];
    }
  }
}

// Staged FP32 form: one tile of blockDim.x consecutive pairs starting at g0,
// for rows of more than kRealMeanMaxSystems systems (complex slices only).
// Every thread of the CTA must call this (it synchronises).
template <int BS, typename TJ>
__device__ __forceinline__ void sweep_tile_f32(const TileRow& R, const SweepIO& io, long long g0, bool x_zero,
                                               float* smem, int smem_floats) {
  const uint32_t total = (uint32_t)R.n * (uint32_t)R.K;
  const uint32_t gs = (uint32_t)g0;
  const uint32_t g = gs + threadIdx.x;
  const int i_first = (int)fdiv(gs, R.divK);
  const uint32_t g_last = min(gs + blockDim.x, total) - 1;
  const int i_last = (int)fdiv(g_last, R.divK);
  const int nodes = i_last - i_first + 1;
  const int p_first = __ldg(R.row_ptr + i_first), p_end = __ldg(R.row_ptr + i_last + 1);
  const int nblk = x_zero ? 0 : (p_end - p_first);
  // blocks, factors and neighbour indices of the tile (uniform over the CTA)
  const bool staged = R.stage && (nblk + nodes) * BS * BS + nblk <= smem_floats;
  float* sJ = smem;
  float* sH = smem + nblk * BS * BS;
  int* sC = reinterpret_cast<int*>(sH + nodes * BS * BS);
  // the right-hand side slice is loaded first, so that it is in flight during the staging
  Cvec<BS, float> s;
  if (g < total) load_slice<BS>((const float*)R.Bt + (size_t)g * 2 * BS, s);
  if (staged) {
    const bool v4 = ((BS * BS) % 4 == 0);
    if (nblk > 0) {
      if constexpr (sizeof(TJ) == 2)
        stage_bf16(sJ, (const __nv_bfloat16*)R.offd + (size_t)p_first * BS * BS, nblk * BS * BS, v4);
      else
        stage_f32(sJ, (const float*)R.offd + (size_t)p_first * BS * BS, nblk * BS * BS, v4);
      stage_i32(sC, R.col_idx + p_first, nblk);
    }
    stage_f32(sH, (const float*)R.hess + (size_t)i_first * BS * BS, nodes * BS * BS, v4);
  }
  __syncthreads();
  if (g < total && !sys_active(io, (int)g - (int)fdiv(g, R.divK) * R.K)) {
    const int i = (int)fdiv(g, R.divK);
    freeze_pair<BS, float>(R, io, i, (int)g - i * R.K, x_zero);
  } else if (g < total) {
    const int i = (int)fdiv(g, R.divK);
    const int k = (int)g - i * R.K;
    if (!x_zero) {
      const float* __restrict__ Xk = (const float*)io.Xin + (size_t)k * 2 * BS;
      const size_t stride = (size_t)R.K * 2 * BS;
      const int p0 = __ldg(R.row_ptr + i), p1 = __ldg(R.row_ptr + i + 1);
      // software pipeline: the next neighbour's slice is in flight while the
      // current one is multiplied
      Cvec<BS, float> xn;
      int cn = 0;  // tagged column of the slice in flight
      if (p0 < p1) {
        cn = staged ? sC[p0 - p_first] : __ldg(R.col_idx + p0);
        load_slice<BS>(Xk + (size_t)col_of(cn) * stride, xn);
      }
      for (int p = p0; p < p1; ++p) {
        Cvec<BS, float> x = xn;
        const int cj = cn;
        if (p + 1 < p1) {
          cn = staged ? sC[p + 1 - p_first] : __ldg(R.col_idx + p + 1);
          load_slice<BS>(Xk + (size_t)col_of(cn) * stride, xn);
        }
        if (cut_of(cj)) continue;  // coupling to another partition: dropped
        if (side_of(cj)) phase_shift<BS, float>(x.re, x.im, side_of(cj), io.phase[k]);
        if (staged) spmv_rows_smem<BS>(sJ + (size_t)(p - p_first) * BS * BS, x, s);
        else spmv_rows_global<BS, TJ>((const TJ*)R.offd + (size_t)p * BS * BS, x, s);
      }
    }
    const float* H = staged ? sH + (size_t)(i - i_first) * BS * BS : (const float*)R.hess + (size_t)i * BS * BS;
    finish_pair<BS, float>(R, io, H, i, k, s);
  }
  __syncthreads();  // the stage buffer is reused by the next tile
}

}  // namespace fnlh
