// FP64 linear residual r_k = B_k - A_k x_k and its per-system 2-norms.
//
// Paper: arXiv 2404.01407, Results, Table fnlh_para (linear-residual
// threshold): each linear solve stops once ||B - A x||_2 has dropped by a
// fixed factor from its initial value, for the mean flow and each harmonic.  Here the residual is
// always formed in FP64 from the FP64 blocks in the original basis, which is
// what lets the mixed-precision sweeps be corrected back to FP64 accuracy.
//
// Determinism: a fixed grid walks tiles of 32 nodes in a fixed pattern; each
// block accumulates per-system sums in tile order through fixed shuffle
// trees, and one final pass sums the block partials in block order.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"

namespace fnlh {

struct ResArgs {
  int32_t n;
  const int32_t* row_ptr;
  const int32_t* col_idx;  // passage-tagged on a periodic mesh (col_of / side_of)
  const double* offd;
  const double* diag;
  const double* D;
  const double* vol;
  const double* B;
  const double* X;
  double* r;        // nullable [n][C][b]
  float* r32rot;    // nullable, internal FP32 layout: Q_i^T r_i in FP32 (r rounded to FP32 first)
  const float* rotf;  // Q_i in FP32 (with r32rot)
  const int32_t* info;  // prep info word, nullable: 0 = the b = 6 frozen-turbulence pattern holds
  int32_t x_zero;     // x is zero: r = B without reading X
  double* partials; // [gridDim][2K]
  Systems sys;
  // float-float form (k_residual_ff): the prep blob's copies and the solve's shadows
  const float2* offdff;  // [nnz][b][b]
  const float2* diagff;  // [n][b][b], J_ii + D_i I
  const float2* bff;     // [n][C][b]
  const float2* xff;     // [n][C][b]
  float2 omega_ff[kMaxSys];  // omega_k as a float-float pair
};

// r for one (node, system) pair; returns ||r||^2 and ||B||^2 contributions.
// The mean flow (k = 0) takes a real-only path.
template <int BS>
__device__ __forceinline__ void residual_pair(const ResArgs& a, int i, int k, double& rs, double& bs) {
  const int C = a.sys.C;
  const int c0 = (k == 0) ? 0 : 2 * k - 1;
  const bool cplx = k > 0;
  double br[BS], bi[BS], rr[BS], ri[BS];
  const double* bp = a.B + ((size_t)i * C + c0) * BS;
#pragma unroll
  for (int t = 0; t < BS; ++t) {
    br[t] = bp[t];
    bi[t] = cplx ? bp[BS + t] : 0.0;
    rr[t] = br[t];
    ri[t] = bi[t];
  }
  const int p0 = a.row_ptr[i], p1 = a.x_zero ? p0 : a.row_ptr[i + 1];
  // frozen turbulence (original basis): rows 0..4 of every block skip column 5
  bool pattern = false;
  if constexpr (BS == 6) pattern = a.info != nullptr && __ldg(a.info) == 0;
  if (cplx) {
    for (int p = p0; p < p1; ++p) {
      const int cj = a.col_idx[p];
      const double* xj = a.X + ((size_t)col_of(cj) * C + c0) * BS;
      double xr[BS], xi[BS];
#pragma unroll
      for (int t = 0; t < BS; ++t) {
        xr[t] = __ldg(xj + t);
        xi[t] = __ldg(xj + BS + t);
      }
      if (side_of(cj)) phase_shift<BS, double>(xr, xi, side_of(cj), a.sys.phase[k]);
      const double* J = a.offd + (size_t)p * BS * BS;
      if (pattern) {
#pragma unroll
        for (int q = 0; q < BS; ++q)
#pragma unroll
          for (int t = 0; t < ((q < BS - 1) ? BS - 1 : BS); ++t) {
            const double jv = __ldg(J + q * BS + t);
            rr[q] -= jv * xr[t];
            ri[q] -= jv * xi[t];
          }
      } else {
#pragma unroll
        for (int q = 0; q < BS; ++q)
#pragma unroll
          for (int t = 0; t < BS; ++t) {
            const double jv = __ldg(J + q * BS + t);
            rr[q] -= jv * xr[t];
            ri[q] -= jv * xi[t];
          }
      }
    }
  } else {
    for (int p = p0; p < p1; ++p) {
      const int j = col_of(a.col_idx[p]);  // the mean flow carries no phase
      const double* xj = a.X + (size_t)j * C * BS;
      double xr[BS];
#pragma unroll
      for (int t = 0; t < BS; ++t) xr[t] = __ldg(xj + t);
      const double* J = a.offd + (size_t)p * BS * BS;
      if (pattern) {
#pragma unroll
        for (int q = 0; q < BS; ++q)
#pragma unroll
          for (int t = 0; t < ((q < BS - 1) ? BS - 1 : BS); ++t) rr[q] -= __ldg(J + q * BS + t) * xr[t];
      } else {
#pragma unroll
        for (int q = 0; q < BS; ++q)
#pragma unroll
          for (int t = 0; t < BS; ++t) rr[q] -= __ldg(J + q * BS + t) * xr[t];
      }
    }
  }
  // diagonal block, D and the spectral term i omega V
  if (!a.x_zero) {
    const double* xp = a.X + ((size_t)i * C + c0) * BS;
    double xr[BS], xi[BS];
#pragma unroll
    for (int t = 0; t < BS; ++t) {
      xr[t] = xp[t];
      xi[t] = cplx ? xp[BS + t] : 0.0;
    }
    const double* P = a.diag + (size_t)i * BS * BS;
    const double Di = a.D[i];
    if (cplx) {
      const double wv = a.sys.omega[k] * a.vol[i];
#pragma unroll
      for (int q = 0; q < BS; ++q) {
#pragma unroll
        for (int t = 0; t < BS; ++t) {
          const double pv = __ldg(P + q * BS + t);
          rr[q] -= pv * xr[t];
          ri[q] -= pv * xi[t];
        }
        rr[q] -= Di * xr[q];
        ri[q] -= Di * xi[q];
        rr[q] += wv * xi[q];
        ri[q] -= wv * xr[q];
      }
    } else {
#pragma unroll
      for (int q = 0; q < BS; ++q) {
#pragma unroll
        for (int t = 0; t < BS; ++t) rr[q] -= __ldg(P + q * BS + t) * xr[t];
        rr[q] -= Di * xr[q];
      }
    }
  }
  rs = 0.0;
  bs = 0.0;
#pragma unroll
  for (int t = 0; t < BS; ++t) {
    rs += rr[t] * rr[t] + ri[t] * ri[t];
    bs += br[t] * br[t] + bi[t] * bi[t];
  }
  if (a.r) {
    double* rp = a.r + ((size_t)i * C + c0) * BS;
#pragma unroll
    for (int t = 0; t < BS; ++t) {
      rp[t] = rr[t];
      if (cplx) rp[BS + t] = ri[t];
    }
  }
  if (a.r32rot) {
    // Q_i^T r in the sweeps' internal FP32 layout (common.cuh, node_stride):
    // the inner solve only needs r to FP32 accuracy
    const float* Q = a.rotf + (size_t)i * BS * BS;
    float fr[BS], fi[BS];
#pragma unroll
    for (int t = 0; t < BS; ++t) {
      fr[t] = (float)rr[t];
      fi[t] = (float)ri[t];
    }
    float* rp = a.r32rot + slice_at<BS, float>(i, a.sys.K, k);
    const bool real = real_mean<float>(a.sys.K) && k == 0;
#pragma unroll
    for (int q = 0; q < BS; ++q) {
      float ar = 0.0f, ai = 0.0f;
#pragma unroll
      for (int t = 0; t < BS; ++t) {
        const float qv = __ldg(Q + t * BS + q);
        ar += qv * fr[t];
        ai += qv * fi[t];
      }
      if (real) {
        rp[mean_pos<BS>(q)] = ar;
      } else {
        rp[2 * q] = ar;
        rp[2 * q + 1] = cplx ? ai : 0.0f;
      }
    }
    if (real)
      for (int e = 0; e < kMeanSlot<BS>; ++e)
        if (mean_pad<BS>(e)) rp[e] = 0.0f;
  }
}

// One block walks tiles of 32 nodes (grid stride), kResidualRound tiles at a
// time: the round's (tile, system) items are dealt round-robin to the warps
// (lane = node), each reduced by a fixed shuffle tree into its own shared
// slot; then the slots are added to the block's per-system sums in tile
// order.  The work is balanced whatever K (the mean flow's real items cost
// half) and the sums are added in the same order as one writer per system
// would, so the result is bit-reproducible.
constexpr int kResidualRound = 8;

template <int BS>
__global__ void __launch_bounds__(kResidualThreads) k_residual(const __grid_constant__ ResArgs a) {
  __shared__ double s_acc[2 * kMaxSys];
  __shared__ double s_item[kResidualRound][2 * kMaxSys];
  const int K = a.sys.K;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int t = threadIdx.x; t < 2 * K; t += blockDim.x) s_acc[t] = 0.0;
  __syncthreads();
  const int tiles = (a.n + 31) / 32;
  const int mine = (tiles > (int)blockIdx.x) ? (tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  for (int m0 = 0; m0 < mine; m0 += kResidualRound) {
    const int rcount = min(kResidualRound, mine - m0);
    for (int it = warp; it < rcount * K; it += nwarps) {
      const int tl = it / K, k = it - tl * K;
      const int i = ((int)blockIdx.x + (m0 + tl) * (int)gridDim.x) * 32 + lane;
      double rs = 0.0, bs = 0.0;
      if (i < a.n) residual_pair<BS>(a, i, k, rs, bs);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        rs += __shfl_xor_sync(0xffffffffu, rs, off);
        bs += __shfl_xor_sync(0xffffffffu, bs, off);
      }
      if (lane == 0) {
        s_item[tl][2 * k] = rs;
        s_item[tl][2 * k + 1] = bs;
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * K; t += blockDim.x)
      for (int tl = 0; tl < rcount; ++tl) s_acc[t] += s_item[tl][t];
    __syncthreads();
  }
  for (int t = threadIdx.x; t < 2 * K; t += blockDim.x) a.partials[(size_t)blockIdx.x * 2 * K + t] = s_acc[t];
}

// Float-float residual of the mixed solve's checks, on the FP32 units: B, x,
// the blocks and J_ii + D_i I as FP32 pairs (hi + lo), each multiply-add of
// the FP64 form as one exact product of the high parts, FP32 cross terms and
// one exact subtraction (ff_sub_prod) -- about 44 bits, so a residual at 1e-8
// of ||B|| keeps ~5 significant digits.  Mapping: a warp takes kFfNodes
// nodes and a lane one row q of one node (30 lanes busy), so that a block's
// rows are read by consecutive lanes and each row, held in registers, serves
// up to kFfSys systems (two: with four 256-thread CTAs per SM at 64 registers
// the c3 mixed solves ran 1.2-1.7% faster than with four systems at 80
// registers and three CTAs); the rotation Q_i^T r to the sweeps' basis gathers the
// node's rows with shuffles.  Writes Q_i^T r (FP32) like the FP64 kernel, and
// per block the sums ||r_k||^2 and ||B_k||^2 (from B's high parts) in a
// fixed order.  Across a periodic edge (harmonics only) the row's product
// y = J_ij x_j is formed on its own and enters the residual as e^{+-i sigma_k} y,
// the phase factor split to float-float (ff_mul, ff_acc below).
constexpr int kFfSys = 2;

// a * b for float-float a and b, renormalised: the high parts' product
// exactly (TwoProduct), the cross terms in FP32, then Fast2Sum.
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  const float e = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, __fmaf_rn(a.x, b.x, -p)));
  const float h = __fadd_rn(p, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, p)));
}

// (h, l) += v for a float-float v: TwoSum of the high parts, the low parts
// added to l (the accumulator form of ff_sub_prod).
__device__ __forceinline__ void ff_acc(float& h, float& l, float2 v) {
  const float t = __fadd_rn(h, v.x);
  const float z = __fsub_rn(t, h);
  const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(t, z)), __fsub_rn(v.x, z));
  h = t;
  l = __fadd_rn(l, __fadd_rn(e, v.y));
}

// (h, l) as a renormalised float-float value (Fast2Sum: |l| small against h).
__device__ __forceinline__ float2 ff_norm(float h, float l) {
  const float t = __fadd_rn(h, l);
  return make_float2(t, __fsub_rn(l, __fsub_rn(t, h)));
}

template <int BS>
__global__ void __launch_bounds__(kResidualThreads, 4) k_residual_ff(const __grid_constant__ ResArgs a) {
  constexpr int kNodes = 30 / BS;  // nodes per warp: 5 for b = 6, 6 for b = 5
  constexpr int kWarps = kResidualThreads / 32;
  __shared__ double s_acc[kWarps][2 * kMaxSys];
  const int K = a.sys.K, C = a.sys.C;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int u = lane / BS, q = lane - u * BS;
  const bool live = lane < kNodes * BS;
  for (int t = lane; t < 2 * K; t += 32) s_acc[warp][t] = 0.0;
  __syncwarp();
  bool pattern = false;
  if constexpr (BS == 6) pattern = a.info != nullptr && __ldg(a.info) == 0;
  const int groups = (a.n + kNodes - 1) / kNodes;
  for (int grp = blockIdx.x * kWarps + warp; grp < groups; grp += gridDim.x * kWarps) {
    const int i = grp * kNodes + u;
    const bool valid = live && i < a.n;
    const int p0 = valid ? a.row_ptr[i] : 0, p1 = valid ? a.row_ptr[i + 1] : 0;
    const float2 vff = valid ? ff_split(a.vol[i]) : make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < K; k0 += kFfSys) {
      float rh[kFfSys], rl[kFfSys], ih[kFfSys], il[kFfSys];
      float bsq[kFfSys];
#pragma unroll
      for (int s = 0; s < kFfSys; ++s) {
        const int k = k0 + s;
        float2 br = make_float2(0.f, 0.f), bi = br;
        if (valid && k < K) {
          const int c0 = (k == 0) ? 0 : 2 * k - 1;
          br = a.bff[((size_t)i * C + c0) * BS + q];
          if (k > 0) bi = a.bff[((size_t)i * C + c0 + 1) * BS + q];
        }
        rh[s] = br.x;
        rl[s] = br.y;
        ih[s] = bi.x;
        il[s] = bi.y;
        bsq[s] = br.x * br.x + bi.x * bi.x;
      }
      // off-diagonal blocks: row q of J_ij times x_j for the pass's systems
      for (int p = p0; p < p1; ++p) {
        const int cj = a.col_idx[p];
        const int j = col_of(cj);
        const uint32_t side = side_of(cj);  // periodic edge: phase factor on the harmonics
        float2 jr[BS];
#pragma unroll
        for (int t = 0; t < BS; ++t) jr[t] = a.offdff[((size_t)p * BS + q) * BS + t];
        const bool skip_last = pattern && q < BS - 1;  // frozen turbulence: structural zero
#pragma unroll
        for (int s = 0; s < kFfSys; ++s) {
          const int k = k0 + s;
          if (k >= K) break;
          const int c0 = (k == 0) ? 0 : 2 * k - 1;
          const float2* xr = a.xff + ((size_t)j * C + c0) * BS;
          if (side != 0 && k > 0) {
            // y = -(J_ij x_j) of row q, then r += e^{+-i sigma_k} y
            float yrh = 0.f, yrl = 0.f, yih = 0.f, yil = 0.f;
#pragma unroll
            for (int t = 0; t < BS; ++t) {
              if (t == BS - 1 && skip_last) continue;
              ff_sub_prod(yrh, yrl, jr[t], xr[t]);
              ff_sub_prod(yih, yil, jr[t], xr[BS + t]);
            }
            const double2 ph = a.sys.phase[k];
            const float2 c = ff_split(ph.x), sn = ff_split(side == kSideNext ? ph.y : -ph.y);
            const float2 yr = ff_norm(yrh, yrl), yi = ff_norm(yih, yil);
            const float2 sy = ff_mul(sn, yi), sx = ff_mul(sn, yr);
            ff_acc(rh[s], rl[s], ff_mul(c, yr));
            ff_acc(rh[s], rl[s], make_float2(-sy.x, -sy.y));
            ff_acc(ih[s], il[s], sx);
            ff_acc(ih[s], il[s], ff_mul(c, yi));
            continue;
          }
#pragma unroll
          for (int t = 0; t < BS; ++t) {
            if (t == BS - 1 && skip_last) continue;
            ff_sub_prod(rh[s], rl[s], jr[t], xr[t]);
            if (k > 0) ff_sub_prod(ih[s], il[s], jr[t], xr[BS + t]);
          }
        }
      }
      // diagonal block (J_ii + D_i I) and the spectral term i omega_k V_i, then the outputs
      float2 pr[BS], qc[BS];
#pragma unroll
      for (int t = 0; t < BS; ++t) {
        pr[t] = valid ? a.diagff[((size_t)i * BS + q) * BS + t] : make_float2(0.f, 0.f);
        qc[t] = make_float2(valid ? __ldg(a.rotf + (size_t)i * BS * BS + t * BS + q) : 0.f, 0.f);  // Q[t][q]
      }
#pragma unroll
      for (int s = 0; s < kFfSys; ++s) {
        const int k = k0 + s;
        if (k >= K) break;  // uniform over the warp
        const int c0 = (k == 0) ? 0 : 2 * k - 1;
        if (valid) {
          const float2* xi = a.xff + ((size_t)i * C + c0) * BS;
#pragma unroll
          for (int t = 0; t < BS; ++t) {
            ff_sub_prod(rh[s], rl[s], pr[t], xi[t]);
            if (k > 0) ff_sub_prod(ih[s], il[s], pr[t], xi[BS + t]);
          }
          if (k > 0) {
            // r -= i w x: re += w x_im, im -= w x_re; w = omega_k V_i as a float-float product
            const float2 om = a.omega_ff[k];
            const float wp = __fmul_rn(om.x, vff.x);
            const float we = __fmaf_rn(om.x, vff.y, __fmaf_rn(om.y, vff.x, __fmaf_rn(om.x, vff.x, -wp)));
            ff_sub_prod(rh[s], rl[s], make_float2(-wp, -we), xi[BS + q]);
            ff_sub_prod(ih[s], il[s], make_float2(wp, we), xi[q]);
          }
        }
        const float r_re = valid ? __fadd_rn(rh[s], rl[s]) : 0.f;
        const float r_im = (valid && k > 0) ? __fadd_rn(ih[s], il[s]) : 0.f;
        // squares summed in FP32 over the warp (the checks need a few digits), added to
        // the block's FP64 sums once per warp and pass
        float rs = r_re * r_re + r_im * r_im;
        float bs = bsq[s];
        // Q_i^T r, row q: sum over the node's rows t, gathered from lanes u BS + t
        float o_re = 0.f, o_im = 0.f;
#pragma unroll
        for (int t = 0; t < BS; ++t) {
          const int src = min(u * BS + t, 31);
          const float vr = __shfl_sync(0xffffffffu, r_re, src);
          const float vi = __shfl_sync(0xffffffffu, r_im, src);
          o_re += qc[t].x * vr;
          o_im += qc[t].x * vi;
        }
        if (valid) {
          float* rp = a.r32rot + slice_at<BS, float>(i, K, k);
          if (!real_mean<float>(K) || k > 0) {
            rp[2 * q] = o_re;
            rp[2 * q + 1] = (k > 0) ? o_im : 0.0f;
          } else {  // a real mean flow: its values, then the pad
            rp[mean_pos<BS>(q)] = o_re;
            if (q == BS - 1)
              for (int e = 0; e < kMeanSlot<BS>; ++e)
                if (mean_pad<BS>(e)) rp[e] = 0.0f;
          }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          rs += __shfl_xor_sync(0xffffffffu, rs, off);
          bs += __shfl_xor_sync(0xffffffffu, bs, off);
        }
        if (lane == 0) {
          s_acc[warp][2 * k] += (double)rs;
          s_acc[warp][2 * k + 1] += (double)bs;
        }
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 2 * K; t += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < kWarps; ++w) v += s_acc[w][t];
    a.partials[(size_t)blockIdx.x * 2 * K + t] = v;
  }
}
// norms[t] = sum over blocks of partials[blk][t], in block order.
__global__ void k_reduce_partials(const double* __restrict__ partials, int nblk, int width, double* __restrict__ norms) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= width) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partials[(size_t)b * width + t];
  norms[t] = s;
}

// Fixed grid (a function of n only), so that repeated calls sum in the same order.
static int residual_grid(int n) {
  const int tiles = (n + 31) / 32;
  return tiles < 1 ? 1 : (tiles < kResidualGrid ? tiles : kResidualGrid);
}

int residual_launch(const fnlh_mesh* m, const fnlh_jacobian* J, const Systems& sys, const double* B,
                    const double* X, double* r, float* r32rot, const float* rotf, int x_zero, double* norms, void* ws,
                    cudaStream_t s) {
  const WsLayout W = ws_layout(J->n_nodes, J->block, sys.K - 1, FNLH_F64);
  ResArgs a{};
  a.n = J->n_nodes;
  a.row_ptr = m->row_ptr;
  a.col_idx = csr_columns(m, J);
  a.offd = J->offd;
  a.diag = J->diag;
  a.D = J->D;
  a.vol = m->vol;
  a.B = B;
  a.X = X;
  a.r = r;
  a.r32rot = r32rot;
  a.rotf = rotf;
  a.info = prep_info(J);
  a.x_zero = x_zero;
  a.partials = at<double>(ws, W.partials);
  a.sys = sys;
  const int grid = residual_grid(a.n);
  const int threads = kResidualThreads;
  if (J->block == 5) k_residual<5><<<grid, threads, 0, s>>>(a);
  else k_residual<6><<<grid, threads, 0, s>>>(a);
  FNLH_LAUNCH_CHECK();
  k_reduce_partials<<<1, 2 * kMaxSys, 0, s>>>(a.partials, grid, 2 * sys.K, norms);
  FNLH_LAUNCH_CHECK();
  return FNLH_OK;
}

// The float-float residual of a mixed solve's check: Q^T r in FP32 into
// r32rot, ||r_k||^2 (and ||B_k||^2 from B's high parts) into norms.  bff, xff:
// the solve's shadows of B and x; the prep blob must hold FNLH_PREP_FF.
int residual_ff_launch(const fnlh_mesh* m, const fnlh_jacobian* J, const Systems& sys, const float2* bff,
                       const float2* xff, float* r32rot, const float* rotf, double* norms, void* ws, cudaStream_t s) {
  const WsLayout W = ws_layout(J->n_nodes, J->block, sys.K - 1, FNLH_F64);
  const PrepLayout L = prep_layout(J->n_nodes, J->nnz, J->block, J->prep_flags);
  if (L.offdff == (size_t)-1) return FNLH_ERR_WORKSPACE;
  ResArgs a{};
  a.n = J->n_nodes;
  a.row_ptr = m->row_ptr;
  a.col_idx = csr_columns(m, J);
  a.offd = nullptr;
  a.diag = nullptr;
  a.D = nullptr;
  a.vol = m->vol;
  a.B = nullptr;
  a.X = nullptr;
  a.r = nullptr;
  a.r32rot = r32rot;
  a.rotf = rotf;
  a.info = prep_info(J);
  a.x_zero = 0;
  a.partials = at<double>(ws, W.partials);
  a.sys = sys;
  a.offdff = at<float2>(J->prep, L.offdff);
  a.diagff = at<float2>(J->prep, L.diagff);
  a.bff = bff;
  a.xff = xff;
  for (int k = 0; k < kMaxSys; ++k) {
    const float h = (float)sys.omega[k];
    a.omega_ff[k] = make_float2(h, (float)(sys.omega[k] - (double)h));
  }
  const int grid = residual_grid(a.n);
  if (J->block == 5) k_residual_ff<5><<<grid, kResidualThreads, 0, s>>>(a);
  else k_residual_ff<6><<<grid, kResidualThreads, 0, s>>>(a);
  FNLH_LAUNCH_CHECK();
  k_reduce_partials<<<1, 2 * kMaxSys, 0, s>>>(a.partials, grid, 2 * sys.K, norms);
  FNLH_LAUNCH_CHECK();
  return FNLH_OK;
}

// ------------------------------------------------------ allocation-free form
//
// fnlh_residual_noalloc runs the same two kernels as fnlh_residual, but keeps
// the per-block partial sums in the file-scope device array below instead of
// in a workspace the caller allocated.  The array holds the largest grid
// (kResidualGrid blocks) times two sums for the largest system count
// (1 + FNLH_MAX_HARMONICS), 1,264,640 bytes, and lives on every device that
// loads the library until the process exits.  Each call writes every slot it
// later reads, so nothing has to be cleared between calls; calls share the
// array, so two calls that may overlap on the GPU (other streams, other host
// threads) race on it.
constexpr size_t kNoAllocScratchDoubles = (size_t)kResidualGrid * 2 * kMaxSys;
static __device__ __align__(256) double g_residual_scratch[kNoAllocScratchDoubles];

// Device address of the scratch array in the current context.  The name
// g_residual_scratch in host code is only a host-side handle; the address is
// looked up on every call (the lookup allocates nothing), so that a context
// created after a device reset, or another context made current on the same
// device, never receives an address from an earlier one.
static int scratch_address(double** out) {
  double* p = nullptr;
  FNLH_CUDA_TRY(cudaGetSymbolAddress((void**)&p, g_residual_scratch));
  if (!p) return FNLH_ERR_CUDA;
  *out = p;
  return FNLH_OK;
}

int residual_noalloc_launch(const fnlh_mesh* m, const fnlh_jacobian* J, const Systems& sys, const double* B,
                            const double* X, double* r, double* norms, cudaStream_t s) {
  const int grid = residual_grid(J->n_nodes);
  if ((size_t)grid * 2 * sys.K > kNoAllocScratchDoubles) return FNLH_ERR_UNSUPPORTED;
  double* partials = nullptr;
  const int rc = scratch_address(&partials);
  if (rc) return rc;
  ResArgs a{};
  a.n = J->n_nodes;
  a.row_ptr = m->row_ptr;
  a.col_idx = csr_columns(m, J);
  a.offd = J->offd;
  a.diag = J->diag;
  a.D = J->D;
  a.vol = m->vol;
  a.B = B;
  a.X = X;
  a.r = r;
  a.r32rot = nullptr;
  a.rotf = nullptr;
  a.info = prep_info(J);
  a.x_zero = 0;
  a.partials = partials;
  a.sys = sys;
  const int threads = kResidualThreads;
  if (J->block == 5) k_residual<5><<<grid, threads, 0, s>>>(a);
  else k_residual<6><<<grid, threads, 0, s>>>(a);
  FNLH_LAUNCH_CHECK();
  k_reduce_partials<<<1, 2 * kMaxSys, 0, s>>>(partials, grid, 2 * sys.K, norms);
  FNLH_LAUNCH_CHECK();
  return FNLH_OK;
}

}  // namespace fnlh
