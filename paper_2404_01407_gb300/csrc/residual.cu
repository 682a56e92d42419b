// FP64 linear residual r_k = B_k - A_k x_k and its per-system 2-norms.
//
// Paper: arXiv 2404.01407, Results ("A fixed threshold of 0.01 is used for the
// linear residual"): the stopping rule compares ||B - A x||_2 with its
// initial value, for the mean flow and each harmonic.  Here the residual is
// always formed in FP64 from the FP64 blocks in the original basis, which is
// what lets the mixed-precision sweeps be corrected back to FP64 accuracy.
//
// Determinism: a fixed grid walks the (node, system) pairs in a fixed
// pattern; every block reduces its pairs per system in index order through
// shared memory, and one final pass sums the block partials in block order.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

namespace fnlh {

struct ResArgs {
  int32_t n;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const double* offd;
  const double* diag;
  const double* D;
  const double* vol;
  const double* B;
  const double* X;
  double* r;        // nullable [n][C][b]
  float* r32rot;    // nullable [n][K][b] complex: Q_i^T r_i in FP32 (r rounded to FP32 first)
  const float* rotf;  // Q_i in FP32 (with r32rot)
  int32_t x_zero;     // x is zero: r = B without reading X
  double* partials; // [gridDim][2K]
  Systems sys;
};

template <int BS>
__global__ void __launch_bounds__(kResidualThreads) k_residual(ResArgs a) {
  __shared__ int s_k[kResidualThreads];
  __shared__ double s_r[kResidualThreads], s_b[kResidualThreads];
  const int K = a.sys.K, C = a.sys.C;
  const long long total = (long long)a.n * K;
  // per-block accumulators: thread t < 2K owns (system t/2, r or b)
  double acc = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += stride) {
    const long long g = base + threadIdx.x;
    double rs = 0.0, bs = 0.0;
    int kk = -1;
    if (g < total) {
      const int i = (int)(g / K);
      const int k = (int)(g - (long long)i * K);
      kk = k;
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
      for (int p = p0; p < p1; ++p) {
        const int j = a.col_idx[p];
        const double* xj = a.X + ((size_t)j * C + c0) * BS;
        double xr[BS], xi[BS];
#pragma unroll
        for (int t = 0; t < BS; ++t) {
          xr[t] = __ldg(xj + t);
          xi[t] = cplx ? __ldg(xj + BS + t) : 0.0;
        }
        const double* J = a.offd + (size_t)p * BS * BS;
#pragma unroll
        for (int q = 0; q < BS; ++q)
#pragma unroll
          for (int t = 0; t < BS; ++t) {
            const double jv = __ldg(J + q * BS + t);
            rr[q] -= jv * xr[t];
            ri[q] -= jv * xi[t];
          }
      }
      // diagonal block, D and the spectral term i omega V
      const double* xp = a.X + ((size_t)i * C + c0) * BS;
      double xr[BS], xi[BS];
#pragma unroll
      for (int t = 0; t < BS; ++t) {
        xr[t] = a.x_zero ? 0.0 : xp[t];
        xi[t] = (cplx && !a.x_zero) ? xp[BS + t] : 0.0;
      }
      const double* P = a.diag + (size_t)i * BS * BS;
      const double Di = a.D[i];
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
        // Q_i^T r in the sweeps' internal layout [n][K][b] complex, in FP32:
        // the inner solve only needs r to FP32 accuracy (the mean flow's
        // imaginary part is written as an exact zero)
        const float* Q = a.rotf + (size_t)i * BS * BS;
        float fr[BS], fi[BS];
#pragma unroll
        for (int t = 0; t < BS; ++t) {
          fr[t] = (float)rr[t];
          fi[t] = (float)ri[t];
        }
        float* rp = a.r32rot + ((size_t)i * K + k) * 2 * BS;
#pragma unroll
        for (int q = 0; q < BS; ++q) {
          float ar = 0.0f, ai = 0.0f;
#pragma unroll
          for (int t = 0; t < BS; ++t) {
            const float qv = __ldg(Q + t * BS + q);
            ar += qv * fr[t];
            ai += qv * fi[t];
          }
          rp[2 * q] = ar;
          rp[2 * q + 1] = cplx ? ai : 0.0f;
        }
      }
    }
    s_k[threadIdx.x] = kk;
    s_r[threadIdx.x] = rs;
    s_b[threadIdx.x] = bs;
    __syncthreads();
    if (threadIdx.x < 2 * K) {
      const int mine = threadIdx.x >> 1;
      const bool want_b = threadIdx.x & 1;
      for (int t = 0; t < blockDim.x; ++t)
        if (s_k[t] == mine) acc += want_b ? s_b[t] : s_r[t];
    }
    __syncthreads();
  }
  if (threadIdx.x < 2 * K) a.partials[(size_t)blockIdx.x * 2 * K + threadIdx.x] = acc;
}

// norms[t] = sum over blocks of partials[blk][t], in block order.
__global__ void k_reduce_partials(const double* __restrict__ partials, int nblk, int width, double* __restrict__ norms) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= width) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partials[(size_t)b * width + t];
  norms[t] = s;
}

int residual_launch(const fnlh_mesh* m, const fnlh_jacobian* J, const Systems& sys, const double* B,
                    const double* X, double* r, float* r32rot, const float* rotf, int x_zero, double* norms, void* ws,
                    cudaStream_t s) {
  const WsLayout W = ws_layout(J->n_nodes, J->block, sys.K - 1, FNLH_F64);
  ResArgs a;
  a.n = J->n_nodes;
  a.row_ptr = m->row_ptr;
  a.col_idx = m->col_idx;
  a.offd = J->offd;
  a.diag = J->diag;
  a.D = J->D;
  a.vol = m->vol;
  a.B = B;
  a.X = X;
  a.r = r;
  a.r32rot = r32rot;
  a.rotf = rotf;
  a.x_zero = x_zero;
  a.partials = at<double>(ws, W.partials);
  a.sys = sys;
  const long long total = (long long)a.n * sys.K;
  long long need = (total + kResidualThreads - 1) / kResidualThreads;
  const int grid = (int)(need < kResidualGrid ? (need > 0 ? need : 1) : kResidualGrid);
  if (J->block == 5) k_residual<5><<<grid, kResidualThreads, 0, s>>>(a);
  else k_residual<6><<<grid, kResidualThreads, 0, s>>>(a);
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

constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mu;
static double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The name
// g_residual_scratch in host code is only a host-side handle, so the address
// is looked up once per device with that device current and cached.
static int scratch_address(double** out) {
  int dev = 0;
  FNLH_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return FNLH_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    double* p = nullptr;
    FNLH_CUDA_TRY(cudaGetSymbolAddress((void**)&p, g_residual_scratch));
    if (!p) return FNLH_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return FNLH_OK;
}

int residual_noalloc_launch(const fnlh_mesh* m, const fnlh_jacobian* J, const Systems& sys, const double* B,
                            const double* X, double* r, double* norms, cudaStream_t s) {
  const long long total = (long long)J->n_nodes * sys.K;
  const long long need = (total + kResidualThreads - 1) / kResidualThreads;
  const int grid = (int)(need < kResidualGrid ? (need > 0 ? need : 1) : kResidualGrid);
  if ((size_t)grid * 2 * sys.K > kNoAllocScratchDoubles) return FNLH_ERR_UNSUPPORTED;
  double* partials = nullptr;
  const int rc = scratch_address(&partials);
  if (rc) return rc;
  ResArgs a;
  a.n = J->n_nodes;
  a.row_ptr = m->row_ptr;
  a.col_idx = m->col_idx;
  a.offd = J->offd;
  a.diag = J->diag;
  a.D = J->D;
  a.vol = m->vol;
  a.B = B;
  a.X = X;
  a.r = r;
  a.r32rot = nullptr;
  a.rotf = nullptr;
  a.x_zero = 0;
  a.partials = partials;
  a.sys = sys;
  if (J->block == 5) k_residual<5><<<grid, kResidualThreads, 0, s>>>(a);
  else k_residual<6><<<grid, kResidualThreads, 0, s>>>(a);
  FNLH_LAUNCH_CHECK();
  k_reduce_partials<<<1, 2 * kMaxSys, 0, s>>>(partials, grid, 2 * sys.K, norms);
  FNLH_LAUNCH_CHECK();
  return FNLH_OK;
}

}  // namespace fnlh
