// Arithmetic peak probe: FP64 and FP32 multiply-add throughput of this GPU
// (the figure the FP64 sweep's roofline is taken against; no library figure
// for FP64 exists here).
//
// Each thread keeps `chains` x `reuse` independent accumulators and, for
// `iters` steps, updates acc[k][r] <- j[k] * x[r] + acc[k][r]: every j[k]
// feeds `reuse` consecutive multiply-adds, the operand pattern of the
// block-times-slice products of the sweeps (one block entry times the real
// and the imaginary part of a slice).  On GB300 the FP64 rate depends on the
// operand pattern: about 1.06 TFLOP/s for a bare dependent chain
// x <- x m + c, 1.16 for pairs sharing an operand, 1.23 for 8 chains x 2
// with every operand in a register (97% of 152 SMs x 2 FMA/clk x 2.07 GHz);
// the search takes the best.  Counted work: 2 flops x chains x reuse x iters
// per thread; the grid is `blocks` x `threads`.  The accumulators' sum goes
// to `sink` (caller-owned device memory, one double per thread), so nothing
// is removed by the compiler.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fnlh_probe.h"

namespace {

// One fused multiply-add per step.  Spelled as a call, not as j * x + acc:
// the product of loop-invariant operands could otherwise be hoisted out of
// the loop, leaving additions to be timed.
__device__ __forceinline__ double fma_op(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_op(float a, float b, float c) { return fmaf(a, b, c); }

template <typename T, int kChains, int kReuse>
__global__ void __launch_bounds__(1024) k_fma(int iters, T m, double* __restrict__ sink) {
  // operands from a run-time value: registers, like the sweeps' block entries
  // (compile-time constants could be taken from the constant bank instead)
  T j[kChains], x[kReuse], acc[kChains][kReuse];
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    j[k] = m - (T)(1e-3 * k);
#pragma unroll
    for (int r = 0; r < kReuse; ++r) acc[k][r] = (T)0;
  }
#pragma unroll
  for (int r = 0; r < kReuse; ++r) x[r] = (T)(1e-7 * (threadIdx.x + 1 + r));
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k)
#pragma unroll
      for (int r = 0; r < kReuse; ++r) acc[k][r] = fma_op(j[k], x[r], acc[k][r]);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k)
#pragma unroll
    for (int r = 0; r < kReuse; ++r) s += acc[k][r];
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = (double)s;
}

template <typename T, int kChains>
cudaError_t launch_reuse(int reuse, int blocks, int threads, int iters, double* sink, cudaStream_t s) {
  if (reuse == 1) k_fma<T, kChains, 1><<<blocks, threads, 0, s>>>(iters, (T)1, sink);
  else if (reuse == 2) k_fma<T, kChains, 2><<<blocks, threads, 0, s>>>(iters, (T)1, sink);
  else k_fma<T, kChains, 4><<<blocks, threads, 0, s>>>(iters, (T)1, sink);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch(int chains, int reuse, int blocks, int threads, int iters, double* sink, cudaStream_t s) {
  if (chains == 4) return launch_reuse<T, 4>(reuse, blocks, threads, iters, sink, s);
  if (chains == 8) return launch_reuse<T, 8>(reuse, blocks, threads, iters, sink, s);
  return launch_reuse<T, 16>(reuse, blocks, threads, iters, sink, s);
}

}  // namespace

extern "C" int fnlh_probe_fma(int32_t precision, int32_t chains, int32_t reuse, int32_t blocks, int32_t threads,
                              int32_t iters, double* sink, float* ms, void* stream) {
  if (blocks <= 0 || iters <= 0 || !sink || !ms || (precision != 0 && precision != 1)) return -1;
  if ((chains != 4 && chains != 8 && chains != 16) || (reuse != 1 && reuse != 2 && reuse != 4)) return -1;
  if (threads < 32 || threads > 1024 || threads % 32) return -1;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess) return -2;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -2;
  }
  int rc = 0;
  if (cudaEventRecord(e0, s) != cudaSuccess) rc = -2;
  if (!rc) {
    const cudaError_t e = (precision == 0) ? launch<double>(chains, reuse, blocks, threads, iters, sink, s)
                                           : launch<float>(chains, reuse, blocks, threads, iters, sink, s);
    if (e != cudaSuccess) rc = -2;
  }
  if (!rc && cudaEventRecord(e1, s) != cudaSuccess) rc = -2;
  if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = -2;
  if (!rc && cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) rc = -2;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}
