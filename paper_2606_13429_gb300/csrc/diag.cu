// Diagnostics with no counterpart in the paper: the arithmetic rates the
// rooflines of the FP64 and FP32 kernels are measured against, and a
// self-test of the bounded mbarrier wait that the bulk-copy kernels use.
#include "common.cuh"
#include "tma.cuh"

#include <cstdio>

namespace dcg {
namespace {

// Eight independent FMA chains per thread (enough to cover the FMA latency
// with 8 warps per scheduler); the result is stored only if it equals a value
// it never takes, which keeps every FMA live without memory traffic.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_rate(T* __restrict__ sink, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x & 7) + (T)k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == (T)-7.25) sink[0] = s;
}

// Waits on an mbarrier that nothing completes (no arrival, no copy in
// flight): the bounded wait must give up after max_polls polls and the kernel
// records it in *err, then returns normally.
__global__ void k_wait_selftest(unsigned max_polls, double* __restrict__ err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0, max_polls);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) *err = 1.0;
}

template <typename T>
int fma_rate(double* tflops, cudaStream_t s) {
  const int ctas = 152 * 8, threads = 256;
  const int iters = sizeof(T) == 8 ? 4096 : 131072;
  T* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = DCG_OK;
  if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    set_error_msg("dcg_measure_fma_rate: setup failed");
    rc = DCG_ERR_CUDA;
  }
  float best = 0.f;
  for (int rep = 0; rep < 4 && rc == DCG_OK; ++rep) {  // first launch warms up
    cudaEventRecord(e0, s);
    k_fma_rate<T><<<ctas, threads, 0, s>>>(sink, iters, (T)0.999999, (T)1e-7);
    note_launches(1);
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      set_error_msg("dcg_measure_fma_rate: launch failed");
      rc = DCG_ERR_CUDA;
      break;
    }
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (rc == DCG_OK) *tflops = 2.0 * 8.0 * iters * (double)ctas * threads / (best * 1e-3) / 1e12;
  if (sink) cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return rc;
}

}  // namespace
}  // namespace dcg

using namespace dcg;

extern "C" int dcg_measure_fma_rate(int precision, double* tflops, void* stream) {
  if (!tflops || (precision != DCG_FP64 && precision != DCG_MIXED)) {
    set_error_msg("dcg_measure_fma_rate: need tflops and precision DCG_FP64 or DCG_MIXED (FP32)");
    return DCG_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  return precision == DCG_FP64 ? fma_rate<double>(tflops, s) : fma_rate<float>(tflops, s);
}

extern "C" int dcg_selftest_bounded_wait(unsigned max_polls, int* gave_up, void* stream) {
  if (!gave_up || max_polls == 0) {
    set_error_msg("dcg_selftest_bounded_wait: need gave_up and max_polls > 0");
    return DCG_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* err = nullptr;
  DCG_CUDA(cudaMalloc(&err, sizeof(double)));
  double h = 0.0;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(double), s);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 128, 0, s>>>(max_polls, err);
    note_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(err);
  if (e != cudaSuccess) {
    set_error("dcg_selftest_bounded_wait", e);
    return DCG_ERR_CUDA;
  }
  *gave_up = h != 0.0 ? 1 : 0;
  return DCG_OK;
}
