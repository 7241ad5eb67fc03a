// Vector kernels: deflation embed/extract (Eq. Vmatrix: V = (1/sqrt d)(v kron I),
// v the indicator of the diagonal components), deterministic dot products,
// copies. FP64, coalesced, grid-stride.
#include "common.cuh"

namespace dcg {
namespace {

// q[a] = (1/sqrt d) * sum_i y[a*b + i*d + i], ||q||^2 reduced.
template <int D>
__global__ void k_extract(const double* __restrict__ y, double* __restrict__ q, long long nn, double isd, Reduce red,
                          bool dot) {
  constexpr int B = D * D;
  double part[1] = {0.0};
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < nn;
       a += (long long)gridDim.x * blockDim.x) {
    double s = y[a * B];
#pragma unroll
    for (int i = 1; i < D; ++i) s += y[a * B + i * D + i];
    const double g = s * isd;
    q[a] = g;
    part[0] = fma(g, g, part[0]);
  }
  if (dot) grid_reduce<1>(part, red);
}

template <int D>
__global__ void k_embed(const double* __restrict__ q, double* __restrict__ y, long long nn, double isd) {
  constexpr int B = D * D;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn * B;
       t += (long long)gridDim.x * blockDim.x) {
    const long long a = t / B;
    const int c = (int)(t % B);
    y[t] = (c % (D + 1) == 0) ? __dmul_rn(isd, q[a]) : 0.0;
  }
}

__global__ void k_dot(const double* __restrict__ a, const double* __restrict__ b, long long n, Reduce red) {
  double part[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    part[0] = fma(a[i], b[i], part[0]);
  grid_reduce<1>(part, red);
}

}  // namespace

int vec_extract(dcg_problem* p, const double* y, double* q, int slot, cudaStream_t s) {
  const int g = grid_for(p->n_nodes, kRedThreads, kRedGrid);
  const double isd = 1.0 / sqrt((double)p->dim);
  Reduce red = make_reduce(p, slot < 0 ? S_TMP0 : slot);
  if (p->dim == 2) k_extract<2><<<g, kRedThreads, 0, s>>>(y, q, p->n_nodes, isd, red, slot >= 0);
  else k_extract<3><<<g, kRedThreads, 0, s>>>(y, q, p->n_nodes, isd, red, slot >= 0);
  DCG_LAUNCH_CHECK();
  return DCG_OK;
}

int vec_embed(dcg_problem* p, const double* q, double* y, cudaStream_t s) {
  const int g = grid_for(p->N, kRedThreads, 8192);
  const double isd = 1.0 / sqrt((double)p->dim);
  if (p->dim == 2) k_embed<2><<<g, kRedThreads, 0, s>>>(q, y, p->n_nodes, isd);
  else k_embed<3><<<g, kRedThreads, 0, s>>>(q, y, p->n_nodes, isd);
  DCG_LAUNCH_CHECK();
  return DCG_OK;
}

int vec_dot(dcg_problem* p, const double* a, const double* b, long long n, int slot, cudaStream_t s) {
  const int g = grid_for(n, kRedThreads, kRedGrid);
  k_dot<<<g, kRedThreads, 0, s>>>(a, b, n, make_reduce(p, slot));
  DCG_LAUNCH_CHECK();
  return DCG_OK;
}

int vec_copy(double* dst, const double* src, long long n, cudaStream_t s) {
  DCG_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  return DCG_OK;
}

int vec_zero(double* dst, long long n, cudaStream_t s) {
  DCG_CUDA(cudaMemsetAsync(dst, 0, sizeof(double) * n, s));
  return DCG_OK;
}

}  // namespace dcg
