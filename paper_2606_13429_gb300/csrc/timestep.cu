// Implicit time stepping (Section 2.3, Eq. weak_IE) and the reconstruction
// of pressure and velocity (Section 5.2) on the device, FP64.
//
// A step solves A_alpha sigma^n = b^n with this library's operator
// A_alpha = M_dev / alpha + K_div (the paper's M + alpha A divided by alpha):
//   implicit Euler  alpha = dt      b = (M/alpha) s1 + F1
//   Crank-Nicolson  alpha = dt/2    b = (M/alpha - K) s1 + F1 + F0
//   BDF2            alpha = 2dt/3   b = (M/alpha)(4/3 s1 - 1/3 s2) + F1
// with (M/alpha) w formed as A_alpha w - K_div w: the assembled product and
// the constant divergence stencil of the uniform Q1 mesh (K_div does not
// depend on nu or dt). The problem is assembled once with alpha, and its
// set-up (inner hierarchy, Z_J = V^T A V, which does not depend on dt) serves
// every step.
#include "common.cuh"

#include <cmath>
#include <cstdio>

namespace dcg {
namespace {

struct DivSt {
  double c[9][27];
};

// y = a1 s1 + a2 s2 (s2 may be null)
__global__ void k_ts_combine(double* __restrict__ y, const double* __restrict__ s1, const double* __restrict__ s2,
                             double a1, double a2, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = s2 ? a1 * s1[i] + a2 * s2[i] : a1 * s1[i];
}

// y = K_div x: component (k, p) of node a is sum_q sum_o G[p][q][o] x_{a+o,(k,q)}
template <int D>
__global__ void k_ts_div_apply(const double* __restrict__ x, double* __restrict__ y, DivSt G, int m, long long nn) {
  constexpr int B = D * D, NO = D == 2 ? 9 : 27;
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < nn; a += (long long)gridDim.x * blockDim.x) {
    int c[3];
    long long r = a;
    c[0] = (int)(r % m);
    r /= m;
    c[1] = (int)(r % m);
    c[2] = D > 2 ? (int)(r / m) : 0;
    double acc[B];
#pragma unroll
    for (int t = 0; t < B; ++t) acc[t] = 0.0;
    for (int o = 0; o < NO; ++o) {
      const int xx = c[0] + o % 3 - 1, yy = c[1] + (o / 3) % 3 - 1, zz = c[2] + o / 9 - 1;
      if (xx < 0 || xx >= m || yy < 0 || yy >= m || (D > 2 && (zz < 0 || zz >= m))) continue;
      const double* xb = x + (xx + (long long)m * (yy + (long long)m * (D > 2 ? zz : 0))) * B;
#pragma unroll
      for (int k = 0; k < D; ++k)
#pragma unroll
        for (int p = 0; p < D; ++p)
#pragma unroll
          for (int q = 0; q < D; ++q) acc[k * D + p] = fma(G.c[p * 3 + q][o], xb[k * D + q], acc[k * D + p]);
    }
#pragma unroll
    for (int t = 0; t < B; ++t) y[a * B + t] = acc[t];
  }
}

// b = t - gamma kw + F1 + beta F0 (F0 may be null)
__global__ void k_ts_rhs(double* __restrict__ b, const double* __restrict__ t, const double* __restrict__ kw,
                         const double* __restrict__ F1, const double* __restrict__ F0, double gamma, double beta,
                         long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = t[i] - gamma * kw[i] + F1[i];
    if (F0) v += beta * F0[i];
    b[i] = v;
  }
}

// p = -(1/d) tr(sigma) at every interior node
template <int D>
__global__ void k_ts_pressure(const double* __restrict__ s, double* __restrict__ pres, long long nn) {
  constexpr int B = D * D;
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < nn; a += (long long)gridDim.x * blockDim.x) {
    double tr = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) tr += s[a * B + i * D + i];
    pres[a] = -tr / D;
  }
}

// (div sigma)_k at element centres: for each axis p the mean over the
// element's 2^(d-1) edges along p of (upper - lower) / h; boundary nodes 0
template <int D>
__global__ void k_ts_divergence(const double* __restrict__ s, double* __restrict__ out, int n, double inv_h,
                                long long ne) {
  constexpr int B = D * D, NC = 1 << D;
  const int m = n - 1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
    int ec[3];
    long long r = e;
    ec[0] = (int)(r % n);
    r /= n;
    ec[1] = (int)(r % n);
    ec[2] = D > 2 ? (int)(r / n) : 0;
    double dv[D];
#pragma unroll
    for (int k = 0; k < D; ++k) dv[k] = 0.0;
#pragma unroll
    for (int bits = 0; bits < NC; ++bits) {
      int nd[3];
      bool inner = true;
#pragma unroll
      for (int ax = 0; ax < D; ++ax) {
        nd[ax] = ec[ax] + ((bits >> ax) & 1);
        inner = inner && nd[ax] > 0 && nd[ax] < n;
      }
      if (!inner) continue;
      long long a = 0, st = 1;
#pragma unroll
      for (int ax = 0; ax < D; ++ax) {
        a += (long long)(nd[ax] - 1) * st;
        st *= m;
      }
#pragma unroll
      for (int p = 0; p < D; ++p) {
        const double g = (((bits >> p) & 1) ? inv_h : -inv_h) * (D == 2 ? 0.5 : 0.25);
#pragma unroll
        for (int k = 0; k < D; ++k) dv[k] = fma(g, s[a * B + k * D + p], dv[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) out[e * D + k] = dv[k];
  }
}

// u += w1 div1 + w0 div0 (div0 may be null)
__global__ void k_ts_velocity(double* __restrict__ u, const double* __restrict__ div1, const double* __restrict__ div0,
                              double w1, double w0, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = u[i] + w1 * div1[i];
    if (div0) v += w0 * div0[i];
    u[i] = v;
  }
}

int gn(long long n) { return grid_for(n, 256, 8192); }

double alpha_of(int scheme, double dt) {
  return scheme == DCG_IMPLICIT_EULER ? dt : scheme == DCG_CRANK_NICOLSON ? dt / 2.0 : 2.0 * dt / 3.0;
}

int div_apply(const dcg_problem* p, const double* x, double* y, cudaStream_t s) {
  DivSt G;
  div_stencil(p->dim, p->n, G.c);
  if (p->dim == 2) k_ts_div_apply<2><<<gn(p->n_nodes), 256, 0, s>>>(x, y, G, p->m, p->n_nodes);
  else k_ts_div_apply<3><<<gn(p->n_nodes), 256, 0, s>>>(x, y, G, p->m, p->n_nodes);
  DCG_LAUNCH_CHECK();
  return DCG_OK;
}

// b from s1, s2 (BDF2), F1 and F0 (CN); w, t, kw: scratch of N doubles
int time_rhs(dcg_problem* p, int scheme, const double* s1, const double* s2, const double* F1, const double* F0,
             double* b, double* w, double* t, double* kw, cudaStream_t s) {
  const long long N = p->N;
  if (scheme == DCG_BDF2) k_ts_combine<<<gn(N), 256, 0, s>>>(w, s1, s2 ? s2 : s1, 4.0 / 3.0, -1.0 / 3.0, N);
  else k_ts_combine<<<gn(N), 256, 0, s>>>(w, s1, nullptr, 1.0, 0.0, N);
  DCG_LAUNCH_CHECK();
  DCG_TRY(spmv_plain(p, w, t, s));
  DCG_TRY(div_apply(p, w, kw, s));
  const bool cn = scheme == DCG_CRANK_NICOLSON;
  k_ts_rhs<<<gn(N), 256, 0, s>>>(b, t, kw, F1, cn ? F0 : nullptr, cn ? 2.0 : 1.0, 1.0, N);
  DCG_LAUNCH_CHECK();
  return DCG_OK;
}

int divergence(const dcg_problem* p, const double* sigma, double* out, cudaStream_t s) {
  long long ne = 1;
  for (int k = 0; k < p->dim; ++k) ne *= p->n;
  if (p->dim == 2) k_ts_divergence<2><<<gn(ne), 256, 0, s>>>(sigma, out, p->n, (double)p->n, ne);
  else k_ts_divergence<3><<<gn(ne), 256, 0, s>>>(sigma, out, p->n, (double)p->n, ne);
  DCG_LAUNCH_CHECK();
  return DCG_OK;
}

bool scheme_ok(int scheme) {
  return scheme == DCG_IMPLICIT_EULER || scheme == DCG_CRANK_NICOLSON || scheme == DCG_BDF2;
}

}  // namespace
}  // namespace dcg

using namespace dcg;

extern "C" {

double dcg_scheme_alpha(int scheme, double dt) { return scheme_ok(scheme) ? alpha_of(scheme, dt) : -1.0; }

int dcg_apply_div(const dcg_problem* p, const double* x, double* y, void* stream) {
  if (!p || !x || !y || p->matrix_free) {
    set_error_msg("dcg_apply_div: need an assembled problem and device arrays x, y");
    return DCG_ERR_INVALID_ARG;
  }
  return div_apply(p, x, y, (cudaStream_t)stream);
}

int dcg_time_rhs(dcg_problem* p, int scheme, const double* s1, const double* s2, const double* F1, const double* F0,
                 double* rhs, void* stream) {
  if (!p || !s1 || !F1 || !rhs || !scheme_ok(scheme) || p->matrix_free ||
      (scheme == DCG_CRANK_NICOLSON && !F0)) {
    set_error_msg("dcg_time_rhs: need an assembled problem, a scheme, s1, F1 (and F0 for Crank-Nicolson), rhs");
    return DCG_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* tmp = nullptr;
  DCG_CUDA(cudaMallocAsync(&tmp, sizeof(double) * 3 * p->N, s));
  const int st = time_rhs(p, scheme, s1, s2, F1, F0, rhs, tmp, tmp + p->N, tmp + 2 * p->N, s);
  cudaFreeAsync(tmp, s);
  return st;
}

int dcg_pressure(const dcg_problem* p, const double* sigma, double* pres, void* stream) {
  if (!p || !sigma || !pres) return DCG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (p->dim == 2) k_ts_pressure<2><<<gn(p->n_nodes), 256, 0, s>>>(sigma, pres, p->n_nodes);
  else k_ts_pressure<3><<<gn(p->n_nodes), 256, 0, s>>>(sigma, pres, p->n_nodes);
  DCG_LAUNCH_CHECK();
  return DCG_OK;
}

int dcg_divergence(const dcg_problem* p, const double* sigma, double* div_elem, void* stream) {
  if (!p || !sigma || !div_elem) return DCG_ERR_INVALID_ARG;
  return divergence(p, sigma, div_elem, (cudaStream_t)stream);
}

int dcg_time_integrate(dcg_problem* p, int scheme, double dt, int nsteps, const double* sigma0,
                       const double* const* F, double* const* sigma_out, double* u_elem, double tol, int max_it,
                       dcg_stats* stats, void* stream) {
  if (!p || !sigma0 || !F || !sigma_out || nsteps < 1 || !scheme_ok(scheme) || !(dt > 0) || !(tol > 0) ||
      p->matrix_free) {
    set_error_msg("dcg_time_integrate: need an assembled problem, a scheme, dt > 0, nsteps >= 1, sigma0, F, "
                  "sigma_out, tol > 0");
    return DCG_ERR_INVALID_ARG;
  }
  for (int k = 0; k <= nsteps; ++k)
    if (!F[k] || (k < nsteps && !sigma_out[k])) return DCG_ERR_INVALID_ARG;
  const double alpha = alpha_of(scheme, dt);
  if (!(std::fabs(p->dt - alpha) <= 1e-12 * alpha)) {
    char buf[200];
    snprintf(buf, sizeof buf, "dcg_time_integrate: the problem was assembled with dt = %.17g, the scheme needs "
             "alpha = %.17g (dcg_scheme_alpha)", p->dt, alpha);
    set_error_msg(buf);
    return DCG_ERR_INVALID_ARG;
  }
  if (!p->is_setup) return DCG_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  const long long N = p->N;
  long long ne = 1;
  for (int k = 0; k < p->dim; ++k) ne *= p->n;
  const long long nd = ne * p->dim;
  double* tmp = nullptr;
  DCG_CUDA(cudaMalloc(&tmp, sizeof(double) * (4 * N + 2 * nd)));
  double *b = tmp, *w = tmp + N, *t = tmp + 2 * N, *kw = tmp + 3 * N;
  double *div_prev = tmp + 4 * N, *div_cur = div_prev + nd;
  int rc = DCG_OK;
  if (u_elem && scheme == DCG_CRANK_NICOLSON) rc = divergence(p, sigma0, div_prev, s);
  for (int k = 0; k < nsteps && rc == DCG_OK; ++k) {
    const double* s1 = k == 0 ? sigma0 : sigma_out[k - 1];
    const double* s2 = k == 0 ? sigma0 : (k == 1 ? sigma0 : sigma_out[k - 2]);
    rc = time_rhs(p, scheme, s1, scheme == DCG_BDF2 ? s2 : nullptr, F[k + 1], F[k], b, w, t, kw, s);
    if (rc != DCG_OK) break;
    // initial guess: the previous step
    if (cudaMemcpyAsync(sigma_out[k], s1, sizeof(double) * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
      rc = DCG_ERR_CUDA;
      break;
    }
    dcg_stats local{};
    dcg_stats* st = stats ? &stats[k] : &local;
    rc = solve_device(p, b, sigma_out[k], tol, max_it, st, s);
    if (rc == DCG_ERR_NOT_CONVERGED || rc == DCG_ERR_BREAKDOWN) break;
    if (rc != DCG_OK) break;
    if (u_elem) {
      rc = divergence(p, sigma_out[k], div_cur, s);
      if (rc != DCG_OK) break;
      if (scheme == DCG_CRANK_NICOLSON)
        k_ts_velocity<<<gn(nd), 256, 0, s>>>(u_elem, div_cur, div_prev, 0.5 * dt, 0.5 * dt, nd);
      else
        k_ts_velocity<<<gn(nd), 256, 0, s>>>(u_elem, div_cur, nullptr, dt, 0.0, nd);
      note_launches(1);
      if (cudaGetLastError() != cudaSuccess) {
        rc = DCG_ERR_CUDA;
        break;
      }
      std::swap(div_prev, div_cur);
    }
  }
  cudaStreamSynchronize(s);
  cudaFree(tmp);
  return rc;
}

}  // extern "C"
