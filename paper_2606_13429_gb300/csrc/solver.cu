// Outer solvers on the device, FP64: plain CG, and the flexible deflated CG
// of Algorithm 2 with the FCG recurrences of Algorithm 1.
//
//   pi(z)   = V Multigrid(V^T z, tau_c)                          (Algorithm 2)
//   M_D(d)  = A (d - pi(A d))                                    (Algorithm 2)
//   f_D     = f - A pi(f)   (the right-hand side of Eq. defl_sys, (I - pi_A)^T f)
//   x_hat   = FCG(f_D, x0, M_D)                                  (Algorithm 1)
//   x       = x_hat - pi(A x_hat) + pi(f)                        (Eq. x_defl)
//
// Outer stop ||r_i|| <= tol ||f|| on the recursive deflated residual
// (Section 4.1). Inner tolerance relative to ||V^T A d||: fixed
// tau_c = c tol (Eq. fixed_tol with c = c_F) or adaptive
// tau_c = c tol ||f|| / ||r_i|| (Eq. tol, c = c_A). pi(f) appears twice in
// Algorithm 2 with the same arguments and is computed once.
// After reconstruction the true residual ||f - A x|| / ||f|| is computed in
// FP64; above tol, the same solver runs on A e = f - A x (same absolute
// threshold) and x += e, at most max_restarts times.
//
// Per outer iteration (kernels, all FP64 except the W-cycle):
//   g = V^T A d            (SpMV reading only the diagonal-component rows)
//   zh = MG(g)             (Algorithm 3; one host read per W-cycle)
//   q = A (d - V zh), d.q  (SpMV with the embed in its operand gather)
//   x += a d, r -= a q, r.r, r.q     (a from device scalars)
//   d = r -+ b d, d.r       (b from device scalars)
// and one host read of ||r|| for the stopping test.
#include "common.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

namespace dcg {
namespace {

enum Rule { R_CG = 0, R_FCG1 = 1, R_FR = 2, R_FCGINF = 3, R_GMRES = 4 };

// x += a d; r -= a q; reduces (r.r, r.q) into (S_RRN, S_RQ);
// a = (FCG ? d.r : r.r) / d.q, zero when d.q <= 0 (breakdown: the host stops).
// V2: all four vectors 16-byte aligned; a thread takes element pairs
// (16-byte accesses, two independent partial sums per value), and the last
// element of an odd n is done by thread 0 of CTA 0.
template <bool V2>
__global__ void k_update(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ d,
                         const double* __restrict__ q, long long n, const double* __restrict__ sc, int use_dr,
                         Reduce red) {
  // one FP64 division per CTA, not per thread (a division is a sequence of
  // FP64 operations, as costly here as a thread's share of the update)
  __shared__ double s_a;
  if (threadIdx.x == 0) {
    const double dq = sc[S_DQ];
    const double num = use_dr ? sc[S_DR] : sc[S_RR];
    s_a = (dq > 0.0) ? num / dq : 0.0;
  }
  __syncthreads();
  const double a = s_a;
  double part[2] = {0.0, 0.0};
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  long long i0 = tid;
  if (V2) {
    double p0b = 0.0, p1b = 0.0;
    const long long n2 = n >> 1;
    for (long long i = tid; i < n2; i += stride) {
      const double2 di = reinterpret_cast<const double2*>(d)[i], qi = reinterpret_cast<const double2*>(q)[i];
      double2 xi = reinterpret_cast<double2*>(x)[i], ri = reinterpret_cast<double2*>(r)[i];
      xi.x = fma(a, di.x, xi.x);
      xi.y = fma(a, di.y, xi.y);
      ri.x = fma(-a, qi.x, ri.x);
      ri.y = fma(-a, qi.y, ri.y);
      reinterpret_cast<double2*>(x)[i] = xi;
      reinterpret_cast<double2*>(r)[i] = ri;
      part[0] = fma(ri.x, ri.x, part[0]);
      p0b = fma(ri.y, ri.y, p0b);
      part[1] = fma(ri.x, qi.x, part[1]);
      p1b = fma(ri.y, qi.y, p1b);
    }
    part[0] += p0b;
    part[1] += p1b;
    i0 = (n & 1) && tid == 0 ? n - 1 : n;  // the odd tail, if any
  }
  for (long long i = i0; i < n; i += (V2 ? n : stride)) {
    const double di = d[i], qi = q[i];
    x[i] = fma(a, di, x[i]);
    const double ri = fma(-a, qi, r[i]);
    r[i] = ri;
    part[0] = fma(ri, ri, part[0]);
    part[1] = fma(ri, qi, part[1]);
  }
  grid_reduce<2>(part, red);
  if (blockIdx.x == 0 && threadIdx.x == 0) ((double*)sc)[S_ALPHA] = a;
}

// FR:   d = r + (rr_new / rr) d
// FCG1: d = r - (rq / dq) d
// then d.r -> S_DR and S_RR <- rr_new
// stop (device flag, may be null): the loop of a captured solve has ended and
// the next direction is not needed (uniform early exit of every CTA)
// V2 as in k_update
template <bool V2>
__global__ void k_direction(double* __restrict__ d, const double* __restrict__ r, long long n, double* __restrict__ sc,
                            int fcg, Reduce red, const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ double s_beta;
  if (threadIdx.x == 0) {
    const double rrn = sc[S_RRN];  // r.r of the new residual (written by k_update)
    s_beta = fcg ? -(sc[S_RQ] / sc[S_DQ]) : rrn / sc[S_RR];
  }
  __syncthreads();
  const double beta = s_beta;
  double part[1] = {0.0};
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  long long i0 = tid;
  if (V2) {
    double pb = 0.0;
    const long long n2 = n >> 1;
    for (long long i = tid; i < n2; i += stride) {
      const double2 ri = reinterpret_cast<const double2*>(r)[i];
      double2 di = reinterpret_cast<double2*>(d)[i];
      di.x = fma(beta, di.x, ri.x);
      di.y = fma(beta, di.y, ri.y);
      reinterpret_cast<double2*>(d)[i] = di;
      part[0] = fma(di.x, ri.x, part[0]);
      pb = fma(di.y, ri.y, pb);
    }
    part[0] += pb;
    i0 = (n & 1) && tid == 0 ? n - 1 : n;
  }
  for (long long i = i0; i < n; i += (V2 ? n : stride)) {
    const double ri = r[i];
    const double di = fma(beta, d[i], ri);
    d[i] = di;
    part[0] = fma(di, ri, part[0]);
  }
  grid_reduce<1>(part, red);  // -> S_DR
  if (blockIdx.x == 0 && threadIdx.x == 0) sc[S_BETA] = beta;
}

// after k_direction has read both: S_RR <- S_RRN
__global__ void k_roll(double* sc, const int* __restrict__ stop) {
  if (stop && *stop) return;
  sc[S_RR] = sc[S_RRN];
}

// FCG with the truncation-restart rule of the remark after Table 4: the
// direction d_i (i = number of directions stored so far, ndir[0]) is
// orthogonalised against the m_i = max{1, mod(i, m_max + 1)} most recent
// ones, d_{i-m_i} .. d_{i-1}, kept in a ring of m_max slots (direction k in
// slot k mod m_max). m_max at least the iteration count is Algorithm 1's
// untruncated FCG(inf); m_max = 0 would be FCG(1), which has its own kernels.
__device__ __forceinline__ int fcg_window(int i, int cap) {
  const int mi = max(1, i % (cap + 1));
  return min(mi, i);
}

// slot of d_i: d, q and (d, q) copied into the ring; ndir[0] += 1
__global__ void k_store_dir(const double* __restrict__ d, const double* __restrict__ q, double* __restrict__ dirs,
                            double* __restrict__ qdirs, const int* __restrict__ ndir, int cap, long long n) {
  const int slot = ndir[0] % cap;
  double* ds = dirs + (size_t)slot * n;
  double* qs = qdirs + (size_t)slot * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    ds[i] = d[i];
    qs[i] = q[i];
  }
}
__global__ void k_store_dq(double* __restrict__ dqs, const double* __restrict__ sc, int* __restrict__ ndir, int cap) {
  dqs[ndir[0] % cap] = sc[S_DQ];
  ndir[0] += 1;
}

// c_j = (r, q_{first + j}) for the window of d_i: one pass over r per group
// of kMultiDot directions (blockIdx.y); per-CTA partial sums go to
// part[j * gridDim.x + blockIdx.x] and k_multi_dot_finish adds them in block
// order (deterministic).
constexpr int kMultiDot = 8;
constexpr int kMultiDotGrid = 2 * 152;  // CTAs along the vector (partials per direction)
__global__ void __launch_bounds__(kRedThreads) k_multi_dot(const double* __restrict__ r, const double* __restrict__ qdirs,
                                                            const int* __restrict__ ndir, int cap, long long n,
                                                            double* __restrict__ part, const int* __restrict__ stop) {
  __shared__ double smem[32 * kMultiDot];
  if (stop && *stop) return;
  const int i = ndir[0];
  const int K = fcg_window(i, cap), first = i - K;
  const int j0 = blockIdx.y * kMultiDot;
  if (j0 >= K) return;  // uniform per CTA
  const double* qk[kMultiDot];
#pragma unroll
  for (int j = 0; j < kMultiDot; ++j) qk[j] = qdirs + (size_t)((first + min(j0 + j, K - 1)) % cap) * n;
  double acc[kMultiDot];
#pragma unroll
  for (int j = 0; j < kMultiDot; ++j) acc[j] = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const double rt = r[t];
#pragma unroll
    for (int j = 0; j < kMultiDot; ++j) acc[j] = fma(rt, __ldg(qk[j] + t), acc[j]);
  }
  block_sum<kMultiDot>(acc, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < kMultiDot; ++j)
      if (j0 + j < K) part[(size_t)(j0 + j) * gridDim.x + blockIdx.x] = acc[j];
  }
}

// coef[j] = (sum over CTAs of part[j][.]) / (d_k, q_k), k = first + j: the
// coefficient of d_k in the orthogonalisation (one CTA per window entry, so
// one division per coefficient)
__global__ void k_multi_dot_finish(const double* __restrict__ part, int nbx, const int* __restrict__ ndir, int cap,
                                   const double* __restrict__ dqs, double* __restrict__ coef,
                                   const int* __restrict__ stop) {
  __shared__ double smem[32];
  if (stop && *stop) return;
  const int K = fcg_window(ndir[0], cap);
  const int j = blockIdx.x;
  if (j >= K) return;
  double v[1] = {0.0};
  for (int b = threadIdx.x; b < nbx; b += blockDim.x) v[0] += part[(size_t)j * nbx + b];
  block_sum<1>(v, smem);
  if (threadIdx.x == 0) coef[j] = v[0] / dqs[(ndir[0] - K + j) % cap];
}

// d_i = r - sum_j coef_j d_{first+j} (coef_j = c_j / dq_{first+j}); (d_i, r) -> red
__global__ void k_orth_direction(double* __restrict__ d, const double* __restrict__ r, const double* __restrict__ dirs,
                                 const double* __restrict__ coef,
                                 const int* __restrict__ ndir, int cap, long long n, Reduce red,
                                 const int* __restrict__ stop) {
  if (stop && *stop) return;
  const int i = ndir[0];
  const int K = fcg_window(i, cap), first = i - K;
  double part[1] = {0.0};
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const double rt = r[t];
    double dt = rt;
    for (int j = 0; j < K; ++j) {
      const int sl = (first + j) % cap;
      dt = fma(-coef[j], dirs[(size_t)sl * n + t], dt);
    }
    d[t] = dt;
    part[0] = fma(dt, rt, part[0]);
  }
  grid_reduce<1>(part, red);
}

// GMRES (the outer solver of the remarks in Sections 4.3 and 5.1): Arnoldi
// with classical Gram-Schmidt applied twice against the basis V (K
// contiguous vectors of n). h[i] = (V_i, w) per group of kMultiDot vectors
// (blockIdx.y), per-CTA partial sums finished in block order.
__global__ void __launch_bounds__(kRedThreads) k_gs_dots(const double* __restrict__ w, const double* __restrict__ V,
                                                          int K, long long n, double* __restrict__ part) {
  __shared__ double smem[32 * kMultiDot];
  const int j0 = blockIdx.y * kMultiDot;
  const double* vj[kMultiDot];
#pragma unroll
  for (int j = 0; j < kMultiDot; ++j) vj[j] = V + (size_t)min(j0 + j, K - 1) * n;
  double acc[kMultiDot];
#pragma unroll
  for (int j = 0; j < kMultiDot; ++j) acc[j] = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const double wt = w[t];
#pragma unroll
    for (int j = 0; j < kMultiDot; ++j) acc[j] = fma(wt, __ldg(vj[j] + t), acc[j]);
  }
  block_sum<kMultiDot>(acc, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < kMultiDot; ++j)
      if (j0 + j < K) part[(size_t)(j0 + j) * gridDim.x + blockIdx.x] = acc[j];
  }
}

__global__ void k_gs_finish(const double* __restrict__ part, int nbx, double* __restrict__ h) {
  __shared__ double smem[32];
  double v[1] = {0.0};
  for (int b = threadIdx.x; b < nbx; b += blockDim.x) v[0] += part[(size_t)blockIdx.x * nbx + b];
  block_sum<1>(v, smem);
  if (threadIdx.x == 0) h[blockIdx.x] = v[0];
}

// w -= sum_i h_i V_i, and ||w||^2 -> red
__global__ void k_gs_update(double* __restrict__ w, const double* __restrict__ V, const double* __restrict__ h, int K,
                            long long n, Reduce red) {
  double part[1] = {0.0};
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double wt = w[t];
    for (int i = 0; i < K; ++i) wt = fma(-h[i], V[(size_t)i * n + t], wt);
    w[t] = wt;
    part[0] = fma(wt, wt, part[0]);
  }
  grid_reduce<1>(part, red);
}

__global__ void k_scale_to(double* __restrict__ y, const double* __restrict__ x, double a, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

// x += sum_i y_i V_i
__global__ void k_multi_axpy(double* __restrict__ x, const double* __restrict__ V, const double* __restrict__ y, int K,
                             long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double v = x[t];
    for (int i = 0; i < K; ++i) v = fma(y[i], V[(size_t)i * n + t], v);
    x[t] = v;
  }
}

// x = xh - V (z1 - zf) (Eq. x_defl with pi(A xh) = V z1, pi(f) = V zf)
template <int D>
__global__ void k_reconstruct(const double* __restrict__ xh, const double* __restrict__ z1, const double* __restrict__ zf,
                              double* __restrict__ x, long long nn, double isd) {
  constexpr int B = D * D;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn * B; t += (long long)gridDim.x * blockDim.x) {
    const long long a = t / B;
    const int c = (int)(t % B);
    double v = xh[t];
    if (c % (D + 1) == 0) v = v - isd * z1[a] + isd * zf[a];
    x[t] = v;
  }
}

__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += x[i];
}

__global__ void k_sub(double* __restrict__ y, const double* __restrict__ x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] -= x[i];
}

__global__ void k_set_slot(double* sc, int dst, int src) { sc[dst] = sc[src]; }

struct Ctx {
  dcg_problem* p;
  cudaStream_t s;
  dcg_stats* st;
  double tol, eps, fnorm;
  int max_it;
  int rule;
};

int grid_n(long long n) { return grid_for(n, kRedThreads, 1184); }

double inner_tol(const Ctx& c, double rnorm) {
  const dcg_options& o = c.p->opts;
  if (o.inner_rule == DCG_INNER_ADAPTIVE) return o.c * c.eps / rnorm;
  return o.c * c.tol;
}

// zh = MG(V^T A x) into `z` (zeroed first), counting cycles
// z = MG(g) from zero (Algorithm 3 on the inner system), counting cycles
int inner_solve(Ctx& c, double* z, double tc, bool in_iter) {
  dcg_problem* p = c.p;
  SolverBuffers& b = p->sb;
  DCG_TRY(vec_zero(z, p->n_nodes, c.s));
  int n = 0;
  DCG_TRY(mg_solve(p, b.g, z, tc, p->opts.inner_nmax, &n, c.s));
  c.st->total_mg_cycles += n;
  if (in_iter) c.st->iter_mg_cycles += n;
  return DCG_OK;
}

int pi_of_Ax(Ctx& c, const double* x, double* z, double tc, bool in_iter) {
  dcg_problem* p = c.p;
  SolverBuffers& b = p->sb;
  DCG_TRY(spmv_vt(p, x, b.g, S_GG, c.s, in_iter && mf_lowp(p)));
  DCG_TRY(vec_zero(z, p->n_nodes, c.s));
  int n = 0;
  DCG_TRY(mg_solve(p, b.g, z, tc, p->opts.inner_nmax, &n, c.s));
  c.st->total_mg_cycles += n;
  if (in_iter) c.st->iter_mg_cycles += n;
  return DCG_OK;
}

// One pass of Algorithm 2 from x0 (or zero). *stalled is set when the pass
// ended because its recursive residual stopped falling (no value below 0.99 x
// the best one for max(stall_window, its/4) iterations): the recursion of an
// inexactly projected operator can lose orthogonality at large dt, and the
// caller then restarts from the true residual of the reconstructed iterate.
int fdcg_pass(Ctx& c, const double* f, double* x, bool use_x0, bool* converged, bool* stalled) {
  dcg_problem* p = c.p;
  SolverBuffers& b = p->sb;
  cudaStream_t s = c.s;
  const long long N = p->N;
  const double tc0 = p->opts.c * c.tol;
  *converged = false;
  // pi(f): zf = MG(V^T f)
  DCG_TRY(vec_extract(p, f, b.g, S_GG, s));
  DCG_TRY(vec_zero(b.zf, p->n_nodes, s));
  {
    int n = 0;
    DCG_TRY(mg_solve(p, b.g, b.zf, tc0, p->opts.inner_nmax, &n, s));
    c.st->total_mg_cycles += n;
  }
  // r = f_D = f - A V zf
  DCG_TRY(spmv_f_minus_avz(p, f, b.zf, b.r, S_RR, s));
  if (use_x0) {
    DCG_TRY(vec_copy(b.xh, x, N, s));
    // r -= M_D x0 = A (x0 - pi(A x0))
    DCG_TRY(pi_of_Ax(c, b.xh, b.zh, tc0, false));
    DCG_TRY(spmv_defl(p, b.xh, b.zh, b.q, S_TMP0, s));
    k_sub<<<grid_n(N), kRedThreads, 0, s>>>(b.r, b.q, N);
    DCG_LAUNCH_CHECK();
    DCG_TRY(vec_dot(p, b.r, b.r, N, S_RR, s));
  } else {
    DCG_TRY(vec_zero(b.xh, N, s));
  }
  DCG_TRY(vec_copy(b.d, b.r, N, s));
  k_set_slot<<<1, 1, 0, s>>>(p->scal, S_DR, S_RR);
  DCG_LAUNCH_CHECK();
  DCG_TRY(read_scalars(p, s));
  double rr = p->scal_host[S_RR];
  if (std::sqrt(rr) <= c.eps) *converged = true;
  const bool fcginf = c.rule == R_FCGINF;
  int ndir = 0;
  if (fcginf) DCG_CUDA(cudaMemsetAsync(b.ndir_dev, 0, sizeof(int), s));
  *stalled = false;
  const int window = p->opts.stall_window;
  double best = std::sqrt(rr);
  int its = 0, its_best = 0;
  while (!*converged && c.st->outer_its < c.max_it) {
    const double rnorm = std::sqrt(rr);
    const double tc = inner_tol(c, rnorm);
    // q = M_D d = A (d - V MG(V^T A d))
    if (b.w) {
      // assembled A: one pass over the matrix gives t = A d (kept in w) and
      // g = V^T t; then q = t - A V zh = t - K_div V zh by stencil, since the
      // mass part of A annihilates V (saves the second product)
      DCG_TRY(spmv_y_vt(p, b.d, b.w, b.g, S_GG, s));
      DCG_TRY(inner_solve(c, b.zh, tc, true));
      DCG_TRY(q_from_t(p, b.w, b.zh, b.d, b.q, S_DQ, s));
    } else {
      DCG_TRY(pi_of_Ax(c, b.d, b.zh, tc, true));
      DCG_TRY(spmv_defl(p, b.d, b.zh, b.q, S_DQ, s, mf_lowp(p)));
    }
    if (fcginf) {
      // d_{i-1}, q_{i-1} and their product into the ring before the update
      DCG_TRY(solver_fcg_store(p, s));
      ++ndir;
    }
    DCG_TRY(solver_update(p, b.xh, b.r, b.d, b.q, c.rule != R_FR, s));
    c.st->outer_its++;
    DCG_TRY(read_scalars(p, s));
    const double dq = p->scal_host[S_DQ];
    const double rrn = p->scal_host[S_RRN];
    if (!(dq > 0.0) || !std::isfinite(dq) || !std::isfinite(rrn)) {
      // FP32 matrix-free products: (d, M_D d) reaches the single-precision
      // noise floor once the residual has fallen far enough; the update was
      // skipped (alpha = 0) and the pass ends like a stall, restarting from
      // the FP64 true residual
      if (mf_lowp(p) && std::isfinite(dq) && std::isfinite(rrn)) {
        *stalled = true;
        break;
      }
      c.st->status = DCG_ERR_BREAKDOWN;
      break;
    }
    if (std::sqrt(rrn) <= c.eps) {
      *converged = true;
      break;
    }
    ++its;
    if (std::sqrt(rrn) < 0.99 * best) {
      best = std::sqrt(rrn);
      its_best = its;
    } else if (window > 0 && its - its_best > std::max(window, its / 4)) {
      *stalled = true;
      break;
    }
    if (fcginf) {
      // window of the truncation-restart rule (host mirror of ndir, for the
      // launch shape and the statistics only)
      const int mi = std::max(1, ndir % (b.ndir_cap + 1));
      const int K = std::min(mi, ndir);
      if (K < ndir) c.st->fcg_truncated++;
      DCG_TRY(solver_fcg_direction(p, s, nullptr, K, K));
    } else {
      DCG_TRY(solver_direction(p, b.d, b.r, c.rule == R_FCG1, s, nullptr));
    }
    rr = rrn;
  }
  // reconstruction x = xh - pi(A xh) + pi(f)
  DCG_TRY(pi_of_Ax(c, b.xh, b.zh, tc0, false));
  const int g = grid_n(N);
  (void)g;
  return solver_reconstruct(p, b.xh, b.zh, b.zf, x, s);
}

// q = M_D v = A (v - pi(A v)) with the inner tolerance tc, into b.q (the
// assembled operator: t = A v with g = V^T t, q = t - K_div V zh)
int apply_md(Ctx& c, const double* v, double tc, bool in_iter) {
  dcg_problem* p = c.p;
  SolverBuffers& b = p->sb;
  if (b.w) {
    DCG_TRY(spmv_y_vt(p, v, b.w, b.g, S_GG, c.s));
    DCG_TRY(inner_solve(c, b.zh, tc, in_iter));
    DCG_TRY(q_from_t(p, b.w, b.zh, v, b.q, S_DQ, c.s));
  } else {
    DCG_TRY(pi_of_Ax(c, v, b.zh, tc, in_iter));
    DCG_TRY(spmv_defl(p, v, b.zh, b.q, S_DQ, c.s, in_iter && mf_lowp(p)));
  }
  return DCG_OK;
}

// One pass of GMRES on the deflated system (restart length m = ndir_cap):
// Arnoldi on the vectors M_D(v_j, tau_c) returns, classical Gram-Schmidt
// twice, Givens rotations on the host give the residual norm after every
// step (the stopping test, and ||r_j|| of Eq. tol); a restart begins from
// the recursive residual f_D - M_D x_hat. Then the reconstruction of
// Eq. x_defl, as in the FCG pass.
int gmres_pass(Ctx& c, const double* f, double* x, bool use_x0, bool* converged) {
  dcg_problem* p = c.p;
  SolverBuffers& b = p->sb;
  cudaStream_t s = c.s;
  const long long N = p->N;
  const double tc0 = p->opts.c * c.tol;
  const int m = b.ndir_cap;
  double* V = b.dirs;  // (m + 1) vectors of N
  *converged = false;
  DCG_TRY(vec_extract(p, f, b.g, S_GG, s));
  DCG_TRY(vec_zero(b.zf, p->n_nodes, s));
  {
    int n = 0;
    DCG_TRY(mg_solve(p, b.g, b.zf, tc0, p->opts.inner_nmax, &n, s));
    c.st->total_mg_cycles += n;
  }
  DCG_TRY(spmv_f_minus_avz(p, f, b.zf, b.r, S_RR, s));
  if (use_x0) {
    DCG_TRY(vec_copy(b.xh, x, N, s));
    DCG_TRY(apply_md(c, b.xh, tc0, false));
    k_sub<<<grid_n(N), kRedThreads, 0, s>>>(b.r, b.q, N);
    DCG_LAUNCH_CHECK();
    DCG_TRY(vec_dot(p, b.r, b.r, N, S_RR, s));
  } else {
    DCG_TRY(vec_zero(b.xh, N, s));
  }
  std::vector<double> h1(m + 1), h2(m + 1), cs(m), sn(m), g(m + 1), y(m);
  std::vector<std::vector<double>> R(m);
  while (!*converged && c.st->outer_its < c.max_it) {
    DCG_TRY(read_scalars(p, s));
    const double beta = std::sqrt(p->scal_host[S_RR]);
    if (!std::isfinite(beta)) {
      c.st->status = DCG_ERR_BREAKDOWN;
      break;
    }
    if (beta <= c.eps) {
      *converged = true;
      break;
    }
    k_scale_to<<<grid_n(N), kRedThreads, 0, s>>>(V, b.r, 1.0 / beta, N);
    DCG_LAUNCH_CHECK();
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    bool lucky = false;
    while (j < m && c.st->outer_its < c.max_it) {
      DCG_TRY(apply_md(c, V + (size_t)j * N, inner_tol(c, std::fabs(g[j])), true));
      const int K = j + 1;
      const dim3 grid(kMultiDotGrid, (K + kMultiDot - 1) / kMultiDot);
      const int prof = prof_begin(p, PC_VEC, s);
      for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
        double* hd = pass == 0 ? b.dqs : b.coef;
        k_gs_dots<<<grid, kRedThreads, 0, s>>>(b.q, V, K, N, b.part);
        DCG_LAUNCH_CHECK();
        k_gs_finish<<<K, kRedThreads, 0, s>>>(b.part, kMultiDotGrid, hd);
        DCG_LAUNCH_CHECK();
        k_gs_update<<<grid_n(N), kRedThreads, 0, s>>>(b.q, V, hd, K, N, make_reduce(p, S_TMP0));
        DCG_LAUNCH_CHECK();
      }
      prof_end(p, prof, s, 8.0 * K * N, 8.0 * N * (4.0 * K + 4.0));
      DCG_CUDA(cudaMemcpyAsync(h1.data(), b.dqs, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
      DCG_CUDA(cudaMemcpyAsync(h2.data(), b.coef, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
      DCG_TRY(read_scalars(p, s));
      std::vector<double> col(K + 1);
      for (int i = 0; i < K; ++i) col[i] = h1[i] + h2[i];
      const double hn = std::sqrt(p->scal_host[S_TMP0]);
      col[K] = hn;
      for (int i = 0; i < j; ++i) {  // earlier rotations on the new column
        const double a = col[i], bb = col[i + 1];
        col[i] = cs[i] * a + sn[i] * bb;
        col[i + 1] = -sn[i] * a + cs[i] * bb;
      }
      const double den = std::hypot(col[j], col[j + 1]);
      if (!(den > 0.0) || !std::isfinite(den)) {
        c.st->status = DCG_ERR_BREAKDOWN;
        break;
      }
      cs[j] = col[j] / den;
      sn[j] = col[j + 1] / den;
      col[j] = den;
      col.resize(K);
      R[j] = col;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      c.st->outer_its++;
      if (hn > 0.0) {
        k_scale_to<<<grid_n(N), kRedThreads, 0, s>>>(V + (size_t)K * N, b.q, 1.0 / hn, N);
        DCG_LAUNCH_CHECK();
      } else {
        lucky = true;
      }
      ++j;
      if (std::fabs(g[j]) <= c.eps || lucky) {
        *converged = true;
        break;
      }
    }
    if (j > 0) {
      for (int i = j - 1; i >= 0; --i) {  // R y = g by back substitution
        double v = g[i];
        for (int k = i + 1; k < j; ++k) v -= R[k][i] * y[k];
        y[i] = v / R[i][i];
      }
      DCG_CUDA(cudaMemcpyAsync(b.coef, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, s));
      k_multi_axpy<<<grid_n(N), kRedThreads, 0, s>>>(b.xh, V, b.coef, j, N);
      DCG_LAUNCH_CHECK();
      DCG_CUDA(cudaStreamSynchronize(s));  // y is a host array
    }
    if (*converged || c.st->status != DCG_OK) break;
    // restart: r = f_D - M_D x_hat
    DCG_TRY(apply_md(c, b.xh, tc0, false));
    DCG_TRY(spmv_f_minus_avz(p, f, b.zf, b.r, S_RR, s));
    k_sub<<<grid_n(N), kRedThreads, 0, s>>>(b.r, b.q, N);
    DCG_LAUNCH_CHECK();
    DCG_TRY(vec_dot(p, b.r, b.r, N, S_RR, s));
  }
  DCG_TRY(pi_of_Ax(c, b.xh, b.zh, tc0, false));
  return solver_reconstruct(p, b.xh, b.zh, b.zf, x, s);
}

int plain_cg(Ctx& c, const double* f, double* x) {
  dcg_problem* p = c.p;
  SolverBuffers& b = p->sb;
  cudaStream_t s = c.s;
  const long long N = p->N;
  DCG_TRY(spmv_residual(p, f, x, b.r, S_RR, s));
  DCG_TRY(vec_copy(b.d, b.r, N, s));
  DCG_TRY(read_scalars(p, s));
  double rr = p->scal_host[S_RR];
  bool conv = std::sqrt(rr) <= c.eps;
  while (!conv && c.st->outer_its < c.max_it) {
    DCG_TRY(spmv_dot(p, b.d, b.q, b.d, S_DQ, s));
    DCG_TRY(solver_update(p, x, b.r, b.d, b.q, 0, s));
    c.st->outer_its++;
    bool check = (c.st->outer_its % std::max(1, p->opts.check_every)) == 0;
    if (check) {
      DCG_TRY(read_scalars(p, s));
      const double dq = p->scal_host[S_DQ];
      const double rrn = p->scal_host[S_RRN];
      if (!(dq > 0.0) || !std::isfinite(rrn)) {
        c.st->status = DCG_ERR_BREAKDOWN;
        break;
      }
      if (std::sqrt(rrn) <= c.eps) {
        conv = true;
        break;
      }
    }
    DCG_TRY(solver_direction(p, b.d, b.r, 0, s, nullptr));
  }
  return DCG_OK;
}

}  // namespace

// Launch wrappers shared by the host-driven loop below and the captured
// solve of graph.cu.
int solver_update(dcg_problem* p, double* x, double* r, const double* d, const double* q, int use_dr,
                  cudaStream_t s) {
  const long long N = p->N;
  const int prof = prof_begin(p, PC_VEC, s);
  if (aligned16(x) && aligned16(r) && aligned16(d) && aligned16(q))
    k_update<true><<<grid_n(N), kRedThreads, 0, s>>>(x, r, d, q, N, p->scal, use_dr, make_reduce(p, S_RRN));
  else
    k_update<false><<<grid_n(N), kRedThreads, 0, s>>>(x, r, d, q, N, p->scal, use_dr, make_reduce(p, S_RRN));
  DCG_LAUNCH_CHECK();
  prof_end(p, prof, s, 8.0 * N, 48.0 * N);
  return DCG_OK;
}

int solver_direction(dcg_problem* p, double* d, const double* r, int fcg, cudaStream_t s, const int* stop) {
  const long long N = p->N;
  const int prof = prof_begin(p, PC_VEC, s);
  if (aligned16(d) && aligned16(r))
    k_direction<true><<<grid_n(N), kRedThreads, 0, s>>>(d, r, N, p->scal, fcg, make_reduce(p, S_DR), stop);
  else
    k_direction<false><<<grid_n(N), kRedThreads, 0, s>>>(d, r, N, p->scal, fcg, make_reduce(p, S_DR), stop);
  DCG_LAUNCH_CHECK();
  prof_end(p, prof, s, 4.0 * N, 24.0 * N);
  k_roll<<<1, 1, 0, s>>>(p->scal, stop);
  DCG_LAUNCH_CHECK();
  return DCG_OK;
}

int solver_fcg_store(dcg_problem* p, cudaStream_t s) {
  SolverBuffers& b = p->sb;
  const long long N = p->N;
  const int prof = prof_begin(p, PC_VEC, s);
  k_store_dir<<<grid_n(N), kRedThreads, 0, s>>>(b.d, b.q, b.dirs, b.qdirs, b.ndir_dev, b.ndir_cap, N);
  DCG_LAUNCH_CHECK();
  k_store_dq<<<1, 1, 0, s>>>(b.dqs, p->scal, b.ndir_dev, b.ndir_cap);
  DCG_LAUNCH_CHECK();
  prof_end(p, prof, s, 0.0, 32.0 * N);
  return DCG_OK;
}

// K: launch shape for the window (the kernels read the actual window from the
// device counter and skip entries beyond it; a captured solve passes the ring
// size)
int solver_fcg_direction(dcg_problem* p, cudaStream_t s, const int* stop, int K, int finish_grid) {
  SolverBuffers& b = p->sb;
  const long long N = p->N;
  const int gy = (K + kMultiDot - 1) / kMultiDot;
  const int prof = prof_begin(p, PC_VEC, s);
  k_multi_dot<<<dim3(kMultiDotGrid, gy), kRedThreads, 0, s>>>(b.r, b.qdirs, b.ndir_dev, b.ndir_cap, N, b.part, stop);
  DCG_LAUNCH_CHECK();
  k_multi_dot_finish<<<finish_grid, kRedThreads, 0, s>>>(b.part, kMultiDotGrid, b.ndir_dev, b.ndir_cap, b.dqs, b.coef,
                                                         stop);
  DCG_LAUNCH_CHECK();
  k_orth_direction<<<grid_n(N), kRedThreads, 0, s>>>(b.d, b.r, b.dirs, b.coef, b.ndir_dev, b.ndir_cap, N,
                                                      make_reduce(p, S_DR), stop);
  DCG_LAUNCH_CHECK();
  prof_end(p, prof, s, 4.0 * K * N, 8.0 * N * (2.0 * K + 2.0 + (double)gy));
  k_roll<<<1, 1, 0, s>>>(p->scal, stop);
  DCG_LAUNCH_CHECK();
  return DCG_OK;
}

int solver_reconstruct(dcg_problem* p, const double* xh, const double* z1, const double* zf, double* x,
                       cudaStream_t s) {
  const int g = grid_n(p->N);
  const double isd = 1.0 / std::sqrt((double)p->dim);
  if (p->dim == 2) k_reconstruct<2><<<g, kRedThreads, 0, s>>>(xh, z1, zf, x, p->n_nodes, isd);
  else k_reconstruct<3><<<g, kRedThreads, 0, s>>>(xh, z1, zf, x, p->n_nodes, isd);
  DCG_LAUNCH_CHECK();
  return DCG_OK;
}

int solver_axpy(dcg_problem* p, double* y, const double* x, cudaStream_t s) {
  k_axpy<<<grid_n(p->N), kRedThreads, 0, s>>>(y, x, p->N);
  DCG_LAUNCH_CHECK();
  return DCG_OK;
}

int read_scalars(dcg_problem* p, cudaStream_t s) {
  DCG_CUDA(cudaMemcpyAsync(p->scal_host, p->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, s));
  DCG_CUDA(cudaStreamSynchronize(s));
  if (p->prof.mask) prof_flush(p);
  if (p->scal_host[S_ERR] != 0.0) {
    set_error_msg("a bounded device wait gave up (bulk copy did not complete)");
    return DCG_ERR_CUDA;
  }
  return DCG_OK;
}

int solve_device(dcg_problem* p, const double* f, double* x, double tol, int max_it, dcg_stats* st,
                 cudaStream_t s) {
  if (graph_solve_supported(p)) return graph_solve(p, f, x, tol, max_it, st, s);
  auto t0 = std::chrono::steady_clock::now();
  *st = dcg_stats{};
  st->status = DCG_OK;
  Ctx c{p, s, st, tol, 0.0, 0.0, max_it, R_CG};
  const dcg_options& o = p->opts;
  if (o.deflate) {
    c.rule = o.recurrence == DCG_FR ? R_FR
             : o.recurrence == DCG_FCG_INF ? R_FCGINF
             : o.recurrence == DCG_GMRES ? R_GMRES
                                          : R_FCG1;
  }
  const long long N = p->N;
  SolverBuffers& b = p->sb;
  DCG_TRY(vec_dot(p, f, f, N, S_FF, s));
  DCG_TRY(vec_dot(p, x, x, N, S_TMP1, s));
  DCG_TRY(read_scalars(p, s));
  c.fnorm = std::sqrt(p->scal_host[S_FF]);
  const bool x0_nonzero = p->scal_host[S_TMP1] != 0.0;
  if (!std::isfinite(c.fnorm) || !std::isfinite(p->scal_host[S_TMP1])) {
    // a NaN or infinite entry in f or x0: no iteration can be formed
    DCG_CUDA(cudaStreamSynchronize(s));
    st->status = DCG_ERR_BREAKDOWN;
    st->true_relres = std::nan("");
    set_error_msg("dcg_solve: non-finite entries in the right-hand side or the initial guess");
    return st->status;
  }
  if (!(c.fnorm > 0.0)) {
    DCG_TRY(vec_zero(x, N, s));
    DCG_CUDA(cudaStreamSynchronize(s));
    st->true_relres = 0.0;
    return DCG_OK;
  }
  c.eps = tol * c.fnorm;
  bool stalled = false;
  if (!o.deflate) {
    DCG_TRY(plain_cg(c, f, x));
  } else {
    if ((c.rule == R_FCGINF || c.rule == R_GMRES) && !b.dirs) return DCG_ERR_STATE;
    bool conv = false;
    if (c.rule == R_GMRES) DCG_TRY(gmres_pass(c, f, x, x0_nonzero, &conv));
    else DCG_TRY(fdcg_pass(c, f, x, x0_nonzero, &conv, &stalled));
  }
  // true residual
  DCG_TRY(spmv_residual(p, f, x, b.u, S_TMP0, s));
  DCG_TRY(read_scalars(p, s));
  st->true_relres = std::sqrt(p->scal_host[S_TMP0]) / c.fnorm;
  if (o.deflate) {
    int claimed = 0;  // restarts after passes that reported convergence
    while (st->true_relres > tol && (stalled || claimed < o.max_restarts) && st->status == DCG_OK &&
           st->outer_its < max_it) {
      if (!stalled) ++claimed;
      st->restarts++;
      bool conv = false;
      if (c.rule == R_GMRES) DCG_TRY(gmres_pass(c, b.u, b.e, false, &conv));
      else DCG_TRY(fdcg_pass(c, b.u, b.e, false, &conv, &stalled));
      DCG_TRY(solver_axpy(p, x, b.e, s));
      DCG_TRY(spmv_residual(p, f, x, b.u, S_TMP0, s));
      DCG_TRY(read_scalars(p, s));
      st->true_relres = std::sqrt(p->scal_host[S_TMP0]) / c.fnorm;
    }
  }
  DCG_CUDA(cudaStreamSynchronize(s));
  if (st->status == DCG_OK && !(st->true_relres <= tol)) st->status = DCG_ERR_NOT_CONVERGED;
  st->avg_inner = st->outer_its ? (double)st->iter_mg_cycles / st->outer_its : 0.0;
  st->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return st->status;
}

}  // namespace dcg
