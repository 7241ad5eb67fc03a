// C ABI of libdcg (declared in include/dcg.h): argument checks, ownership of
// device memory, and dispatch to the kernels of the other translation units.
#include "common.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

namespace dcg {

long long g_launch_count = 0;

namespace {
thread_local std::string g_err;
}

void set_error(const char* what, cudaError_t e) {
  g_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
}
void set_error_msg(const std::string& msg) { g_err = msg; }

namespace {

long long ipow_ll(long long b, int e) {
  long long r = 1;
  for (int k = 0; k < e; ++k) r *= b;
  return r;
}

int check_options(const dcg_options* o, int dim) {
  if (!o) return DCG_ERR_INVALID_ARG;
  bool ok = o->max_levels >= 1 && o->patch >= 1 && o->overlap >= 0 && 2 * o->overlap <= o->patch && o->m1 >= 0 &&
            o->m2 >= 0 && (o->inner_rule >= 0 && o->inner_rule <= 2) && o->c > 0 && o->inner_nmax >= 1 &&
            (o->recurrence >= 0 && o->recurrence <= 2) && (o->precision == DCG_FP64 || o->precision == DCG_MIXED) &&
            (o->ras_inverse == DCG_INV_FP32 || o->ras_inverse == DCG_INV_BF16) &&
            (o->ras_weights == 0 || o->ras_weights == 1) && (o->deflate == 0 || o->deflate == 1) &&
            o->max_restarts >= 0 && o->fcg_max_dirs >= 0 && o->check_every >= 1;
  if (!ok) {
    set_error_msg("invalid dcg_options field");
    return DCG_ERR_INVALID_ARG;
  }
  long long box = ipow_ll(o->patch + 2 * o->overlap, dim);
  if (box > 256) {
    set_error_msg("RAS box (patch + 2*overlap)^dim exceeds 256 nodes");
    return DCG_ERR_UNSUPPORTED;
  }
  return DCG_OK;
}

void free_solver_buffers(dcg_problem* p) {
  SolverBuffers& b = p->sb;
  double* all[] = {b.xh, b.r, b.d, b.q, b.u, b.e, b.g, b.zh, b.zf, b.rin, b.dirs, b.qdirs, b.coef};
  for (double* v : all) cudaFree(v);
  b = SolverBuffers{};
}

int alloc_vec(double** v, long long n) {
  DCG_CUDA(cudaMalloc(v, sizeof(double) * (n > 0 ? n : 1)));
  return DCG_OK;
}

}  // namespace

cudaEvent_t prof_event(dcg_problem* p) {
  Prof& P = p->prof;
  if (!P.pool.empty()) {
    cudaEvent_t e = P.pool.back();
    P.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

int prof_begin(dcg_problem* p, int cls, cudaStream_t s, bool capture) {
  Prof& P = p->prof;
  if (!(P.mask & (1u << cls))) return -1;
  ProfPair pr;
  pr.a = prof_event(p);
  pr.b = prof_event(p);
  pr.cls = cls;
  if (capture) {
    cudaEventRecordWithFlags(pr.a, s, cudaEventRecordExternal);
    P.graph.push_back(pr);
    return (int)P.graph.size() - 1;
  }
  cudaEventRecord(pr.a, s);
  P.pending.push_back(pr);
  return (int)P.pending.size() - 1;
}

void prof_end(dcg_problem* p, int idx, cudaStream_t s, double flops, double bytes, bool capture) {
  if (idx < 0) return;
  Prof& P = p->prof;
  ProfPair& pr = capture ? P.graph[idx] : P.pending[idx];
  pr.flops = flops;
  pr.bytes = bytes;
  if (capture) cudaEventRecordWithFlags(pr.b, s, cudaEventRecordExternal);
  else cudaEventRecord(pr.b, s);
}

static void prof_account(Prof& P, const ProfPair& pr) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, pr.a, pr.b) == cudaSuccess) {
    P.ms[pr.cls] += ms;
    P.flops[pr.cls] += pr.flops;
    P.bytes[pr.cls] += pr.bytes;
    P.launches[pr.cls] += 1;
  }
}

void prof_flush(dcg_problem* p) {
  Prof& P = p->prof;
  for (auto& pr : P.pending) {
    prof_account(P, pr);
    P.pool.push_back(pr.a);
    P.pool.push_back(pr.b);
  }
  P.pending.clear();
}

void prof_flush_graph(dcg_problem* p) {
  Prof& P = p->prof;
  for (auto& pr : P.graph) prof_account(P, pr);
}

void prof_clear_graph(dcg_problem* p) {
  Prof& P = p->prof;
  for (auto& pr : P.graph) {
    P.pool.push_back(pr.a);
    P.pool.push_back(pr.b);
  }
  P.graph.clear();
}

}  // namespace dcg

using namespace dcg;

extern "C" {

void dcg_default_options(dcg_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->max_levels = 4;
  o->patch = 4;
  o->overlap = 1;
  o->m1 = 2;
  o->m2 = 2;
  o->inner_rule = DCG_INNER_FIXED;
  o->c = 0.01;
  o->inner_nmax = 100;
  o->recurrence = DCG_FCG1;
  o->precision = DCG_FP64;
  o->ras_inverse = DCG_INV_FP32;
  o->ras_weights = DCG_RAS_MULTIPLICITY;
  o->deflate = 1;
  o->max_restarts = 3;
  o->fcg_max_dirs = 0;
  o->check_every = 1;
}

const char* dcg_status_string(int s) {
  switch (s) {
    case DCG_OK: return "ok";
    case DCG_ERR_INVALID_ARG: return "invalid argument";
    case DCG_ERR_NOT_CONVERGED: return "not converged";
    case DCG_ERR_BREAKDOWN: return "breakdown";
    case DCG_ERR_CUDA: return "CUDA error";
    case DCG_ERR_OOM: return "out of device memory";
    case DCG_ERR_UNSUPPORTED: return "unsupported configuration";
    case DCG_ERR_STATE: return "call order violated";
    default: return "unknown status";
  }
}

const char* dcg_last_error(void) { return g_err.c_str(); }

int dcg_assemble(const dcg_mesh* mesh, double dt, double nu, const double* nu_elem, int matrix_free,
                 dcg_problem** out, void* stream) {
  if (!mesh || !out || (mesh->dim != 2 && mesh->dim != 3) || mesh->n < 2 || !(dt > 0) || !(nu > 0) ||
      !std::isfinite(dt) || !std::isfinite(nu)) {
    set_error_msg("dcg_assemble: need dim in {2,3}, n >= 2, dt > 0, nu > 0, out != NULL");
    return DCG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (matrix_free) {
    set_error_msg("matrix-free assembly is not available in this build");
    return DCG_ERR_UNSUPPORTED;
  }
  if (nu_elem) {
    long long ne = ipow_ll(mesh->n, mesh->dim);
    for (long long e = 0; e < ne; ++e)
      if (!(nu_elem[e] > 0) || !std::isfinite(nu_elem[e])) {
        set_error_msg("dcg_assemble: per-element viscosity must be finite and > 0");
        return DCG_ERR_INVALID_ARG;
      }
  }
  cudaStream_t s = (cudaStream_t)stream;
  dcg_problem* p = new (std::nothrow) dcg_problem();
  if (!p) return DCG_ERR_OOM;
  p->dim = mesh->dim;
  p->n = mesh->n;
  p->m = mesh->n - 1;
  p->b = p->dim * p->dim;
  p->n_nodes = ipow_ll(p->m, p->dim);
  p->N = p->n_nodes * p->b;
  p->nnzb = ipow_ll(3LL * p->m - 2, p->dim);
  p->dt = dt;
  p->nu = nu;
  p->matrix_free = matrix_free;
  if (p->nnzb >= (1LL << 31) || p->n_nodes >= (1LL << 31)) {
    delete p;
    set_error_msg("dcg_assemble: mesh too large for int32 BSR indices");
    return DCG_ERR_UNSUPPORTED;
  }
  int st = DCG_OK;
  auto fail = [&](int code) {
    dcg_destroy(p);
    return code;
  };
  if (cudaMalloc(&p->partials, sizeof(double) * kMaxVals * kMaxRedCtas) != cudaSuccess ||
      cudaMalloc(&p->counters, sizeof(unsigned) * kNumCounters) != cudaSuccess ||
      cudaMalloc(&p->scal, sizeof(double) * S_COUNT) != cudaSuccess ||
      cudaMallocHost(&p->scal_host, sizeof(double) * S_COUNT) != cudaSuccess) {
    set_error_msg("dcg_assemble: allocation of reduction scratch failed");
    return fail(DCG_ERR_OOM);
  }
  if (cudaMemsetAsync(p->counters, 0, sizeof(unsigned) * kNumCounters, s) != cudaSuccess ||
      cudaMemsetAsync(p->scal, 0, sizeof(double) * S_COUNT, s) != cudaSuccess) {
    set_error_msg("dcg_assemble: memset failed");
    return fail(DCG_ERR_CUDA);
  }
  st = assemble_device(p, nu_elem, s);
  if (st != DCG_OK) return fail(st);
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    set_error("dcg_assemble", cudaGetLastError());
    return fail(DCG_ERR_CUDA);
  }
  *out = p;
  return DCG_OK;
}

int dcg_setup(dcg_problem* p, const dcg_options* opts, void* stream) {
  if (!p) return DCG_ERR_INVALID_ARG;
  DCG_TRY(check_options(opts, p->dim));
  cudaStream_t s = (cudaStream_t)stream;
  p->is_setup = false;
  free_solver_buffers(p);
  mg_free(p);
  p->opts = *opts;
  SolverBuffers& b = p->sb;
  const long long N = p->N, nn = p->n_nodes;
  DCG_TRY(alloc_vec(&b.xh, N));
  DCG_TRY(alloc_vec(&b.r, N));
  DCG_TRY(alloc_vec(&b.d, N));
  DCG_TRY(alloc_vec(&b.q, N));
  DCG_TRY(alloc_vec(&b.u, N));
  DCG_TRY(alloc_vec(&b.e, N));
  if (opts->deflate) {
    DCG_TRY(alloc_vec(&b.g, nn));
    DCG_TRY(alloc_vec(&b.zh, nn));
    DCG_TRY(alloc_vec(&b.zf, nn));
    if (opts->recurrence == DCG_FCG_INF) {
      long long cap = opts->fcg_max_dirs;
      if (cap <= 0) {
        long long budget = (8LL << 30) / (16LL * N);
        cap = budget < 256 ? budget : 256;
        if (cap < 1) cap = 1;
      }
      b.ndir_cap = (int)cap;
      DCG_TRY(alloc_vec(&b.dirs, cap * N));
      DCG_TRY(alloc_vec(&b.qdirs, cap * N));
      DCG_TRY(alloc_vec(&b.coef, 2 * cap));
    }
    DCG_TRY(mg_setup(p, s));
  }
  DCG_CUDA(cudaStreamSynchronize(s));
  p->is_setup = true;
  return DCG_OK;
}

int dcg_solve(dcg_problem* p, const double* f_dev, double* x_dev, double tol, int max_it, dcg_stats* stats,
              void* stream) {
  if (!p || !f_dev || !x_dev || !(tol > 0) || max_it < 0) {
    set_error_msg("dcg_solve: need problem, f, x, tol > 0, max_it >= 0");
    return DCG_ERR_INVALID_ARG;
  }
  if (!p->is_setup) {
    set_error_msg("dcg_solve before dcg_setup");
    return DCG_ERR_STATE;
  }
  dcg_stats local;
  dcg_stats* st = stats ? stats : &local;
  int r = solve_device(p, f_dev, x_dev, tol, max_it, st, (cudaStream_t)stream);
  if (r != DCG_OK && r != DCG_ERR_NOT_CONVERGED && r != DCG_ERR_BREAKDOWN) st->status = r;
  return r;
}

int dcg_solve_host(dcg_problem* p, const double* f_host, double* x_host, double tol, int max_it, dcg_stats* stats,
                   void* stream) {
  if (!p || !f_host || !x_host) return DCG_ERR_INVALID_ARG;
  if (!p->is_setup) return DCG_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  if (!p->fine_f64) {
    DCG_TRY(alloc_vec(&p->fine_f64, p->N));
    DCG_TRY(alloc_vec(&p->fine_x64, p->N));
  }
  DCG_CUDA(cudaMemcpyAsync(p->fine_f64, f_host, sizeof(double) * p->N, cudaMemcpyHostToDevice, s));
  DCG_CUDA(cudaMemcpyAsync(p->fine_x64, x_host, sizeof(double) * p->N, cudaMemcpyHostToDevice, s));
  int r = dcg_solve(p, p->fine_f64, p->fine_x64, tol, max_it, stats, stream);
  if (r != DCG_OK && r != DCG_ERR_NOT_CONVERGED && r != DCG_ERR_BREAKDOWN) return r;
  DCG_CUDA(cudaMemcpyAsync(x_host, p->fine_x64, sizeof(double) * p->N, cudaMemcpyDeviceToHost, s));
  DCG_CUDA(cudaStreamSynchronize(s));
  return r;
}

int dcg_solve_batched(int nprob, dcg_problem* const* probs, int nrhs, const double* const* f_dev,
                      double* const* x_dev, double tol, int max_it, dcg_stats* stats, void* stream) {
  if (nprob < 0 || nrhs < 1 || (nprob > 0 && (!probs || !f_dev || !x_dev || !stats))) return DCG_ERR_INVALID_ARG;
  int worst = DCG_OK;
  for (int pi = 0; pi < nprob; ++pi)
    for (int r = 0; r < nrhs; ++r) {
      const int k = pi * nrhs + r;
      int st = dcg_solve(probs[pi], f_dev[k], x_dev[k], tol, max_it, &stats[k], stream);
      if (st != DCG_OK && st != DCG_ERR_NOT_CONVERGED && st != DCG_ERR_BREAKDOWN) return st;
      if (st != DCG_OK && worst == DCG_OK) worst = st;
    }
  return worst;
}

void dcg_destroy(dcg_problem* p) {
  if (!p) return;
  mg_free(p);
  prof_flush(p);
  prof_clear_graph(p);
  for (cudaEvent_t e : p->prof.pool) cudaEventDestroy(e);
  free_solver_buffers(p);
  cudaFree(p->row_ptr);
  cudaFree(p->col_idx);
  cudaFree(p->vals);
  cudaFree(p->inv_nu_elem);
  cudaFree(p->partials);
  cudaFree(p->counters);
  cudaFree(p->scal);
  cudaFreeHost(p->scal_host);
  cudaFree(p->fine_f64);
  cudaFree(p->fine_x64);
  delete p;
}

int dcg_problem_info(const dcg_problem* p, long long* n_unknowns, long long* n_nodes, long long* nnzb, int* levels) {
  if (!p) return DCG_ERR_INVALID_ARG;
  if (n_unknowns) *n_unknowns = p->N;
  if (n_nodes) *n_nodes = p->n_nodes;
  if (nnzb) *nnzb = p->matrix_free ? 0 : p->nnzb;
  if (levels) *levels = (int)p->levels.size();
  return DCG_OK;
}

int dcg_export_pattern(const dcg_problem* p, int* row_ptr, int* col_idx) {
  if (!p || !row_ptr || !col_idx || p->matrix_free) return DCG_ERR_INVALID_ARG;
  DCG_CUDA(cudaMemcpy(row_ptr, p->row_ptr, sizeof(int) * (p->n_nodes + 1), cudaMemcpyDeviceToHost));
  DCG_CUDA(cudaMemcpy(col_idx, p->col_idx, sizeof(int) * p->nnzb, cudaMemcpyDeviceToHost));
  return DCG_OK;
}

int dcg_export_values(const dcg_problem* p, double* values) {
  if (!p || !values || p->matrix_free) return DCG_ERR_INVALID_ARG;
  DCG_CUDA(cudaMemcpy(values, p->vals, sizeof(double) * p->nnzb * p->b * p->b, cudaMemcpyDeviceToHost));
  return DCG_OK;
}

int dcg_spmv(const dcg_problem* p, const double* x, double* y, void* stream) {
  if (!p || !x || !y) return DCG_ERR_INVALID_ARG;
  return spmv_plain(const_cast<dcg_problem*>(p), x, y, (cudaStream_t)stream);
}

int dcg_extract(const dcg_problem* p, const double* y, double* q, void* stream) {
  if (!p || !y || !q) return DCG_ERR_INVALID_ARG;
  return vec_extract(const_cast<dcg_problem*>(p), y, q, -1, (cudaStream_t)stream);
}

int dcg_embed(const dcg_problem* p, const double* q, double* y, void* stream) {
  if (!p || !y || !q) return DCG_ERR_INVALID_ARG;
  return vec_embed(const_cast<dcg_problem*>(p), q, y, (cudaStream_t)stream);
}

int dcg_inner_apply(const dcg_problem* p, const double* z, double* y, void* stream) {
  if (!p || !z || !y) return DCG_ERR_INVALID_ARG;
  if (!p->is_setup || p->levels.empty()) return DCG_ERR_STATE;
  return mg_inner_apply(const_cast<dcg_problem*>(p), z, y, (cudaStream_t)stream);
}

int dcg_mg_cycles(dcg_problem* p, const double* g, double* z, int ncycles, void* stream) {
  if (!p || !g || !z || ncycles < 0) return DCG_ERR_INVALID_ARG;
  if (!p->is_setup || p->levels.empty()) return DCG_ERR_STATE;
  return mg_cycles(p, g, z, ncycles, (cudaStream_t)stream);
}

int dcg_mg_solve(dcg_problem* p, const double* g, double* z, double tol, int nmax, int* ncycles, void* stream) {
  if (!p || !g || !z || !ncycles || !(tol > 0) || nmax < 0) return DCG_ERR_INVALID_ARG;
  if (!p->is_setup || p->levels.empty()) return DCG_ERR_STATE;
  return mg_solve(p, g, z, tol, nmax, ncycles, (cudaStream_t)stream);
}

int dcg_ras_step(dcg_problem* p, int level, const double* f, double* z, void* stream) {
  if (!p || !f || !z) return DCG_ERR_INVALID_ARG;
  if (!p->is_setup || p->levels.empty()) return DCG_ERR_STATE;
  return mg_ras_step_hook(p, level, f, z, (cudaStream_t)stream);
}

int dcg_coarse_solve(dcg_problem* p, const double* f, double* z, void* stream) {
  if (!p || !f || !z) return DCG_ERR_INVALID_ARG;
  if (!p->is_setup || p->levels.empty()) return DCG_ERR_STATE;
  return mg_coarse_hook(p, f, z, (cudaStream_t)stream);
}

int dcg_profile_enable(dcg_problem* p, unsigned mask, void* stream) {
  if (!p) return DCG_ERR_INVALID_ARG;
  DCG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  prof_flush(p);
  Prof& P = p->prof;
  for (int c = 0; c < PC_COUNT; ++c) {
    P.ms[c] = P.flops[c] = P.bytes[c] = 0.0;
    P.launches[c] = 0;
  }
  const bool rebuild = P.mask != mask;
  P.mask = mask;
  if (rebuild && p->is_setup) return mg_rebuild_graph(p);
  return DCG_OK;
}

int dcg_profile_read(dcg_problem* p, int cls, double* ms, long long* launches, double* flops, double* bytes,
                     void* stream) {
  if (!p || cls < 0 || cls >= PC_COUNT) return DCG_ERR_INVALID_ARG;
  DCG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  prof_flush(p);
  const Prof& P = p->prof;
  if (ms) *ms = P.ms[cls];
  if (launches) *launches = P.launches[cls];
  if (flops) *flops = P.flops[cls];
  if (bytes) *bytes = P.bytes[cls];
  return DCG_OK;
}

long long dcg_kernel_launches(void) { return g_launch_count; }

}  // extern "C"
