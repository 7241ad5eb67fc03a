// C ABI of libdcg (declared in include/dcg.h): argument checks, ownership of
// device memory, and dispatch to the kernels of the other translation units.
#include "common.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <set>
#include <thread>

namespace dcg {

std::atomic<long long> g_launch_count{0};
thread_local bool t_capturing = false;
thread_local long long t_capture_launches = 0;

namespace {
thread_local std::string g_err;
constexpr int kBatchWorkers = 16;  // host workers (and streams) of dcg_solve_batched
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
            (o->recurrence >= 0 && o->recurrence <= 3) && (o->precision == DCG_FP64 || o->precision == DCG_MIXED) &&
            (o->ras_inverse == DCG_INV_FP32 || o->ras_inverse == DCG_INV_BF16) &&
            (o->ras_weights == 0 || o->ras_weights == 1) && (o->deflate == 0 || o->deflate == 1) &&
            o->max_restarts >= 0 && o->fcg_max_dirs >= 0 && o->check_every >= 1 && o->stall_window >= 0 &&
            (o->device_loop == 0 || o->device_loop == 1);
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
  double* all[] = {b.xh, b.r, b.d, b.q, b.u, b.e, b.g, b.zh, b.zf, b.rin, b.dirs, b.qdirs, b.dqs, b.coef, b.part, b.w};
  for (double* v : all) cudaFree(v);
  cudaFree(b.ndir_dev);
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
  o->stall_window = 200;
  o->device_loop = 1;
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
  if (matrix_free && (mesh->dim != 3 || mesh->n < 4)) {
    set_error_msg("dcg_assemble: the matrix-free operator is implemented for 3D meshes with n >= 4");
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
  if ((!matrix_free && p->nnzb >= (1LL << 31)) || p->n_nodes >= (1LL << 31)) {
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
  graph_free(p);
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
    if (!p->matrix_free) DCG_TRY(alloc_vec(&b.w, N));
    DCG_TRY(alloc_vec(&b.g, nn));
    DCG_TRY(alloc_vec(&b.zh, nn));
    DCG_TRY(alloc_vec(&b.zf, nn));
    if (opts->recurrence == DCG_FCG_INF || opts->recurrence == DCG_GMRES) {
      const bool gm = opts->recurrence == DCG_GMRES;
      long long cap = opts->fcg_max_dirs;
      if (cap <= 0) {
        long long budget = (8LL << 30) / (16LL * N);
        cap = budget < 256 ? budget : 256;
        if (cap < 1) cap = 1;
      }
      b.ndir_cap = (int)cap;
      // FCG: directions d_k and q_k = M_D d_k; GMRES: the Arnoldi basis
      // (m + 1 vectors)
      DCG_TRY(alloc_vec(&b.dirs, (gm ? cap + 1 : cap) * N));
      DCG_TRY(alloc_vec(&b.qdirs, gm ? 1 : cap * N));
      DCG_TRY(alloc_vec(&b.dqs, cap));
      DCG_TRY(alloc_vec(&b.coef, cap));
      DCG_TRY(alloc_vec(&b.part, cap * 2 * 152));
      DCG_CUDA(cudaMalloc(&b.ndir_dev, sizeof(int)));
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
  if (nprob < 0 || nrhs < 1 || (nprob > 0 && (!probs || !f_dev || !x_dev || !stats)) || !(tol > 0) || max_it < 0) {
    set_error_msg("dcg_solve_batched: need nprob >= 0, nrhs >= 1, arrays, tol > 0");
    return DCG_ERR_INVALID_ARG;
  }
  std::set<const dcg_problem*> seen;
  for (int i = 0; i < nprob; ++i) {
    if (!probs[i] || !probs[i]->is_setup || !seen.insert(probs[i]).second) {
      set_error_msg("dcg_solve_batched: every problem must be set up and appear once");
      return probs[i] && !probs[i]->is_setup ? DCG_ERR_STATE : DCG_ERR_INVALID_ARG;
    }
    for (int r = 0; r < nrhs; ++r)
      if (!f_dev[i * nrhs + r] || !x_dev[i * nrhs + r]) return DCG_ERR_INVALID_ARG;
  }
  if (nprob == 0) return DCG_OK;
  bool graph_ok = true;
  for (int i = 0; i < nprob; ++i)
    graph_ok = graph_ok && graph_solve_supported(probs[i]);
  if (graph_ok) {
    // one CUDA graph for the whole batch: every pair stops at its own
    // device-side convergence test, problems run as independent branches
    const int rc = graph_solve_batched(nprob, probs, nrhs, f_dev, x_dev, tol, max_it, stats, (cudaStream_t)stream);
    if (rc != DCG_OK) return rc;
    int worst = DCG_OK;
    for (int k = 0; k < nprob * nrhs; ++k)
      if (stats[k].status != DCG_OK && worst == DCG_OK) worst = stats[k].status;
    return worst;
  }
  // Problems are independent: a pool of host workers drives them on their own
  // non-blocking streams (each problem's right-hand sides in order), so the
  // GPU overlaps the latency-bound kernels of different problems. Work starts
  // after everything already queued on the caller's stream, and the caller's
  // stream waits for every worker.
  cudaStream_t caller = (cudaStream_t)stream;
  int dev = 0;
  DCG_CUDA(cudaGetDevice(&dev));
  cudaEvent_t start = nullptr;
  DCG_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  DCG_CUDA(cudaEventRecord(start, caller));
  const int nworkers = nprob < kBatchWorkers ? nprob : kBatchWorkers;
  std::atomic<int> next{0};
  std::vector<int> wstatus(nworkers, DCG_OK);
  std::vector<std::string> werr(nworkers);
  std::vector<std::thread> pool;
  for (int w = 0; w < nworkers; ++w) {
    pool.emplace_back([&, w]() {
      cudaSetDevice(dev);
      cudaStream_t ws = nullptr;
      cudaEvent_t done = nullptr;
      if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess ||
          cudaStreamWaitEvent(ws, start, 0) != cudaSuccess) {
        wstatus[w] = DCG_ERR_CUDA;
        werr[w] = "dcg_solve_batched: worker stream setup failed";
      } else {
        for (;;) {
          const int pi = next.fetch_add(1);
          if (pi >= nprob) break;
          for (int r = 0; r < nrhs; ++r) {
            const int k = pi * nrhs + r;
            const int st = solve_device(probs[pi], f_dev[k], x_dev[k], tol, max_it, &stats[k], ws);
            if (st != DCG_OK && st != DCG_ERR_NOT_CONVERGED && st != DCG_ERR_BREAKDOWN) {
              stats[k].status = st;
              if (wstatus[w] == DCG_OK) {
                wstatus[w] = st;
                werr[w] = dcg_last_error();
              }
            }
          }
        }
        cudaEventRecord(done, ws);
        cudaStreamWaitEvent(caller, done, 0);
        cudaStreamSynchronize(ws);
      }
      if (done) cudaEventDestroy(done);
      if (ws) cudaStreamDestroy(ws);
    });
  }
  for (auto& t : pool) t.join();
  cudaEventDestroy(start);
  for (int w = 0; w < nworkers; ++w)
    if (wstatus[w] != DCG_OK) {
      set_error_msg(werr[w]);
      return wstatus[w];
    }
  int worst = DCG_OK;
  for (int k = 0; k < nprob * nrhs; ++k)
    if (stats[k].status != DCG_OK && worst == DCG_OK) worst = stats[k].status;
  return worst;
}

int dcg_autotune(dcg_problem* p, const dcg_options* base, const double* f_dev, double inner_tol, int reps,
                 dcg_options* best, double* best_ms, void* stream) {
  if (!p || !base || !f_dev || !best || !best_ms || !(inner_tol > 0) || reps < 1) {
    set_error_msg("dcg_autotune: need problem, base, f, best, best_ms, inner_tol > 0, reps >= 1");
    return DCG_ERR_INVALID_ARG;
  }
  if (!base->deflate || base->inner_rule == DCG_INNER_EXACT) {
    set_error_msg("dcg_autotune: only W-cycle (deflated, non-exact) options have tunables");
    return DCG_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<dcg_options> cand;
  const int tiles[4][2] = {{4, 1}, {8, 1}, {8, 2}, {12, 2}};
  for (int lv = 2; lv <= 4; ++lv)
    for (const auto& t : tiles)
      for (int inv = 0; inv < (base->precision == DCG_MIXED ? 2 : 1); ++inv) {
        dcg_options o = *base;
        o.max_levels = lv;
        o.patch = t[0];
        o.overlap = t[1];
        if (base->precision == DCG_MIXED) o.ras_inverse = inv ? DCG_INV_BF16 : DCG_INV_FP32;
        long long box = 1;
        for (int a = 0; a < p->dim; ++a) box *= o.patch + 2 * o.overlap;
        if (box > 256) continue;
        if (lv > 2 && (int)level_sizes(p->n, lv).size() < lv) continue;  // mesh allows fewer levels
        cand.push_back(o);
      }
  double *g = nullptr, *z = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = DCG_OK;
  float best_t = 0.f;
  bool have = false;
  auto cleanup = [&]() {
    if (g) cudaFree(g);
    if (z) cudaFree(z);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaMalloc(&g, sizeof(double) * p->n_nodes) != cudaSuccess ||
      cudaMalloc(&z, sizeof(double) * p->n_nodes) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    cleanup();
    set_error_msg("dcg_autotune: allocation failed");
    return DCG_ERR_OOM;
  }
  for (const dcg_options& o : cand) {
    if ((rc = dcg_setup(p, &o, stream)) != DCG_OK) {
      if (rc == DCG_ERR_UNSUPPORTED || rc == DCG_ERR_INVALID_ARG) continue;  // candidate outside the kernels
      break;
    }
    if ((rc = vec_extract(p, f_dev, g, -1, s)) != DCG_OK) break;
    int ncyc = 0;
    // one untimed solve builds and warms the W-cycle graph
    if ((rc = cudaMemsetAsync(z, 0, sizeof(double) * p->n_nodes, s) == cudaSuccess ? DCG_OK : DCG_ERR_CUDA) ||
        (rc = mg_solve(p, g, z, inner_tol, o.inner_nmax, &ncyc, s)) != DCG_OK)
      break;
    if (ncyc >= o.inner_nmax) continue;
    float ms = 0.f;
    if (cudaEventRecord(e0, s) != cudaSuccess) { rc = DCG_ERR_CUDA; break; }
    for (int r = 0; r < reps && rc == DCG_OK; ++r) {
      if (cudaMemsetAsync(z, 0, sizeof(double) * p->n_nodes, s) != cudaSuccess) rc = DCG_ERR_CUDA;
      else rc = mg_solve(p, g, z, inner_tol, o.inner_nmax, &ncyc, s);
    }
    if (rc != DCG_OK) break;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = DCG_ERR_CUDA;
      break;
    }
    if (!have || ms < best_t) {
      best_t = ms;
      *best = o;
      have = true;
    }
  }
  cleanup();
  if (rc != DCG_OK) return rc;
  if (!have) {
    set_error_msg("dcg_autotune: no candidate reached inner_tol within inner_nmax cycles");
    return DCG_ERR_NOT_CONVERGED;
  }
  *best_ms = best_t / reps;
  return dcg_setup(p, best, stream);
}

void dcg_destroy(dcg_problem* p) {
  if (!p) return;
  graph_free(p);
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

int dcg_level_nodes(const dcg_problem* p, int level, long long* nodes) {
  if (!p || !nodes) return DCG_ERR_INVALID_ARG;
  if (!p->is_setup || p->levels.empty()) return DCG_ERR_STATE;
  if (level < 1 || level > (int)p->levels.size()) {
    set_error_msg("dcg_level_nodes: level out of range");
    return DCG_ERR_INVALID_ARG;
  }
  *nodes = p->levels[level - 1].nn;
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

int dcg_spmv_prec(const dcg_problem* p, const double* x, double* y, int precision, void* stream) {
  if (!p || !x || !y || (precision != DCG_FP64 && precision != DCG_MIXED)) {
    set_error_msg("dcg_spmv_prec: need problem, x, y and precision DCG_FP64 or DCG_MIXED");
    return DCG_ERR_INVALID_ARG;
  }
  if (precision == DCG_MIXED && !p->matrix_free) {
    set_error_msg("dcg_spmv_prec: FP32 arithmetic is implemented for the matrix-free operator only");
    return DCG_ERR_UNSUPPORTED;
  }
  return spmv_plain(const_cast<dcg_problem*>(p), x, y, (cudaStream_t)stream, precision == DCG_MIXED);
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
  graph_free(p);
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

long long dcg_kernel_launches(void) { return g_launch_count.load(); }

}  // extern "C"
