// Deflated-CG solves captured whole into one CUDA graph, with every loop of
// the method a conditional WHILE node whose condition a one-thread control
// kernel sets on the device: the restart loop around Algorithm 2's passes,
// the FCG iteration of Algorithm 1 (stop on ||r_i|| <= tol ||f||, Section
// 4.1) and each Multigrid call of Algorithm 3 (stop on the inner tolerance
// tau_c or n_max). A solve is then one graph launch and one read of the
// statistics at its end: no host round trip per iteration or per W-cycle.
//
// The kernels and their order are those of the host-driven solver
// (solver.cu), so for a zero initial guess the two give the same iterates
// bit for bit. A nonzero initial guess x0 is handled as the residual equation
// A e = f - A x0 (the form the restarts use), which converges to the same
// solution by a different sequence. The stall restart, the breakdown test,
// the adaptive inner tolerance (Eq. tol) and FCG with the truncation-restart
// rule run in the control kernels exactly as on the host.
//
// Batches (dcg_solve_batched): every (problem, right-hand side) pair is
// captured into one graph, the pairs of one problem in sequence (they share
// its buffers), different problems as independent branches; each pair stops
// at its own convergence test through its own conditional nodes, so the
// whole batch is one launch.
#include "common.cuh"

#include <chrono>
#include <cmath>
#include <cstring>

namespace dcg {

// Device-resident state of one solve (one per problem: the pairs of a
// problem run in sequence and save their statistics at their end).
struct GState {
  double tol, eps, fnorm, c, mg_tol, mg_gn, best, relres;
  int max_it, nmax, rule_adaptive, fcginf, fcg_cap, window, max_restarts, mf_lowp;
  int outer_its, total_cycles, iter_cycles, restarts, claimed, fcg_truncated, status, passes;
  int its_pass, its_best, stalled, stop, mg_n, mg_in_iter, ndir, first;
};

namespace {

__global__ void k_g_zero(double* __restrict__ v, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    v[i] = 0.0;
}

__global__ void k_g_copy(double* __restrict__ dst, const double* __restrict__ src, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// x = 0 when the right-hand side is zero (that is the solution)
__global__ void k_g_zero_if_no_rhs(double* __restrict__ x, long long n, const GState* __restrict__ S) {
  if (S->fnorm != 0.0) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = 0.0;
}

// after (f, f) -> S_FF: the solve's threshold eps = tol ||f||; counters reset
__global__ void k_g_begin(GState* S, const double* __restrict__ sc, double tol, int max_it) {
  S->tol = tol;
  S->max_it = max_it;
  S->fnorm = sqrt(sc[S_FF]);
  S->eps = tol * S->fnorm;
  S->outer_its = S->total_cycles = S->iter_cycles = S->restarts = S->claimed = S->fcg_truncated = 0;
  S->passes = 0;
  S->stalled = 0;
  S->first = 1;
  S->relres = 0.0;
  S->status = isfinite(S->fnorm) ? DCG_OK : DCG_ERR_BREAKDOWN;
}

// after u = f - A x (||u||^2 -> S_TMP0): the solver's restart rule (true
// relative residual above tol, within the iteration cap, and a pass budget:
// the first pass, a pass after a stall, or at most max_restarts more after
// passes that converged)
__global__ void k_g_pass_check(GState* S, const double* __restrict__ sc, cudaGraphConditionalHandle h) {
  bool run = false;
  if (S->status == DCG_OK && S->fnorm > 0.0) {
    S->relres = sqrt(sc[S_TMP0]) / S->fnorm;
    if (!isfinite(S->relres)) {
      S->status = DCG_ERR_BREAKDOWN;
    } else if (S->relres > S->tol && S->outer_its < S->max_it) {
      if (S->first) {
        run = true;
      } else if (S->stalled || S->claimed < S->max_restarts) {
        if (!S->stalled) S->claimed += 1;
        S->restarts += 1;
        run = true;
      }
    }
  }
  S->first = 0;
  if (run) S->passes += 1;
  cudaGraphSetConditional(h, run ? 1u : 0u);
}

// r = f_D and d = r at the start of a pass (S_DR <- S_RR); first outer test
__global__ void k_g_outer_init(GState* S, double* __restrict__ sc, int* __restrict__ ndir,
                               cudaGraphConditionalHandle h) {
  sc[S_DR] = sc[S_RR];
  const double rn = sqrt(sc[S_RR]);
  S->its_pass = 0;
  S->its_best = 0;
  S->best = rn;
  S->stalled = 0;
  S->ndir = 0;
  if (ndir) *ndir = 0;
  const bool run = !(rn <= S->eps) && S->outer_its < S->max_it;
  S->stop = run ? 0 : 1;
  cudaGraphSetConditional(h, run ? 1u : 0u);
}

// inner tolerance of an outer iteration: c tol (Eq. fixed_tol) or
// c tol ||f|| / ||r_i|| (Eq. tol); c tol for the other inner solves
__global__ void k_g_inner_tol(GState* S, const double* __restrict__ sc, int in_iter) {
  S->mg_tol = (in_iter && S->rule_adaptive) ? S->c * S->eps / sqrt(sc[S_RR]) : S->c * S->tol;
  S->mg_in_iter = in_iter;
}

// Algorithm 3's test before each cycle: n < n_max and ||g - Z z|| / ||g|| > tol
__global__ void k_g_mg_check(GState* S, const double* __restrict__ sc, int first, cudaGraphConditionalHandle h) {
  if (first) {
    S->mg_n = 0;
    S->mg_gn = sqrt(sc[S_TMP1]);
  } else {
    S->mg_n += 1;
    S->total_cycles += 1;
    if (S->mg_in_iter) S->iter_cycles += 1;
  }
  const double rn = sqrt(sc[S_TMP0]);
  const bool run = S->mg_gn > 0.0 && rn / S->mg_gn > S->mg_tol && S->mg_n < S->nmax;
  cudaGraphSetConditional(h, run ? 1u : 0u);
}

// after the update (S_DQ, S_RRN): breakdown, convergence, stall and cap
// tests of the outer iteration, in the host-driven loop's order
__global__ void k_g_outer_check(GState* S, const double* __restrict__ sc, cudaGraphConditionalHandle h) {
  S->outer_its += 1;
  const double dq = sc[S_DQ], rrn = sc[S_RRN];
  bool stop = false;
  if (S->fcginf) S->ndir += 1;  // d_{i-1} was stored before the update
  if (!(dq > 0.0) || !isfinite(dq) || !isfinite(rrn)) {
    if (S->mf_lowp && isfinite(dq) && isfinite(rrn)) S->stalled = 1;
    else S->status = DCG_ERR_BREAKDOWN;
    stop = true;
  } else if (sqrt(rrn) <= S->eps) {
    stop = true;
  } else {
    S->its_pass += 1;
    const double rn = sqrt(rrn);
    if (rn < 0.99 * S->best) {
      S->best = rn;
      S->its_best = S->its_pass;
    } else if (S->window > 0 && S->its_pass - S->its_best > max(S->window, S->its_pass / 4)) {
      S->stalled = 1;
      stop = true;
    }
  }
  if (!stop && S->outer_its >= S->max_it) stop = true;
  if (!stop && S->fcginf) {
    // d_i is built from the m_i = max{1, mod(i, m_max + 1)} latest directions
    const int i = S->ndir;
    if (min(max(1, i % (S->fcg_cap + 1)), i) < i) S->fcg_truncated += 1;
  }
  S->stop = stop ? 1 : 0;
  cudaGraphSetConditional(h, stop ? 0u : 1u);
}

__global__ void k_g_finish(GState* S, GState* save) {
  if (S->fnorm == 0.0 && S->status == DCG_OK) S->relres = 0.0;
  else if (S->status == DCG_OK && !(S->relres <= S->tol)) S->status = DCG_ERR_NOT_CONVERGED;
  if (save) *save = *S;
}

// A pool of capture streams, one per nesting depth of conditional bodies.
struct Capture {
  std::vector<cudaStream_t> streams;
  int depth = 0;
  int acquire(cudaStream_t* out) {
    if ((int)streams.size() <= depth) {
      cudaStream_t t = nullptr;
      DCG_CUDA(cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking));
      streams.push_back(t);
    }
    *out = streams[depth++];
    return DCG_OK;
  }
  void release() { --depth; }
  ~Capture() {
    for (auto t : streams) cudaStreamDestroy(t);
  }
};

// Kernels each loop body launches per iteration (nested loops excluded):
// with the loop counters they give the launches of a graph run.
struct BodyCounts {
  long long top = 0, pass = 0, outer = 0, mg = 0;
};

struct Builder {
  dcg_problem* p;
  GState* S;
  Capture* cap;
  BodyCounts* counts;
  long long nested = 0;  // kernels captured by loop bodies nested in the current one

  int handle(cudaStream_t s, cudaGraphConditionalHandle* h) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    DCG_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    DCG_CUDA(cudaGraphConditionalHandleCreate(h, g, 0, 0));
    return DCG_OK;
  }

  // WHILE node on handle h after what `s` has captured; `fn(bs)` captures the
  // body on a stream of the next nesting depth. *direct = kernels the body
  // launches itself (its nested loops excluded).
  template <typename Fn>
  int loop(cudaStream_t s, cudaGraphConditionalHandle h, long long* direct, Fn fn) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    DCG_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    DCG_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp));
    DCG_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaStream_t bs = nullptr;
    DCG_TRY(cap->acquire(&bs));
    DCG_CUDA(cudaStreamBeginCaptureToGraph(bs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal));
    const long long start = t_capture_launches, outer_nested = nested;
    nested = 0;
    const int st = fn(bs);
    const long long all = t_capture_launches - start;
    *direct = all - nested;
    nested = outer_nested + all;
    cudaGraph_t out = nullptr;
    const cudaError_t e = cudaStreamEndCapture(bs, &out);
    cap->release();
    if (st != DCG_OK) return st;
    if (e != cudaSuccess) {
      set_error("cudaStreamEndCapture (loop body)", e);
      return DCG_ERR_CUDA;
    }
    return DCG_OK;
  }

  int zero(double* v, long long n, cudaStream_t s) {
    k_g_zero<<<grid_for(n, 256, 8192), 256, 0, s>>>(v, n);
    DCG_LAUNCH_CHECK();
    return DCG_OK;
  }

  // Algorithm 3 on g -> z from z = 0 with the tolerance k_g_inner_tol set
  int multigrid(const double* g, double* z, cudaStream_t s, int in_iter) {
    k_g_inner_tol<<<1, 1, 0, s>>>(S, p->scal, in_iter);
    DCG_LAUNCH_CHECK();
    DCG_TRY(zero(z, p->n_nodes, s));
    DCG_TRY(mg_graph_residual(p, g, z, true, s));
    cudaGraphConditionalHandle h = 0;
    DCG_TRY(handle(s, &h));
    k_g_mg_check<<<1, 1, 0, s>>>(S, p->scal, 1, h);
    DCG_LAUNCH_CHECK();
    return loop(s, h, &counts->mg, [&](cudaStream_t bs) -> int {
      DCG_TRY(mg_graph_wcycle(p, bs));
      DCG_TRY(mg_graph_accumulate(p, z, bs));
      DCG_TRY(mg_graph_residual(p, g, z, false, bs));
      k_g_mg_check<<<1, 1, 0, bs>>>(S, p->scal, 0, h);
      DCG_LAUNCH_CHECK();
      return DCG_OK;
    });
  }

  // One pass of Algorithm 2 on A e = u from zero (e in b.e), then x += e and
  // the true residual u = f - A x (||u||^2 -> S_TMP0)
  int pass(const double* f, double* x, cudaStream_t s) {
    SolverBuffers& b = p->sb;
    const long long N = p->N;
    // pi(u): zf = MG(V^T u)
    DCG_TRY(vec_extract(p, b.u, b.g, S_GG, s));
    DCG_TRY(multigrid(b.g, b.zf, s, 0));
    // r = f_D = u - A V zf; xh = 0; d = r
    DCG_TRY(spmv_f_minus_avz(p, b.u, b.zf, b.r, S_RR, s));
    DCG_TRY(zero(b.xh, N, s));
    k_g_copy<<<grid_for(N, 256, 8192), 256, 0, s>>>(b.d, b.r, N);
    DCG_LAUNCH_CHECK();
    cudaGraphConditionalHandle ho = 0;
    DCG_TRY(handle(s, &ho));
    k_g_outer_init<<<1, 1, 0, s>>>(S, p->scal, b.ndir_dev, ho);
    DCG_LAUNCH_CHECK();
    const int rec = p->opts.recurrence;
    DCG_TRY(loop(s, ho, &counts->outer, [&](cudaStream_t bs) -> int {
      // q = M_D d: t = A d with g = V^T t, zh = MG(g, tau_c), q = t - K_div V zh
      DCG_TRY(spmv_y_vt(p, b.d, b.w, b.g, S_GG, bs));
      DCG_TRY(multigrid(b.g, b.zh, bs, 1));
      DCG_TRY(q_from_t(p, b.w, b.zh, b.d, b.q, S_DQ, bs));
      if (rec == DCG_FCG_INF) DCG_TRY(solver_fcg_store(p, bs));
      DCG_TRY(solver_update(p, b.xh, b.r, b.d, b.q, rec != DCG_FR, bs));
      k_g_outer_check<<<1, 1, 0, bs>>>(S, p->scal, ho);
      DCG_LAUNCH_CHECK();
      // the next direction (skipped by the kernels once the loop stops)
      if (rec == DCG_FCG_INF) DCG_TRY(solver_fcg_direction(p, bs, &S->stop, b.ndir_cap, b.ndir_cap));
      else DCG_TRY(solver_direction(p, b.d, b.r, rec == DCG_FCG1, bs, &S->stop));
      return DCG_OK;
    }));
    // reconstruction e = xh - pi(A xh) + pi(u)
    DCG_TRY(spmv_vt(p, b.xh, b.g, S_GG, s));
    DCG_TRY(multigrid(b.g, b.zh, s, 0));
    DCG_TRY(solver_reconstruct(p, b.xh, b.zh, b.zf, b.e, s));
    DCG_TRY(solver_axpy(p, x, b.e, s));
    DCG_TRY(spmv_residual(p, f, x, b.u, S_TMP0, s));
    return DCG_OK;
  }

  // the whole solve of (f, x) on the capturing stream s
  int solve(const double* f, double* x, double tol, int max_it, GState* save, cudaStream_t s) {
    const long long N = p->N;
    SolverBuffers& b = p->sb;
    const long long k0 = t_capture_launches;
    nested = 0;
    DCG_TRY(vec_dot(p, f, f, N, S_FF, s));
    k_g_begin<<<1, 1, 0, s>>>(S, p->scal, tol, max_it);
    DCG_LAUNCH_CHECK();
    k_g_zero_if_no_rhs<<<grid_for(N, 256, 8192), 256, 0, s>>>(x, N, S);
    DCG_LAUNCH_CHECK();
    DCG_TRY(spmv_residual(p, f, x, b.u, S_TMP0, s));
    cudaGraphConditionalHandle hp = 0;
    DCG_TRY(handle(s, &hp));
    k_g_pass_check<<<1, 1, 0, s>>>(S, p->scal, hp);
    DCG_LAUNCH_CHECK();
    DCG_TRY(loop(s, hp, &counts->pass, [&](cudaStream_t bs) -> int {
      DCG_TRY(pass(f, x, bs));
      k_g_pass_check<<<1, 1, 0, bs>>>(S, p->scal, hp);
      DCG_LAUNCH_CHECK();
      return DCG_OK;
    }));
    k_g_finish<<<1, 1, 0, s>>>(S, save);
    DCG_LAUNCH_CHECK();
    counts->top += t_capture_launches - k0 - nested;
    return DCG_OK;
  }
};

// Host copy of the constant fields of a problem's device state.
GState state_constants(const dcg_problem* p) {
  GState h{};
  const dcg_options& o = p->opts;
  h.c = o.c;
  h.nmax = o.inner_nmax;
  h.rule_adaptive = o.inner_rule == DCG_INNER_ADAPTIVE;
  h.fcginf = o.recurrence == DCG_FCG_INF;
  h.fcg_cap = p->sb.ndir_cap;
  h.window = o.stall_window;
  h.max_restarts = o.max_restarts;
  h.mf_lowp = mf_lowp(p) ? 1 : 0;
  return h;
}

void stats_from(const GState& h, dcg_stats* st) {
  *st = dcg_stats{};
  st->status = h.status;
  st->outer_its = h.outer_its;
  st->total_mg_cycles = h.total_cycles;
  st->iter_mg_cycles = h.iter_cycles;
  st->restarts = h.restarts;
  st->true_relres = h.relres;
  st->fcg_truncated = h.fcg_truncated;
  st->avg_inner = h.outer_its ? (double)h.iter_cycles / h.outer_its : 0.0;
}

long long launches_of(const GState& h, const BodyCounts& c) {
  return c.top + (long long)h.passes * c.pass + (long long)h.outer_its * c.outer + (long long)h.total_cycles * c.mg;
}

// Captures `build(capture_stream)` into a graph and instantiates it.
template <typename Fn>
int capture_graph(Fn build, cudaGraphExec_t* exec) {
  cudaStream_t cs = nullptr;
  DCG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    set_error("cudaStreamBeginCapture", e);
    return DCG_ERR_CUDA;
  }
  const bool was = t_capturing;
  const long long saved = t_capture_launches;
  t_capturing = true;
  t_capture_launches = 0;
  int st = build(cs);
  t_capturing = was;
  t_capture_launches = saved;
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cs, &graph);
  cudaStreamDestroy(cs);
  if (st != DCG_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) {
    set_error("cudaStreamEndCapture", e);
    return DCG_ERR_CUDA;
  }
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    set_error("cudaGraphInstantiate (solve graph)", e);
    return DCG_ERR_CUDA;
  }
  return DCG_OK;
}

}  // namespace

bool graph_solve_supported(const dcg_problem* p) {
  return p->opts.device_loop && p->opts.deflate && !mg_exact(p) && !p->matrix_free && p->prof.mask == 0 &&
         p->sb.w != nullptr && p->opts.recurrence != DCG_GMRES;
}

void graph_free(dcg_problem* p) {
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  p->gexec = nullptr;
  cudaFree(p->gstate);
  p->gstate = nullptr;
  p->gkey_f = nullptr;
  p->gkey_x = nullptr;
}

int graph_solve(dcg_problem* p, const double* f, double* x, double tol, int max_it, dcg_stats* st, cudaStream_t s) {
  auto t0 = std::chrono::steady_clock::now();
  if (!p->gstate) DCG_CUDA(cudaMalloc(&p->gstate, sizeof(GState)));
  GState* S = static_cast<GState*>(p->gstate);
  if (!p->gexec || p->gkey_f != f || p->gkey_x != x || p->gkey_tol != tol || p->gkey_maxit != max_it) {
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
    BodyCounts counts;
    Capture cap;
    Builder B{p, S, &cap, &counts};
    DCG_TRY(capture_graph([&](cudaStream_t cs) { return B.solve(f, x, tol, max_it, nullptr, cs); }, &p->gexec));
    p->gcounts[0] = counts.top;
    p->gcounts[1] = counts.pass;
    p->gcounts[2] = counts.outer;
    p->gcounts[3] = counts.mg;
    p->gkey_f = f;
    p->gkey_x = x;
    p->gkey_tol = tol;
    p->gkey_maxit = max_it;
  }
  const GState h0 = state_constants(p);
  DCG_CUDA(cudaMemcpyAsync(S, &h0, sizeof(GState), cudaMemcpyHostToDevice, s));
  DCG_CUDA(cudaGraphLaunch(p->gexec, s));
  GState h{};
  DCG_CUDA(cudaMemcpyAsync(&h, S, sizeof(GState), cudaMemcpyDeviceToHost, s));
  DCG_CUDA(cudaStreamSynchronize(s));
  if (p->scal_host) {
    // the bounded device waits of the bulk-copy kernels report here
    DCG_CUDA(cudaMemcpy(p->scal_host, p->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost));
    if (p->scal_host[S_ERR] != 0.0) {
      set_error_msg("a bounded device wait gave up (bulk copy did not complete)");
      return DCG_ERR_CUDA;
    }
  }
  stats_from(h, st);
  if (h.status == DCG_ERR_BREAKDOWN && (!std::isfinite(h.fnorm) || !std::isfinite(h.relres)))
    set_error_msg("dcg_solve: non-finite entries in the right-hand side or the initial guess");
  const BodyCounts c{p->gcounts[0], p->gcounts[1], p->gcounts[2], p->gcounts[3]};
  g_launch_count += launches_of(h, c);
  st->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return st->status;
}

// One graph for a whole batch: problem i's pairs in sequence on branch i.
int graph_solve_batched(int nprob, dcg_problem* const* probs, int nrhs, const double* const* f, double* const* x,
                        double tol, int max_it, dcg_stats* stats, cudaStream_t s) {
  GState* saves = nullptr;
  DCG_CUDA(cudaMalloc(&saves, sizeof(GState) * (size_t)nprob * nrhs));
  std::vector<BodyCounts> counts(nprob);
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaStream_t> branch(nprob, nullptr);
  std::vector<cudaEvent_t> evs;
  int rc = DCG_OK;
  for (int i = 0; i < nprob && rc == DCG_OK; ++i) {
    dcg_problem* p = probs[i];
    if (!p->gstate && cudaMalloc(&p->gstate, sizeof(GState)) != cudaSuccess) rc = DCG_ERR_OOM;
    if (rc == DCG_OK && cudaStreamCreateWithFlags(&branch[i], cudaStreamNonBlocking) != cudaSuccess) rc = DCG_ERR_CUDA;
  }
  if (rc == DCG_OK) {
    rc = capture_graph(
        [&](cudaStream_t cs) -> int {
          cudaEvent_t fork = nullptr;
          DCG_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
          evs.push_back(fork);
          DCG_CUDA(cudaEventRecord(fork, cs));
          for (int i = 0; i < nprob; ++i) {
            dcg_problem* p = probs[i];
            DCG_CUDA(cudaStreamWaitEvent(branch[i], fork, 0));
            Capture cap;
            Builder B{p, static_cast<GState*>(p->gstate), &cap, &counts[i]};
            for (int r = 0; r < nrhs; ++r) {
              const int k = i * nrhs + r;
              DCG_TRY(B.solve(f[k], x[k], tol, max_it, saves + k, branch[i]));
            }
            cudaEvent_t join = nullptr;
            DCG_CUDA(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
            evs.push_back(join);
            DCG_CUDA(cudaEventRecord(join, branch[i]));
            DCG_CUDA(cudaStreamWaitEvent(cs, join, 0));
          }
          return DCG_OK;
        },
        &exec);
  }
  if (rc == DCG_OK) {
    for (int i = 0; i < nprob && rc == DCG_OK; ++i) {
      const GState h0 = state_constants(probs[i]);
      if (cudaMemcpyAsync(probs[i]->gstate, &h0, sizeof(GState), cudaMemcpyHostToDevice, s) != cudaSuccess)
        rc = DCG_ERR_CUDA;
    }
  }
  std::vector<GState> hs((size_t)nprob * nrhs);
  if (rc == DCG_OK) {
    cudaError_t e = cudaGraphLaunch(exec, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hs.data(), saves, sizeof(GState) * hs.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error("dcg_solve_batched (graph launch)", e);
      rc = DCG_ERR_CUDA;
    }
  }
  if (rc == DCG_OK) {
    for (int i = 0; i < nprob; ++i)
      for (int r = 0; r < nrhs; ++r) {
        const int k = i * nrhs + r;
        stats_from(hs[k], &stats[k]);
        g_launch_count += launches_of(hs[k], BodyCounts{counts[i].top / nrhs, counts[i].pass, counts[i].outer,
                                                        counts[i].mg});
      }
  }
  if (exec) cudaGraphExecDestroy(exec);
  for (auto e : evs) cudaEventDestroy(e);
  for (auto b : branch)
    if (b) cudaStreamDestroy(b);
  cudaFree(saves);
  return rc;
}

}  // namespace dcg
