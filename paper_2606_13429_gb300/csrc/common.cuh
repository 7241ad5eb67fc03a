// Common device helpers and the problem object of libdcg.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dcg.h"

namespace dcg {

void set_error(const char* what, cudaError_t e);
void set_error_msg(const std::string& msg);

#define DCG_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e__ = (call);                            \
    if (e__ != cudaSuccess) {                            \
      ::dcg::set_error(#call, e__);                      \
      return e__ == cudaErrorMemoryAllocation ? DCG_ERR_OOM : DCG_ERR_CUDA; \
    }                                                    \
  } while (0)

#define DCG_TRY(expr)          \
  do {                         \
    int s__ = (expr);          \
    if (s__ != DCG_OK) return s__; \
  } while (0)

// Every kernel launch is followed by DCG_LAUNCH_CHECK(), which also counts it
// (launches captured into the W-cycle graph are counted per replay instead).
extern std::atomic<long long> g_launch_count;
extern thread_local bool t_capturing;           // this thread is capturing the W-cycle graph
extern thread_local long long t_capture_launches;
inline void note_launches(long long n) {
  if (t_capturing) t_capture_launches += n;
  else g_launch_count += n;
}
#define DCG_LAUNCH_CHECK()                 \
  do {                                     \
    ::dcg::note_launches(1);               \
    DCG_CUDA(cudaGetLastError());          \
  } while (0)

constexpr int kMaxDim = 3;
constexpr int kRedThreads = 256;

// ---------------------------------------------------------------------------
// Deterministic reductions: every CTA writes its partial sums (fixed
// partition of the index range), the last CTA to finish sums the partials
// in block order and writes the result; results do not depend on timing.
// ---------------------------------------------------------------------------
struct Reduce {
  double* partials;   // [max_ctas * kMaxVals]
  unsigned* counter;  // one per reduction slot, zero between launches
  double* out;        // destination scalars (device)
};
constexpr int kMaxVals = 4;
constexpr int kMaxRedCtas = 65536;
// grid of the kernels that end in grid_reduce: a few CTAs per SM, each
// thread looping over several items, so that the per-thread share of the
// block reduction (FP64 shuffles and adds, which this GPU issues slowly)
// is amortised
constexpr int kRedGrid = 8 * 152;

// Block-wide sums of NV doubles per thread, left in thread 0. This GPU
// issues FP64 at 2 lanes per clock per SM, so a warp-wide FP64 add costs 16
// SM clocks whatever its lanes do. Blocks of up to kRedTree threads (whole
// warps) therefore stage their partials in shared memory, warp 0 adds the
// nwarp values of each lane (nwarp - 1 FP64 warp instructions per value) and
// folds its 32 lanes (5 more): 12 instructions per value for 256 threads,
// against 45 for a shuffle tree in every warp. Fixed order: deterministic.
constexpr int kRedTree = 256;
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* smem /*[32*NV]*/) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarp = (blockDim.x + 31) >> 5;
  if (blockDim.x <= kRedTree && (blockDim.x & 31) == 0) {
    __shared__ double stage[kRedTree * NV];
    const int bd = blockDim.x;
    __syncthreads();  // a previous call's readers are done with the stage
#pragma unroll
    for (int k = 0; k < NV; ++k) stage[k * bd + threadIdx.x] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        double x = stage[k * bd + lane];
        for (int w = 1; w < nwarp; ++w) x += stage[k * bd + w * 32 + lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        v[k] = x;
      }
    }
    return;
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    v[k] = x;
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) smem[warp * NV + k] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = lane < nwarp ? smem[lane * NV + k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      v[k] = x;
    }
  }
}

// Called by every thread of every CTA after its partials are final.
// out[k] = sum over CTAs of partial k. Thread 0 of CTA 0..grid-1 contributes.
template <int NV>
__device__ __forceinline__ void grid_reduce(double (&v)[NV], const Reduce& r) {
  __shared__ double smem[32 * NV];
  __shared__ bool last;
  block_sum<NV>(v, smem);
  const unsigned nb = gridDim.x;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) r.partials[(size_t)k * kMaxRedCtas + blockIdx.x] = v[k];
    __threadfence();
    unsigned t = atomicAdd(r.counter, 1u);
    last = (t == nb - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = 0.0;
    for (unsigned b = threadIdx.x; b < nb; b += blockDim.x)
      s += __ldcg(&r.partials[(size_t)k * kMaxRedCtas + b]);
    acc[k] = s;
  }
  block_sum<NV>(acc, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) r.out[k] = acc[k];
    *r.counter = 0u;
  }
}

// ---------------------------------------------------------------------------
// Constant 3^d stencil of one multigrid level (index (dx+1) + 3(dy+1) + 9(dz+1)).
// ---------------------------------------------------------------------------
template <typename T>
struct Stencil {
  T c[27];
};

// RAS tile geometry along one axis of a level.
struct Tiles1D {
  int m, P, o, ntile;
  __host__ __device__ int ext_lo(int t) const { int v = t * P - o; return v < 0 ? 0 : v; }
  __host__ __device__ int ext_hi(int t) const { int v = (t + 1) * P + o; return v > m ? m : v; }
  __host__ __device__ int core_lo(int t) const { return t * P; }
  __host__ __device__ int core_hi(int t) const { int v = (t + 1) * P; return v > m ? m : v; }
};

struct RasClass {
  int len[kMaxDim];   // box extent per axis
  int np;             // prod(len)
  int npp;            // np rounded up to a multiple of 4 (row length of the stored inverse)
  int npk;            // np rounded up to a multiple of 16 (tensor-core N and K)
  int local_off;      // offset of the class's packed local coordinates
  int nb;             // boxes per work item (batch width of the product)
  long long inv_off;  // offset of the inverse in the level's inverse array
  int fdm_s[kMaxDim]; // fast diagonalisation: offset of each axis's sine matrix in the level's table
  long long fdm_tri;  // fast diagonalisation: offset of the line-solve factors along the last axis
};

struct Level {
  int n = 0, m = 0;
  long long nn = 0;                 // m^d nodes
  Stencil<double> st64{};
  Stencil<float> st32{};
  // 2D stencil with 8 equal neighbour coefficients (the Q1 Laplacian):
  // Z z = box_c0 z + box_c1 (3 x 3 box sum), box_c0 = centre - box_c1
  bool box = false;
  double box_c0 = 0.0, box_c1 = 0.0;
  // RAS
  Tiles1D tiles{};
  int npatch = 0, nclass = 0, npmax = 0;
  std::vector<RasClass> classes;
  int* d_patch_class = nullptr;     // [npatch]
  int* d_work = nullptr;            // [nwork * 3] (class, first index into d_class_patches, count)
  int* d_class_patches = nullptr;   // patch ids grouped by class
  RasClass* d_classes = nullptr;
  int4* d_origin = nullptr;         // [npatch] box origin coordinates and node
  int* d_local = nullptr;           // packed local coordinates of every class
  int4* d_axis_tab = nullptr;       // [m] boxes containing each coordinate
  int2* d_core = nullptr;           // [npatch] core tile in box-local coordinates
  int* d_local_node = nullptr;      // per class: node offset of each local node from the box origin
  long long* d_item_off = nullptr;  // [nwork] offset of each work item's results in y
  int* d_ysrc = nullptr;            // [nn * 2^d] index in y of each node's box results, -1 = none
  void* r = nullptr;                // residual f - Z z (cycle precision)
  int nwork = 0;
  long long ylen = 0;
  long long ras_np2 = 0;            // sum over boxes of np^2 (FMAs of one smoothing product)
  long long gmax = 0;               // max over classes of np * nb (residual tile elements)
  bool tc = false;                  // RAS products on the tensor cores (BF16 inverses)
  bool fdm = false;                 // FP64 local solves by fast diagonalisation and line solves
  int fdm_lmax = 0;                 // largest box extent along an axis (register bound of the kernel)
  double* d_fdm = nullptr;          // sine matrices and line-solve factors of every class
  double fdm_flops = 0.0;           // algorithmic flops of one fast-diagonalisation smoothing product
  void* d_inv = nullptr;            // inverses in the W-cycle precision (row-major, symmetric)
  void* d_inv_bf16 = nullptr;       // optional BF16 copy
  // vectors in the W-cycle precision
  void* f = nullptr;
  void* z = nullptr;
  void* y = nullptr;                // RAS box results, work-item layout [item][np][nb]
};

struct Coarse {
  int m = 0;          // interior nodes per axis on the coarsest level
  double* S64 = nullptr;   // m x m orthonormal sine matrix
  float* S32 = nullptr;
  // line solves along the last axis. FFT route (m = 2^q - 1): cyclic
  // reduction, tri_l = beta_k, tri_w = gamma_k ([q][m^(d-1)] each), tri_e
  // unused. Dense route: Thomas multipliers l and reciprocal pivots 1/w (m^d
  // each, layout of the data) and off-diagonals e (m^(d-1))
  double *tri_l64 = nullptr, *tri_w64 = nullptr, *tri_e64 = nullptr;
  float *tri_l32 = nullptr, *tri_w32 = nullptr, *tri_e32 = nullptr;
  void* tmp = nullptr;     // work vector (m^d, precision of the cycle)
  // FFT route when m + 1 is a power of two: log2(2(m+1)) (0: dense passes)
  // and the twiddles e^{-2 pi i j / (2(m+1))}, j < m + 1
  int log2n2 = 0;
  double2* tw64 = nullptr;
  float2* tw32 = nullptr;
};

struct SolverBuffers {
  double *xh = nullptr, *r = nullptr, *d = nullptr, *q = nullptr, *u = nullptr, *e = nullptr;
  double *g = nullptr, *zh = nullptr, *zf = nullptr, *rin = nullptr;  // inner FP64 (n_nodes)
  double* w = nullptr;     // operand d - V zh of the deflated product (assembled A)
  // FCG(inf) with the truncation-restart rule: ring of ndir_cap = m_max slots
  double* dirs = nullptr;  // [m_max][N] directions d_k (slot k mod m_max)
  double* qdirs = nullptr; // [m_max][N] q_k = M_D d_k
  double* dqs = nullptr;   // [m_max] (d_k, q_k)
  double* coef = nullptr;  // [m_max] (r_i, q_k) of the current window
  double* part = nullptr;  // [m_max * 304] per-CTA partial sums of the window's dot products
  int* ndir_dev = nullptr; // directions stored in the current pass (device counter)
  int ndir_cap = 0;
};

// ---------------------------------------------------------------------------
// Optional per-kernel-class timing with CUDA events (off by default). Direct
// launches record an event pair on their stream; launches inside the
// captured W-cycle graph carry external event-record nodes, read after each
// graph replay.
// ---------------------------------------------------------------------------
enum ProfClass {
  PC_SPMV = 0, PC_VEC, PC_RAS_SOLVE, PC_RAS_UPDATE, PC_TRANSFER, PC_COARSE, PC_INNER_RES, PC_COUNT
};
struct ProfPair {
  cudaEvent_t a = nullptr, b = nullptr;
  int cls = 0;
  double flops = 0, bytes = 0;
};
struct Prof {
  unsigned mask = 0;               // bit per ProfClass
  std::vector<cudaEvent_t> pool;
  std::vector<ProfPair> pending;   // direct launches since the last flush
  std::vector<ProfPair> graph;     // pairs inside the W-cycle graph
  double ms[PC_COUNT] = {}, flops[PC_COUNT] = {}, bytes[PC_COUNT] = {};
  long long launches[PC_COUNT] = {};
};

// Per-problem multigrid runtime state: the captured W-cycle graph and the
// stream used to capture it.
struct MGState {
  cudaStream_t cap = nullptr;
  cudaGraphExec_t wexec = nullptr;
  bool fp32 = false;
  long long graph_kernels = 0;  // kernel launches captured into the W-cycle graph
};

}  // namespace dcg

struct dcg_problem {
  int dim = 0, n = 0, m = 0, b = 0;
  long long n_nodes = 0, N = 0, nnzb = 0;
  double dt = 0, nu = 1;
  int matrix_free = 0;
  // BSR (device)
  int* row_ptr = nullptr;
  int* col_idx = nullptr;
  double* vals = nullptr;
  double* inv_nu_elem = nullptr;   // per-element 1/nu (device, matrix-free or assembly)
  // scratch for reductions
  double* partials = nullptr;
  unsigned* counters = nullptr;    // kNumCounters
  double* scal = nullptr;          // device scalars
  double* scal_host = nullptr;     // pinned mirror
  // setup
  bool is_setup = false;
  dcg_options opts{};
  std::vector<dcg::Level> levels;  // index 0 = coarsest
  dcg::Coarse coarse;
  dcg::SolverBuffers sb;
  double* fine_f64 = nullptr;      // staging for host-array solves (N)
  double* fine_x64 = nullptr;
  dcg::Prof prof;
  dcg::MGState mg;
  // solve captured into one CUDA graph (graph.cu): device state, the
  // instantiated graph and the arguments it was captured for, and the
  // kernels its loop bodies launch per iteration (top, pass, outer, cycle)
  void* gstate = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const double* gkey_f = nullptr;
  double* gkey_x = nullptr;
  double gkey_tol = 0.0;
  int gkey_maxit = 0;
  long long gcounts[4] = {0, 0, 0, 0};
};

namespace dcg {

// device scalar slots
// Pairs written by one two-value reduction are consecutive:
// (S_RRN, S_RQ) by the CG update, (S_TMP0, S_TMP1) by the inner residual.
enum Scal {
  S_DQ = 0, S_DR, S_RR, S_RRN, S_RQ, S_GG, S_FF, S_TMP0, S_TMP1, S_ALPHA, S_BETA, S_RES, S_ERR,
  S_COUNT = 16
};
constexpr int kNumCounters = 8;

inline Reduce make_reduce(dcg_problem* p, int slot, int counter = 0) {
  return Reduce{p->partials, p->counters + counter, p->scal + slot};
}

// 16-byte aligned (vector loads of two doubles allowed)
inline bool aligned16(const void* p) { return (reinterpret_cast<unsigned long long>(p) & 15ull) == 0; }

inline int grid_for(long long n, int threads, int cap = kMaxRedCtas) {
  long long g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// profiling (api.cu): prof_begin returns a pair index or -1 when the class
// is not profiled; capture = true inside W-cycle graph capture.
int prof_begin(dcg_problem* p, int cls, cudaStream_t s, bool capture = false);
void prof_end(dcg_problem* p, int idx, cudaStream_t s, double flops, double bytes, bool capture = false);
void prof_flush(dcg_problem* p);        // after a synchronisation of the stream
void prof_flush_graph(dcg_problem* p);  // after a synchronised W-cycle replay
void prof_clear_graph(dcg_problem* p);

// launchers implemented in the .cu files
int assemble_device(dcg_problem* p, const double* nu_elem_host, cudaStream_t s);
int spmv_plain(dcg_problem* p, const double* x, double* y, cudaStream_t s, bool lowp = false);
// y = A x with dot(dv, y) into scal[slot] when dv != nullptr
int spmv_dot(dcg_problem* p, const double* x, double* y, const double* dv, int slot, cudaStream_t s);
// y = f - A x, ||y||^2 into scal[slot]
int spmv_residual(dcg_problem* p, const double* f, const double* x, double* y, int slot, cudaStream_t s);
// g = V^T A x, ||g||^2 into scal[slot]
int spmv_vt(dcg_problem* p, const double* x, double* g, int slot, cudaStream_t s, bool lowp = false);
// q = A (x - V zh) (zh may be null => x), dot(x, q) into scal[slot]; if x null: q = A (V zh)
int spmv_defl(dcg_problem* p, const double* x, const double* zh, double* q, int slot, cudaStream_t s,
              bool lowp = false);
// y = f - A(V zh), ||y||^2 into scal[slot]
int spmv_f_minus_avz(dcg_problem* p, const double* f, const double* zh, double* y, int slot, cudaStream_t s);
// assembled operator: t = A x and g = V^T t in one pass (||g||^2 -> slot)
int spmv_y_vt(dcg_problem* p, const double* x, double* t, double* g, int slot, cudaStream_t s);
// q = t - A V zh through the divergence stencil (M_dev V = 0); (dv, q) -> slot
int q_from_t(dcg_problem* p, const double* t, const double* zh, const double* dv, double* q, int slot,
             cudaStream_t s);
// divergence stencil G[p*3+q][offset] of the uniform Q1 mesh (d = 2, 3)
void div_stencil(int d, int n, double (*gs)[27]);
// matrix-free 3D product (mf.cu): operand mode xm (0 x, 1 x - V zh, 2 V zh),
// output mode om (0 y, 1 f - y, 2 V^T y), fused dot when `dot`, FP32
// arithmetic when `lowp`
int mf_product(dcg_problem* p, int xm, int om, bool dot, bool lowp, const double* x, const double* zh,
               const double* f, double* y, const double* dvec, Reduce red, cudaStream_t s);
// FP32 matrix-free products inside the outer iterations (mixed precision)
// inner stencil of a matrix-free problem, and its check against the operator
int mf_probe_stencil(dcg_problem* p, double* stencil, cudaStream_t s);
int mf_check_stencil(dcg_problem* p, cudaStream_t s);
inline bool mf_lowp(const dcg_problem* p) { return p->matrix_free && p->opts.precision == DCG_MIXED; }

// vectors
int vec_extract(dcg_problem* p, const double* y, double* q, int slot, cudaStream_t s);
int vec_embed(dcg_problem* p, const double* q, double* y, cudaStream_t s);
int vec_dot(dcg_problem* p, const double* a, const double* b, long long n, int slot, cudaStream_t s);
int vec_copy(double* dst, const double* src, long long n, cudaStream_t s);
int vec_zero(double* dst, long long n, cudaStream_t s);

// solver
int solve_device(dcg_problem* p, const double* f, double* x, double tol, int max_it, dcg_stats* st, cudaStream_t s);
// launch wrappers of the outer iteration shared with the captured solve;
// stop: device flag that makes the direction kernels skip (may be null)
int solver_update(dcg_problem* p, double* x, double* r, const double* d, const double* q, int use_dr,
                  cudaStream_t s);
int solver_direction(dcg_problem* p, double* d, const double* r, int fcg, cudaStream_t s, const int* stop);
int solver_fcg_store(dcg_problem* p, cudaStream_t s);
int solver_fcg_direction(dcg_problem* p, cudaStream_t s, const int* stop, int K, int finish_grid);
int solver_reconstruct(dcg_problem* p, const double* xh, const double* z1, const double* zf, double* x,
                       cudaStream_t s);
int solver_axpy(dcg_problem* p, double* y, const double* x, cudaStream_t s);
// the whole solve as one CUDA graph with device-side loop control (graph.cu)
bool graph_solve_supported(const dcg_problem* p);
int graph_solve(dcg_problem* p, const double* f, double* x, double tol, int max_it, dcg_stats* st, cudaStream_t s);
int graph_solve_batched(int nprob, dcg_problem* const* probs, int nrhs, const double* const* f, double* const* x,
                        double tol, int max_it, dcg_stats* stats, cudaStream_t s);
void graph_free(dcg_problem* p);
int read_scalars(dcg_problem* p, cudaStream_t s);

// multigrid
int mg_setup(dcg_problem* p, cudaStream_t s);
int mg_rebuild_graph(dcg_problem* p);
void mg_free(dcg_problem* p);
int mg_inner_apply(dcg_problem* p, const double* z, double* y, cudaStream_t s);
int mg_cycles(dcg_problem* p, const double* g, double* z, int ncycles, cudaStream_t s);
int mg_solve(dcg_problem* p, const double* g, double* z, double tol, int nmax, int* ncyc, cudaStream_t s);
std::vector<int> level_sizes(int n, int max_levels);  // mesh sizes n_J, n_J/2, ... (finest first)
int mg_ras_step_hook(dcg_problem* p, int level, const double* f, double* z, cudaStream_t s);
// pieces of Algorithm 3 for the graph-captured solve (graph.cu)
int mg_graph_residual(dcg_problem* p, const double* g, const double* z, bool with_g, cudaStream_t s);
int mg_graph_wcycle(dcg_problem* p, cudaStream_t s);
int mg_graph_accumulate(dcg_problem* p, double* z, cudaStream_t s);
bool mg_exact(const dcg_problem* p);
int mg_coarse_hook(dcg_problem* p, const double* f, double* z, cudaStream_t s);

}  // namespace dcg
