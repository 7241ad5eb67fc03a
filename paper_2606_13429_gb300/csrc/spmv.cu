// FP64 BSR SpMV for the pseudo-stress operator, with the deflation
// embed/extract and the CG dot products fused into its prologue/epilogue.
//
// Mapping in 2D (4 x 4 blocks): a CTA owns 32 consecutive block rows; warp w
// computes scalar row R(w) of each of them (lane = block row). Every warp
// therefore executes one row pattern, so the structural zeros of the block
// (Section 3.1: the block is (1/dt) mt D_d + kron(I_d, G), 10 of 16 entries)
// are skipped without divergence. A lane reads the 4 contiguous doubles of
// its block row chunk (one 32-byte sector) and the 4 doubles of x at the
// column block. 3D (9 x 9 blocks, 33 of 81 entries nonzero): k_spmv3 below,
// one thread per structural nonzero.
//
// Variants (x operand / output):
//   x            : y = A x
//   x - V zh     : q = A (d - V zh)          (M_D of Algorithm 2, second product)
//   V zh         : y = A V zh                 (A pi(f) for f_D)
//   out = y / f - y / V^T y (only the d diagonal-component rows are computed:
//   g = V^T A x reads half (2D) or a third (3D) of the matrix).
#include "common.cuh"

namespace dcg {
namespace {

enum XMode { XM_X = 0, XM_X_MINUS_VZ = 1, XM_VZ = 2 };
enum OMode { OM_Y = 0, OM_FMY = 1, OM_VT = 2, OM_YVT = 3 };

struct SpmvArgs {
  const int* row_ptr;
  const int* col_idx;
  const double* vals;
  long long n_nodes;
  const double* x;
  const double* zh;
  const double* f;
  double* y;
  double* g;           // V^T y for OM_YVT
  const double* dvec;  // dot(dvec, y) for OM_Y
  double isd;          // 1/sqrt(d)
  Reduce red;
};

template <int D, int XM>
__device__ __forceinline__ double xval(const SpmvArgs& A, long long c, int col) {
  constexpr int B = D * D;
  const bool diag = (col % (D + 1)) == 0;  // positions l*D+l
  if (XM == XM_X) return __ldg(A.x + c * B + col);
  if (XM == XM_VZ) return diag ? __dmul_rn(A.isd, __ldg(A.zh + c)) : 0.0;
  // XM_X_MINUS_VZ
  double v = __ldg(A.x + c * B + col);
  return diag ? __dsub_rn(v, __dmul_rn(A.isd, __ldg(A.zh + c))) : v;
}

// 2D: the 4 doubles of the row chunk and of the x block are 32-byte aligned
// and read with two 16-byte loads each; the block loop is unrolled so the
// loads of several blocks are in flight together.
template <int R, int XM>
__device__ __forceinline__ double row_sum_2d(const SpmvArgs& A, int j0, int j1) {
  constexpr int k = R / 2, i = R % 2;
  double acc = 0.0;
#pragma unroll 3
  for (int j = j0; j < j1; ++j) {
    const long long c = __ldg(A.col_idx + j);
    const double2* v2 = reinterpret_cast<const double2*>(A.vals + (long long)j * 16 + R * 4);
    const double2 va = __ldg(v2), vb = __ldg(v2 + 1);
    const double v[4] = {va.x, va.y, vb.x, vb.y};
    double xv[4];
    if (XM == XM_VZ) {
      const double zz = __dmul_rn(A.isd, __ldg(A.zh + c));
      xv[0] = zz; xv[1] = 0.0; xv[2] = 0.0; xv[3] = zz;
    } else {
      const double2* x2 = reinterpret_cast<const double2*>(A.x + c * 4);
      const double2 xa = __ldg(x2), xb = __ldg(x2 + 1);
      xv[0] = xa.x; xv[1] = xa.y; xv[2] = xb.x; xv[3] = xb.y;
      if (XM == XM_X_MINUS_VZ) {
        const double zz = __dmul_rn(A.isd, __ldg(A.zh + c));
        xv[0] = __dsub_rn(xv[0], zz);
        xv[3] = __dsub_rn(xv[3], zz);
      }
    }
    if (k == i) {
      acc = fma(v[0], xv[0], acc);
      acc = fma(v[3], xv[3], acc);
      acc = fma(v[k * 2 + (1 - k)], xv[k * 2 + (1 - k)], acc);
    } else {
      acc = fma(v[k * 2], xv[k * 2], acc);
      acc = fma(v[k * 2 + 1], xv[k * 2 + 1], acc);
    }
  }
  return acc;
}

template <int D, int XM>
__device__ __forceinline__ double row_dispatch(const SpmvArgs& A, int R, int j0, int j1) {
  static_assert(D == 2, "the 3D product is k_spmv3");
  switch (R) {
    case 0: return row_sum_2d<0, XM>(A, j0, j1);
    case 1: return row_sum_2d<1, XM>(A, j0, j1);
    case 2: return row_sum_2d<2, XM>(A, j0, j1);
    case 3: return row_sum_2d<3, XM>(A, j0, j1);
    default: return 0.0;
  }
}

template <int D, int XM, int OM, bool DOT>
__global__ void k_spmv(SpmvArgs A) {
  constexpr int B = D * D;
  constexpr int NW = (OM == OM_VT) ? D : B;
  __shared__ double s_rows[NW][32];
  static_assert(OM != OM_YVT || NW == B, "all rows");
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int R = (OM == OM_VT) ? w * D + w : w;
  double part[1] = {0.0};
  for (long long base = (long long)blockIdx.x * 32; base < A.n_nodes; base += (long long)gridDim.x * 32) {
    const long long a = base + lane;
    double acc = 0.0;
    if (a < A.n_nodes) {
      const int j0 = __ldg(A.row_ptr + a), j1 = __ldg(A.row_ptr + a + 1);
      acc = row_dispatch<D, XM>(A, R, j0, j1);
    }
    if (OM == OM_VT) {
      s_rows[w][lane] = acc;
      __syncthreads();
      if (w == 0 && a < A.n_nodes) {
        double s = s_rows[0][lane];
#pragma unroll
        for (int l = 1; l < D; ++l) s += s_rows[l][lane];
        const double g = s * A.isd;
        A.y[a] = g;
        if (DOT) part[0] = fma(g, g, part[0]);
      }
      __syncthreads();
    } else if (OM == OM_YVT) {
      // all rows of t = A x, and g = V^T t from the diagonal-component rows
      if (a < A.n_nodes) A.y[a * B + R] = acc;
      s_rows[w][lane] = acc;
      __syncthreads();
      if (w == 0 && a < A.n_nodes) {
        double s = s_rows[0][lane];
#pragma unroll
        for (int l = 1; l < D; ++l) s += s_rows[l * D + l][lane];
        const double g = s * A.isd;
        A.g[a] = g;
        if (DOT) part[0] = fma(g, g, part[0]);
      }
      __syncthreads();
    } else if (a < A.n_nodes) {
      const long long row = a * B + R;
      double out = acc;
      if (OM == OM_FMY) out = __dsub_rn(A.f[row], acc);
      A.y[row] = out;
      if (DOT) {
        if (OM == OM_FMY) part[0] = fma(out, out, part[0]);
        else part[0] = fma(A.dvec[row], out, part[0]);
      }
    }
  }
  if (DOT) grid_reduce<1>(part, A.red);
}


// 3D (9 x 9 blocks), entry-parallel: a CTA of 256 threads takes 7 block
// rows at a time; thread t < 231 owns the structural nonzero number t % 33
// (Section 3.1: 33 of the 81 entries of a block) of every block of block
// row t / 33 and walks that row's blocks. The 33 threads of a block row read
// their entries of each block's 648 contiguous bytes together, the 48
// structural zeros are neither read nor multiplied, and x[col * 9 + c] is
// shared by the threads of column c. A row's partial sums are added in
// shared memory in the order of its entries (deterministic).
__host__ __device__ constexpr bool nz3(int r, int c) {
  // row r = (k, i) = (r / 3, r % 3): diagonal rows (k == i) couple the
  // diagonal components l*3+l and the components k*3+q; the others only k*3+q
  return (r / 3 == r % 3) ? (c % 4 == 0 || c / 3 == r / 3) : (c / 3 == r / 3);
}
// the nonzeros r*9 + c in row-major order, and where each row starts (the
// lists are checked against nz3 at compile time)
#define DCG_NZ3_RC 0, 1, 2, 4, 8, 9, 10, 11, 18, 19, 20, 30, 31, 32, 36, 39, 40, 41, 44, 48, 49, 50, 60, 61, 62, \
                   69, 70, 71, 72, 76, 78, 79, 80
#define DCG_NZ3_ROW 0, 5, 8, 11, 14, 19, 22, 25, 28, 33
constexpr int kNz3 = 33, kRows3 = 7;
constexpr unsigned char kNz3Rc[kNz3] = {DCG_NZ3_RC};
constexpr unsigned char kNz3Row[10] = {DCG_NZ3_ROW};
constexpr bool nz3_tables_ok() {
  int e = 0;
  for (int r = 0; r < 9; ++r) {
    if (kNz3Row[r] != e) return false;
    for (int c = 0; c < 9; ++c)
      if (nz3(r, c)) {
        if (e >= kNz3 || kNz3Rc[e] != r * 9 + c) return false;
        ++e;
      }
  }
  return e == kNz3 && kNz3Row[9] == kNz3;
}
static_assert(nz3_tables_ok(), "3D block nonzero tables");
__constant__ unsigned char c_nz3_rc[kNz3] = {DCG_NZ3_RC};
__constant__ unsigned char c_nz3_row[10] = {DCG_NZ3_ROW};

template <int XM, int OM, bool DOT>
__global__ void __launch_bounds__(256) k_spmv3(SpmvArgs A) {
  constexpr int B = 9;
  __shared__ double s_part[kRows3][kNz3];
  __shared__ double s_out[kRows3][9];
  const int t = threadIdx.x;
  const int lb = t / kNz3, e = t - lb * kNz3;
  const int rc = t < kRows3 * kNz3 ? c_nz3_rc[e] : 0, r = rc / 9, c = rc - r * 9;
  const bool act = t < kRows3 * kNz3 && (OM != OM_VT || r % 4 == 0);
  double part[1] = {0.0};
  for (long long base = (long long)blockIdx.x * kRows3; base < A.n_nodes; base += (long long)gridDim.x * kRows3) {
    const long long a = base + lb;
    double acc = 0.0;
    if (act && a < A.n_nodes) {
      const int j0 = __ldg(A.row_ptr + a), j1 = __ldg(A.row_ptr + a + 1);
#pragma unroll 4
      for (int j = j0; j < j1; ++j) {
        const long long col = __ldg(A.col_idx + j);
        acc = fma(__ldg(A.vals + (long long)j * 81 + rc), xval<3, XM>(A, col, c), acc);
      }
    }
    if (t < kRows3 * kNz3) s_part[lb][e] = acc;
    __syncthreads();
    if (t < kRows3 * 9) {
      const int b2 = t / 9, r2 = t - b2 * 9;
      const long long a2 = base + b2;
      const int e0 = c_nz3_row[r2], e1 = c_nz3_row[r2 + 1];
      double sum = s_part[b2][e0];
      for (int k = e0 + 1; k < e1; ++k) sum += s_part[b2][k];
      if (a2 < A.n_nodes) {
        const long long row = a2 * B + r2;
        if (OM == OM_Y) {
          A.y[row] = sum;
          if (DOT) part[0] = fma(A.dvec[row], sum, part[0]);
        } else if (OM == OM_FMY) {
          const double out = __dsub_rn(A.f[row], sum);
          A.y[row] = out;
          if (DOT) part[0] = fma(out, out, part[0]);
        } else if (OM == OM_YVT) {
          A.y[row] = sum;
        }
      }
      s_out[b2][r2] = sum;
    }
    if (OM == OM_VT || OM == OM_YVT) {
      __syncthreads();
      if (t < kRows3 && base + t < A.n_nodes) {
        const double g = (s_out[t][0] + s_out[t][4] + s_out[t][8]) * A.isd;
        if (OM == OM_VT) A.y[base + t] = g;
        else A.g[base + t] = g;
        if (DOT) part[0] = fma(g, g, part[0]);
      }
    }
    __syncthreads();
  }
  if (DOT) grid_reduce<1>(part, A.red);
}

// w = x - V zh (node-major, the d diagonal components of each node shifted):
// formed once per node instead of once per stored block that reads it, which
// keeps the FP64 arithmetic of the deflated product at that of A x
template <int D>
__global__ void k_x_minus_vz(const double* __restrict__ x, const double* __restrict__ zh, double* __restrict__ w,
                             long long nn, double isd) {
  constexpr int B = D * D;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn * B;
       t += (long long)gridDim.x * blockDim.x) {
    const long long a = t / B;
    const int c = (int)(t - a * B);
    const double v = x[t];
    w[t] = (c % (D + 1) == 0) ? __dsub_rn(v, __dmul_rn(isd, __ldg(zh + a))) : v;
  }
}

template <int XM, int OM, bool DOT>
int launch(dcg_problem* p, SpmvArgs a, cudaStream_t s, bool lowp = false) {
  if (p->matrix_free) return mf_product(p, XM, OM, DOT, lowp, a.x, a.zh, a.f, a.y, a.dvec, a.red, s);
  a.row_ptr = p->row_ptr;
  a.col_idx = p->col_idx;
  a.vals = p->vals;
  a.n_nodes = p->n_nodes;
  a.isd = 1.0 / sqrt((double)p->dim);
  const int grid = grid_for(p->n_nodes, 32, DOT ? 2 * kRedGrid : kMaxRedCtas);
  // algorithmic work: structural FMAs and the bytes the product must move
  const int D = p->dim, B = D * D;
  const double nnzb = (double)p->nnzb, nn = (double)p->n_nodes, N = (double)p->N;
  const int rows_read = (OM == OM_VT) ? D : B;  // OM_YVT reads all rows
  const double fma_blk = (OM == OM_VT) ? D * (2 * D - 1) : (D == 2 ? 10 : 33);
  double bytes = nnzb * (rows_read * B * 8.0 + 4.0) + (nn + 1) * 4.0;
  bytes += (XM == XM_VZ) ? nn * 8.0 : N * 8.0;          // operand
  if (XM == XM_X_MINUS_VZ) bytes += nn * 8.0;           // zh
  bytes += (OM == OM_VT) ? nn * 8.0 : N * 8.0;          // output
  if (OM == OM_YVT) bytes += nn * 8.0;                  // g
  if (OM == OM_FMY) bytes += N * 8.0;                   // f
  const int prof = prof_begin(p, PC_SPMV, s);
  if (p->dim == 2) {
    const int threads = 32 * (OM == OM_VT ? 2 : 4);
    k_spmv<2, XM, OM, DOT><<<grid, threads, 0, s>>>(a);
  } else {
    const int grid3 = grid_for((p->n_nodes + kRows3 - 1) / kRows3, 1, DOT ? 2 * kRedGrid : kMaxRedCtas);
    k_spmv3<XM, OM, DOT><<<grid3, 256, 0, s>>>(a);
  }
  DCG_LAUNCH_CHECK();
  prof_end(p, prof, s, 2.0 * fma_blk * nnzb, bytes);
  return DCG_OK;
}

}  // namespace

int spmv_plain(dcg_problem* p, const double* x, double* y, cudaStream_t s, bool lowp) {
  SpmvArgs a{};
  a.x = x;
  a.y = y;
  return launch<XM_X, OM_Y, false>(p, a, s, lowp);
}

int spmv_dot(dcg_problem* p, const double* x, double* y, const double* dv, int slot, cudaStream_t s) {
  SpmvArgs a{};
  a.x = x;
  a.y = y;
  a.dvec = dv;
  a.red = make_reduce(p, slot);
  if (!dv) return launch<XM_X, OM_Y, false>(p, a, s);
  return launch<XM_X, OM_Y, true>(p, a, s);
}

int spmv_residual(dcg_problem* p, const double* f, const double* x, double* y, int slot, cudaStream_t s) {
  SpmvArgs a{};
  a.x = x;
  a.f = f;
  a.y = y;
  a.red = make_reduce(p, slot);
  return launch<XM_X, OM_FMY, true>(p, a, s);
}

int spmv_vt(dcg_problem* p, const double* x, double* g, int slot, cudaStream_t s, bool lowp) {
  SpmvArgs a{};
  a.x = x;
  a.y = g;
  a.red = make_reduce(p, slot);
  return launch<XM_X, OM_VT, true>(p, a, s, lowp);
}

int spmv_defl(dcg_problem* p, const double* x, const double* zh, double* q, int slot, cudaStream_t s, bool lowp) {
  SpmvArgs a{};
  a.x = x;
  a.zh = zh;
  a.y = q;
  a.dvec = x;
  a.red = make_reduce(p, slot);
  if (!x) return launch<XM_VZ, OM_Y, false>(p, a, s, lowp);
  if (!zh) return launch<XM_X, OM_Y, true>(p, a, s, lowp);
  if (!p->matrix_free && p->sb.w) {
    const double isd = 1.0 / std::sqrt((double)p->dim);
    const int g = grid_for(p->N, 256, 8192);
    const int prof = prof_begin(p, PC_VEC, s);
    if (p->dim == 2) k_x_minus_vz<2><<<g, 256, 0, s>>>(x, zh, p->sb.w, p->n_nodes, isd);
    else k_x_minus_vz<3><<<g, 256, 0, s>>>(x, zh, p->sb.w, p->n_nodes, isd);
    DCG_LAUNCH_CHECK();
    prof_end(p, prof, s, 2.0 * p->n_nodes * p->dim, 8.0 * (2.0 * p->N + p->n_nodes));
    a.x = p->sb.w;  // dvec stays x: the fused dot is (x, A w)
    return launch<XM_X, OM_Y, true>(p, a, s, lowp);
  }
  return launch<XM_X_MINUS_VZ, OM_Y, true>(p, a, s, lowp);
}

int spmv_y_vt(dcg_problem* p, const double* x, double* t, double* g, int slot, cudaStream_t s) {
  if (p->dim == 2) {
    // 2D: the plain product (which streams the matrix at the rate of the
    // lane-per-block-row layout) and the extraction g = V^T t as a separate
    // pass over t: cheaper than the in-kernel exchange between the warps of
    // the diagonal-component rows
    SpmvArgs a{};
    a.x = x;
    a.y = t;
    DCG_TRY((launch<XM_X, OM_Y, false>(p, a, s)));
    const int prof = prof_begin(p, PC_VEC, s);
    DCG_TRY(vec_extract(p, t, g, slot, s));
    prof_end(p, prof, s, 2.0 * p->n_nodes * p->dim, 8.0 * (2.0 * p->n_nodes + p->n_nodes));
    return DCG_OK;
  }
  SpmvArgs a{};
  a.x = x;
  a.y = t;
  a.g = g;
  a.red = make_reduce(p, slot);
  return launch<XM_X, OM_YVT, true>(p, a, s);
}

// Divergence part of the element blocks summed over elements: for the uniform
// Q1 mesh a constant 3^d-point stencil per component pair (p, q),
//   G[p][q][o] = sum over the elements holding a and a+o of int d_p phi_a d_q phi_{a+o},
// each element integral a product of 1D factors (mass h/3 | h/6, stiffness
// +-1/h, mixed +-1/2). Offsets o = ox + 3 oy (+ 9 oz in 3D), each shifted by
// +1; entries for p, q >= d or o >= 3^d are zero.
void div_stencil(int d, int n, double (*gs)[27]) {
  const double h = 1.0 / n;
  for (int o = 0; o < 27; ++o) {
    const int off[3] = {o % 3 - 1, (o / 3) % 3 - 1, d == 3 ? o / 9 - 1 : 0};
    for (int p = 0; p < 3; ++p)
      for (int q = 0; q < 3; ++q) {
        double sum = 0.0;
        const bool used = p < d && q < d && (d == 3 || o < 9);
        for (int sb = 0; used && sb < (1 << d); ++sb) {
          double v = 1.0;
          bool ok = true;
          for (int ax = 0; ax < d && ok; ++ax) {
            const int la = ((sb >> ax) & 1) == 0 ? 1 : 0, lb = la + off[ax];
            if (lb < 0 || lb > 1) {
              ok = false;
              break;
            }
            double f;
            if (ax == p && ax == q) f = la == lb ? 1.0 / h : -1.0 / h;
            else if (ax == p) f = la == 0 ? -0.5 : 0.5;
            else if (ax == q) f = lb == 0 ? -0.5 : 0.5;
            else f = la == lb ? h / 3.0 : h / 6.0;
            v *= f;
          }
          if (ok) sum += v;
        }
        gs[p * 3 + q][o] = sum;
      }
  }
}

namespace {

struct DivStencil {
  double c[9][27];
};

// q = t - A V zh for the assembled operator, with A V zh = K_div V zh (the
// mass part annihilates V exactly): component (k, p) of node a is
//   t - (1/sqrt d) sum_o G[p][k][o] zh[a+o].
// Also reduces (dv, q).
template <int D>
__global__ void k_q_from_t(const double* __restrict__ t, const double* __restrict__ zh, const double* __restrict__ dv,
                           double* __restrict__ q, DivStencil G, int m, long long nn, double isd, Reduce red) {
  constexpr int B = D * D, NO = D == 2 ? 9 : 27;
  double part[1] = {0.0};
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < nn; a += (long long)gridDim.x * blockDim.x) {
    int c[3];
    long long r = a;
    c[0] = (int)(r % m);
    r /= m;
    c[1] = (int)(r % m);
    c[2] = D > 2 ? (int)(r / m) : 0;
    double zn[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
      const int x = c[0] + ox, y = c[1] + oy, z = c[2] + oz;
      const bool in = x >= 0 && x < m && y >= 0 && y < m && (D == 2 || (z >= 0 && z < m));
      zn[o] = in ? __ldg(zh + x + (long long)m * (y + (long long)m * (D > 2 ? z : 0))) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
      for (int p = 0; p < D; ++p) {
        double acc = 0.0;
#pragma unroll
        for (int o = 0; o < NO; ++o) {
          const int off[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
          if (p != k && (off[p] == 0 || off[k] == 0)) continue;  // cross stencil vanishes there
          acc = fma(G.c[p * 3 + k][o], zn[o], acc);
        }
        const long long row = a * B + k * D + p;
        const double v = t[row] - isd * acc;
        q[row] = v;
        part[0] = fma(dv[row], v, part[0]);
      }
  }
  grid_reduce<1>(part, red);
}

// 2D: the same product in separable form. The stencils of div_stencil are
// products of 1D factors: G[x][x] = K1 (x) M1, G[y][y] = M1 (x) K1 and
// G[x][y] = G[y][x] = (+-1/2 first differences along both axes), h cancelling
// in 2D. With the row quantities of column x at row y'
//   u = z(x-1) + z(x+1),  kx = 2 z(x) - u,  mx = 4 z(x) + u,  cx = z(x+1) - z(x-1)
// the three distinct products at row y are
//   G_xx zh = (kx(y-1) + kx(y+1) + 4 kx(y)) / 6
//   G_yy zh = (2 mx(y) - mx(y-1) - mx(y+1)) / 6
//   G_xy zh = (cx(y-1) - cx(y+1)) / 4,
// computed with row quantities that slide along y: 17 FP64 operations per
// node (with the four updates and the dot product) instead of 34. A thread
// walks kQSeg rows of one column (consecutive threads, consecutive columns);
// the 1D grid holds column blocks x row segments for the grid reduction.
constexpr int kQSeg = 16, kQThreads = 128, kQU = 2;

__global__ void __launch_bounds__(kQThreads) k_q_from_t_2d(const double* __restrict__ t, const double* __restrict__ zh,
                                                           const double* __restrict__ dv, double* __restrict__ q,
                                                           int m, int gx, double isd, Reduce red) {
  double part[1] = {0.0};
  const int bx = blockIdx.x % gx, by = blockIdx.x / gx;
  const int x = bx * kQThreads + threadIdx.x;
  if (x < m) {
    auto rowq = [&](int y, double& kx, double& mx, double& cx) {
      kx = mx = cx = 0.0;
      if (y < 0 || y >= m) return;
      const double* r = zh + (long long)m * y;
      const double zc = __ldg(r + x);
      const double zl = x > 0 ? __ldg(r + x - 1) : 0.0;
      const double zr = x + 1 < m ? __ldg(r + x + 1) : 0.0;
      const double u = zl + zr;
      kx = fma(2.0, zc, -u);
      mx = fma(4.0, zc, u);
      cx = zr - zl;
    };
    const double axx = isd / 6.0, axy = isd / 4.0;
    const int y0 = by * kQSeg, y1 = min(y0 + kQSeg, m);
    double km, mm, cm, k0, m0, c0;
    rowq(y0 - 1, km, mm, cm);
    rowq(y0, k0, m0, c0);
    // kQU rows at a time: the row quantities of the next rows and the t, dv
    // entries of the current ones are loaded together
    for (int y = y0; y < y1; y += kQU) {
      double kp[kQU], mp[kQU], cp[kQU];
      double2 ta[kQU], tb[kQU], da[kQU], db[kQU];
#pragma unroll
      for (int u = 0; u < kQU; ++u) {
        rowq(y + u + 1, kp[u], mp[u], cp[u]);
        if (y + u < y1) {
          const long long a = x + (long long)m * (y + u);
          const double2* t2 = reinterpret_cast<const double2*>(t + 4 * a);
          const double2* d2 = reinterpret_cast<const double2*>(dv + 4 * a);
          ta[u] = __ldg(t2);
          tb[u] = __ldg(t2 + 1);
          da[u] = __ldg(d2);
          db[u] = __ldg(d2 + 1);
        }
      }
#pragma unroll
      for (int u = 0; u < kQU; ++u) {
        if (y + u < y1) {
          const double gxx = fma(4.0, k0, km + kp[u]);
          const double gyy = fma(2.0, m0, -(mm + mp[u]));
          const double gxy = cm - cp[u];
          const long long a = x + (long long)m * (y + u);
          // components (k, p) = xx, xy, yx, yy
          const double q0 = fma(-axx, gxx, ta[u].x), q1 = fma(-axy, gxy, ta[u].y);
          const double q2 = fma(-axy, gxy, tb[u].x), q3 = fma(-axx, gyy, tb[u].y);
          double2* o2 = reinterpret_cast<double2*>(q + 4 * a);
          o2[0] = make_double2(q0, q1);
          o2[1] = make_double2(q2, q3);
          part[0] = fma(da[u].x, q0, part[0]);
          part[0] = fma(da[u].y, q1, part[0]);
          part[0] = fma(db[u].x, q2, part[0]);
          part[0] = fma(db[u].y, q3, part[0]);
        }
        km = k0; mm = m0; cm = c0;
        k0 = kp[u]; m0 = mp[u]; c0 = cp[u];
      }
    }
  }
  grid_reduce<1>(part, red);
}

}  // namespace

int q_from_t(dcg_problem* p, const double* t, const double* zh, const double* dv, double* q, int slot,
             cudaStream_t s) {
  const double isd = 1.0 / std::sqrt((double)p->dim);
  const int prof = prof_begin(p, PC_VEC, s);
  const int gx = (p->m + kQThreads - 1) / kQThreads, gy = (p->m + kQSeg - 1) / kQSeg;
  if (p->dim == 2 && (long long)gx * gy <= kMaxRedCtas) {
    k_q_from_t_2d<<<gx * gy, kQThreads, 0, s>>>(t, zh, dv, q, p->m, gx, isd, make_reduce(p, slot));
  } else {
    DivStencil G;
    div_stencil(p->dim, p->n, G.c);
    const int g = grid_for(p->n_nodes, 256, kRedGrid);
    if (p->dim == 2) k_q_from_t<2><<<g, 256, 0, s>>>(t, zh, dv, q, G, p->m, p->n_nodes, isd, make_reduce(p, slot));
    else k_q_from_t<3><<<g, 256, 0, s>>>(t, zh, dv, q, G, p->m, p->n_nodes, isd, make_reduce(p, slot));
  }
  DCG_LAUNCH_CHECK();
  prof_end(p, prof, s, 2.0 * p->N * (p->dim == 2 ? 6.5 : 15.0), 8.0 * (3.0 * p->N + p->n_nodes));
  return DCG_OK;
}

int spmv_f_minus_avz(dcg_problem* p, const double* f, const double* zh, double* y, int slot, cudaStream_t s) {
  SpmvArgs a{};
  a.zh = zh;
  a.f = f;
  a.y = y;
  a.red = make_reduce(p, slot);
  return launch<XM_VZ, OM_FMY, true>(p, a, s);
}

}  // namespace dcg
