// Multigrid for the inner system Z_J z = g (Algorithms 3 and 4) on the device.
//
// Inner matrix: Z_J = V^T A V (Algorithm 2 setup). It is extracted from the
// assembled A on the device, row by row, and checked to be one constant 3^d
// stencil (Corollary 1: V^T A V = (1/d) sum_i B_ii, the Q1 Laplacian, with
// the dt- and nu-dependent mass part cancelling). Levels are therefore
// applied as constant stencils; coarse stencils come from the Galerkin
// product Z_{k-1} = P^T Z_k P evaluated on the stencil (Algorithm 2 setup
// loop; P = nodal bilinear/trilinear interpolation, the natural embedding
// of nested Q1 spaces, and R = P^T, the reading of Section 4.2's L2
// projection pair for nested spaces).
//
// Smoother (Section 4.2): RAS with boxes = core tiles of P nodes per axis
// extended by `overlap`, local matrices R_i Z_k R_i^T inverted once per box
// shape on the device (Gauss-Jordan, FP64), weights 1/multiplicity or 0/1 on
// the core. One step z <- z + sum_i R_i^T D_i Z_i^-1 R_i (f - Z_k z) is two
// kernels: (1) per batch of equal-shape boxes: residual on the box,
// multiplication by the shared inverse (a small dense GEMM), results to a
// patch-major buffer; (2) per node: weighted sum of the box results.
//
// Coarsest level (Algorithm 4, k = 1): exact solve by fast diagonalisation:
// Z_1 = (1/d) sum_i (x)_ax {K1 if ax = i else M1} with 1D Q1 matrices
// K1, M1 diagonalised by the orthonormal sine basis S. Transformed by S
// along every axis but the last, Z_1 falls apart into independent
// tridiagonal systems along the last axis, one per transformed line, so
// Z_1^-1 = (S (x) .. (x) S (x) I) T^-1 (S (x) .. (x) S (x) I): d - 1 passes of
// S, one pass of line solves, d - 1 passes of S. The coarse Galerkin stencil
// is checked against the closed form before use.
//
// W-cycle recursion (Algorithm 4) runs in the set-up precision (FP32 in
// mixed mode, FP64 otherwise) and is captured once into a CUDA graph. The
// driver (Algorithm 3) keeps z and the residual g - Z_J z in FP64 and applies
// each cycle as a correction: z <- z + W(g - Z_J z, 0), which equals
// W(g, z) for the affine W-cycle iteration.
#include "common.cuh"
#include "tma.cuh"

#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <map>

namespace dcg {
namespace {

constexpr int kKC = 32;       // K chunk of the inverse staged in shared memory
constexpr int kFdmBatch = 16; // boxes per work item of the fast-diagonalisation smoother
// boxes per work item of the tensor-core smoother: rows of the M = 128 MMA
// beyond them are zero; smaller items spread a level over more SMs
constexpr int kTcBatch = 64;
constexpr int kFdmThreads = 192;
constexpr int kRasThreads = 256;
constexpr int kMaxNp = 256;   // largest box (nodes) supported

// ---------------------------------------------------------------------------
// Setup kernels
// ---------------------------------------------------------------------------

__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
  // v >= 0: IEEE order equals unsigned integer order
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// rows[a*27 + off] = (V^T A V)[a, a+off]; ref node gets copied by the host.
template <int D>
__global__ void k_zj_rows(const int* __restrict__ row_ptr, const int* __restrict__ col_idx,
                          const double* __restrict__ vals, int m, long long nn, double inv_d,
                          double* __restrict__ rows, double* __restrict__ maxA) {
  constexpr int B = D * D;
  long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (a >= nn) return;
  double row[27];
#pragma unroll
  for (int k = 0; k < 27; ++k) row[k] = 0.0;
  int ca[3] = {(int)(a % m), (int)((a / m) % m), D > 2 ? (int)(a / ((long long)m * m)) : 0};
  double mx = 0.0;
  for (int j = row_ptr[a]; j < row_ptr[a + 1]; ++j) {
    const long long c = col_idx[j];
    int cc[3] = {(int)(c % m), (int)((c / m) % m), D > 2 ? (int)(c / ((long long)m * m)) : 0};
    int o = (cc[0] - ca[0] + 1) + 3 * (cc[1] - ca[1] + 1) + (D > 2 ? 9 * (cc[2] - ca[2] + 1) : 0);
    const double* blk = vals + (long long)j * B * B;
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int l = 0; l < D; ++l) {
        double v = blk[(i * D + i) * B + (l * D + l)];
        s += v;
        mx = fmax(mx, fabs(v));
      }
    row[o] = s * inv_d;
  }
  for (int k = 0; k < 27; ++k) rows[a * 27 + k] = row[k];
  atomic_max_pos(maxA, mx);
}

// max over nodes of |row(a) - ref| restricted to neighbours inside the grid
template <int D>
__global__ void k_zj_check(const double* __restrict__ rows, const double* __restrict__ ref, int m, long long nn,
                           double* __restrict__ maxdev) {
  long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (a >= nn) return;
  int ca[3] = {(int)(a % m), (int)((a / m) % m), D > 2 ? (int)(a / ((long long)m * m)) : 0};
  double dev = 0.0;
  for (int o = 0; o < (D == 2 ? 9 : 27); ++o) {
    int off[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
    bool in = true;
    for (int k = 0; k < D; ++k) in = in && (ca[k] + off[k] >= 0 && ca[k] + off[k] < m);
    double want = in ? ref[o] : 0.0;
    dev = fmax(dev, fabs(rows[a * 27 + o] - want));
  }
  atomic_max_pos(maxdev, dev);
}

// Galerkin product on a constant stencil: S_c(D) = sum_{al,be} w(al) w(be) S_f(2D + be - al)
template <int D>
__global__ void k_galerkin(const double* __restrict__ sf, double* __restrict__ sc) {
  int o = threadIdx.x;
  if (o >= (D == 2 ? 9 : 27)) return;
  int dl[3] = {o % 3 - 1, (o / 3) % 3 - 1, D > 2 ? o / 9 - 1 : 0};
  double s = 0.0;
  for (int ia = 0; ia < (D == 2 ? 9 : 27); ++ia) {
    int al[3] = {ia % 3 - 1, (ia / 3) % 3 - 1, D > 2 ? ia / 9 - 1 : 0};
    double wa = 1.0;
    for (int k = 0; k < D; ++k) wa *= al[k] ? 0.5 : 1.0;
    for (int ib = 0; ib < (D == 2 ? 9 : 27); ++ib) {
      int be[3] = {ib % 3 - 1, (ib / 3) % 3 - 1, D > 2 ? ib / 9 - 1 : 0};
      double wb = 1.0;
      int so[3];
      bool in = true;
      for (int k = 0; k < D; ++k) {
        wb *= be[k] ? 0.5 : 1.0;
        so[k] = 2 * dl[k] + be[k] - al[k];
        in = in && so[k] >= -1 && so[k] <= 1;
      }
      if (!in) continue;
      int si = (so[0] + 1) + 3 * (so[1] + 1) + (D > 2 ? 9 * (so[2] + 1) : 0);
      s += wa * wb * sf[si];
    }
  }
  sc[o] = s;
}

// Dense local matrix of a box (np nodes, x fastest) from the stencil.
template <int D>
__global__ void k_box_matrix(Stencil<double> st, int lx, int ly, int lz, double* __restrict__ M) {
  const int np = lx * ly * lz;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)np * np) return;
  int i = (int)(t / np), j = (int)(t % np);
  int ci[3] = {i % lx, (i / lx) % ly, i / (lx * ly)};
  int cj[3] = {j % lx, (j / lx) % ly, j / (lx * ly)};
  int off[3];
  bool near = true;
  for (int k = 0; k < 3; ++k) {
    off[k] = cj[k] - ci[k];
    near = near && off[k] >= -1 && off[k] <= 1;
  }
  double v = 0.0;
  if (near) v = st.c[(off[0] + 1) + 3 * (off[1] + 1) + (D > 2 ? 9 * (off[2] + 1) : 0)];
  M[t] = v;
}

// In-place Gauss-Jordan inversion of an SPD matrix (no pivoting), one CTA.
__global__ void k_gauss_jordan(double* __restrict__ a, int n) {
  extern __shared__ double fcol[];
  for (int k = 0; k < n; ++k) {
    const double piv = a[(long long)k * n + k];
    for (int i = threadIdx.x; i < n; i += blockDim.x) fcol[i] = a[(long long)i * n + k];
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x)
      a[(long long)k * n + j] = (j == k) ? 1.0 / piv : a[(long long)k * n + j] / piv;
    __syncthreads();
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
      int i = (int)(t / n), j = (int)(t % n);
      if (i == k) continue;
      const double f = fcol[i];
      if (j == k) a[t] = -f * a[(long long)k * n + k];
      else a[t] = a[t] - f * a[(long long)k * n + j];
    }
    __syncthreads();
  }
}

// symmetrised inverse in the cycle precision, rows padded to npp (zeros)
template <typename T>
__global__ void k_sym_convert(const double* __restrict__ a, T* __restrict__ out, int n, int npp) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n * npp) return;
  int i = (int)(t / npp), j = (int)(t % npp);
  out[t] = j < n ? (T)(0.5 * (a[(long long)i * n + j] + a[(long long)j * n + i])) : (T)0;
}

// sine basis S[i][j] = sqrt(2/(m+1)) sin((i+1)(j+1) pi/(m+1))
__global__ void k_fdm_setup(int m, double* __restrict__ S) {
  const int n1 = m + 1;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < (long long)m * m) {
    int i = (int)(t / m), j = (int)(t % m);
    long long ij = (long long)(i + 1) * (j + 1) % (2 * n1);
    S[t] = sqrt(2.0 / n1) * sin(M_PI * (double)ij / n1);
  }
}

// Line-solve factors of the coarsest solve along the last axis. With the
// sine indices j_k of a line on the other d - 1 axes (kappa_k = (2/h)(1 -
// cos th_k), mu_k = (h/3)(2 + cos th_k), th_k = pi (j_k + 1) / (m + 1): the
// eigenvalues of K1 and M1), Z_1 restricted to the transformed line is
//   T_j = a_j M1 + b_j K1,  a_j = (1/d) sum_i kappa_i prod_{k != i} mu_k,
//                           b_j = (1/d) prod_k mu_k,
// tridiagonal, symmetric and Toeplitz with diagonal a (2h/3) + b (2/h) and
// off-diagonal e = a h/6 - b/h, strictly diagonally dominant (a, b > 0).
// Tabulated per line: the elimination multipliers l_y = e / w_{y-1} (l_0 = 0)
// and the reciprocal pivots 1/w_y, w_y = diagonal - l_y e, both in the
// data's layout [y][j]; and e_j.
template <int D>
__global__ void k_tri_setup(int m, double* __restrict__ fl, double* __restrict__ fw, double* __restrict__ fe) {
  long long M1 = 1;
  for (int k = 0; k < D - 1; ++k) M1 *= m;
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= M1) return;
  const int n1 = m + 1;
  const double h = 1.0 / n1;
  double kap[3], mu[3];
  long long r = j;
  for (int k = 0; k < D - 1; ++k) {
    const int jk = (int)(r % m);
    r /= m;
    const double th = M_PI * (jk + 1) / n1;
    kap[k] = (2.0 / h) * (1.0 - cos(th));
    mu[k] = (h / 3.0) * (2.0 + cos(th));
  }
  double a = 0.0, b = 1.0;
  for (int i = 0; i < D - 1; ++i) {
    double t = kap[i];
    for (int k = 0; k < D - 1; ++k)
      if (k != i) t *= mu[k];
    a += t;
    b *= mu[i];
  }
  a /= D;
  b /= D;
  const double dg = a * (2.0 * h / 3.0) + b * (2.0 / h);
  const double e = a * (h / 6.0) - b / h;
  double w = dg;
  fl[j] = 0.0;
  fw[j] = 1.0 / w;
  for (int y = 1; y < m; ++y) {
    const double l = e / w;
    w = dg - l * e;
    fl[j + M1 * y] = l;
    fw[j + M1 * y] = 1.0 / w;
  }
  fe[j] = e;
}

// Cyclic-reduction coefficients of the same line systems when m = 2^q - 1
// (the FFT route). T_j is Toeplitz, tridiag(e, dg, e), with x_0 = x_{m+1} = 0;
// eliminating the odd unknowns leaves the even ones in a Toeplitz system of
// size 2^(q-1) - 1 with e' = -e^2/dg, dg' = dg - 2 e^2/dg, and so on down to
// one unknown. Tabulated per level k < q, layout [k][j]: beta_k = e_k / dg_k
// and gamma_k = 1 / dg_k.
template <int D>
__global__ void k_cr_setup(int m, int q, double* __restrict__ beta, double* __restrict__ gamma) {
  long long M1 = 1;
  for (int k = 0; k < D - 1; ++k) M1 *= m;
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= M1) return;
  const int n1 = m + 1;
  const double h = 1.0 / n1;
  double kap[3], mu[3];
  long long r = j;
  for (int k = 0; k < D - 1; ++k) {
    const int jk = (int)(r % m);
    r /= m;
    const double th = M_PI * (jk + 1) / n1;
    kap[k] = (2.0 / h) * (1.0 - cos(th));
    mu[k] = (h / 3.0) * (2.0 + cos(th));
  }
  double a = 0.0, b = 1.0;
  for (int i = 0; i < D - 1; ++i) {
    double t = kap[i];
    for (int k = 0; k < D - 1; ++k)
      if (k != i) t *= mu[k];
    a += t;
    b *= mu[i];
  }
  a /= D;
  b /= D;
  double dg = a * (2.0 * h / 3.0) + b * (2.0 / h);
  double e = a * (h / 6.0) - b / h;
  for (int k = 0; k < q; ++k) {
    const double bk = e / dg;
    beta[k * M1 + j] = bk;
    gamma[k * M1 + j] = 1.0 / dg;
    const double e2 = e * bk;  // e^2 / dg
    dg = dg - 2.0 * e2;
    e = -e2;
  }
}

template <typename T>
__global__ void k_to_t(const double* __restrict__ a, T* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (T)a[i];
}

// ---------------------------------------------------------------------------
// W-cycle kernels
// ---------------------------------------------------------------------------

template <int D>
__device__ __forceinline__ void coords_of(long long a, int m, int (&c)[3]) {
  // node counts stay below 2^31: 32-bit unsigned division (64-bit division
  // is emulated and costs about a hundred instructions)
  const unsigned ua = (unsigned)a, um = (unsigned)m;
  const unsigned q = ua / um;
  c[0] = (int)(ua - q * um);
  if (D > 2) {
    const unsigned q2 = q / um;
    c[1] = (int)(q - q2 * um);
    c[2] = (int)q2;
  } else {
    c[1] = (int)q;
    c[2] = 0;
  }
}

template <typename T, int D>
__device__ __forceinline__ T stencil_apply(const Stencil<T>& st, const T* __restrict__ z, int m, const int (&c)[3]) {
  T acc = 0;
  const long long mm = (long long)m * m;
#pragma unroll
  for (int dz = (D > 2 ? -1 : 0); dz <= (D > 2 ? 1 : 0); ++dz) {
    const int zc = c[2] + dz;
    if (D > 2 && (zc < 0 || zc >= m)) continue;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int yc = c[1] + dy;
      if (yc < 0 || yc >= m) continue;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int xc = c[0] + dx;
        if (xc < 0 || xc >= m) continue;
        const T w = st.c[(dx + 1) + 3 * (dy + 1) + (D > 2 ? 9 * (dz + 1) : 0)];
        acc += w * __ldg(z + xc + (long long)m * yc + (D > 2 ? mm * zc : 0));
      }
    }
  }
  return acc;
}

// y = f - Z z
template <typename T, int D>
__global__ void k_apply(Stencil<T> st, const T* __restrict__ z, T* __restrict__ y, int m, long long nn) {
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < nn; a += (long long)gridDim.x * blockDim.x) {
    int c[3];
    coords_of<D>(a, m, c);
    y[a] = stencil_apply<T, D>(st, z, m, c);
  }
}

template <typename T, int D>
__global__ void k_residual(Stencil<T> st, const T* __restrict__ f, const T* __restrict__ z, T* __restrict__ y, int m,
                           long long nn) {
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < nn; a += (long long)gridDim.x * blockDim.x) {
    int c[3];
    coords_of<D>(a, m, c);
    y[a] = f[a] - stencil_apply<T, D>(st, z, m, c);
  }
}

// 2D levels whose 8 neighbour coefficients are equal (the Q1 Laplacian):
//   (Z z)_a = c1 (sum of the 3 x 3 box around a) + (c_centre - c1) z_a,
// with the box sum formed from row sums s(y) = z(x-1,y) + z(x,y) + z(x+1,y)
// that slide along y: a residual takes 4 additions and 2 FMAs per node
// instead of 9 FMAs and a subtraction (FP64 issue is what the FP64 cycle
// spends). A thread walks kBoxSeg rows of one column; consecutive threads
// take consecutive columns, so every row access is coalesced. Entries
// outside the grid are zero (Dirichlet nodes eliminated).
constexpr int kBoxSeg = 8;
constexpr int kBoxThreads = 128;

template <typename T>
__device__ __forceinline__ T box_row(const T* __restrict__ z, int x, int y, int m, T& centre) {
  centre = (T)0;
  if (y < 0 || y >= m) return (T)0;
  const T* row = z + (long long)m * y;
  centre = __ldg(row + x);
  T s = centre;
  if (x > 0) s = __ldg(row + x - 1) + s;
  if (x + 1 < m) s = s + __ldg(row + x + 1);
  return s;
}

// Walks rows y0 .. y0 + kBoxSeg - 1 of column x and calls
// body(a, r_a) with r_a = f_a - (Z z)_a. Rows are loaded kBoxU at a time
// (all their loads in flight together) before the sums slide over them.
constexpr int kBoxU = 4;
template <typename T, typename F, typename Body>
__device__ __forceinline__ void box_residual_walk(T c0, T c1, const F* __restrict__ f, const T* __restrict__ z, int m,
                                                  int x, int y0, Body&& body) {
  const int y1 = min(y0 + kBoxSeg, m);
  T cm, c0v;
  T sm = box_row(z, x, y0 - 1, m, cm);
  T s0 = box_row(z, x, y0, m, c0v);
  for (int y = y0; y < y1; y += kBoxU) {
    T sp[kBoxU], cp[kBoxU], fv[kBoxU];
#pragma unroll
    for (int u = 0; u < kBoxU; ++u) {
      sp[u] = box_row(z, x, y + u + 1, m, cp[u]);
      fv[u] = y + u < y1 ? (T)__ldg(f + x + (long long)m * (y + u)) : (T)0;
    }
#pragma unroll
    for (int u = 0; u < kBoxU; ++u) {
      if (y + u < y1) {
        const T box = (sm + s0) + sp[u];
        body(x + (long long)m * (y + u), fma(-c1, box, fma(-c0, c0v, fv[u])));
      }
      sm = s0;
      s0 = sp[u];
      c0v = cp[u];
    }
  }
}

// y = f - Z z on a box-sum level (grid: columns / kBoxThreads x rows / kBoxSeg)
template <typename T>
__global__ void __launch_bounds__(kBoxThreads) k_residual_box(T c0, T c1, const T* __restrict__ f,
                                                              const T* __restrict__ z, T* __restrict__ y, int m) {
  const int x = blockIdx.x * kBoxThreads + threadIdx.x;
  if (x >= m) return;
  box_residual_walk<T, T>(c0, c1, f, z, m, x, blockIdx.y * kBoxSeg, [&](long long a, T r) { y[a] = r; });
}

// coarse[I] = sum_al w(al) fine[2I+1+al]  (P^T), weights 1, 1/2, 1/4, 1/8:
// per axis the line is folded as f[c] + (f[c-1] + f[c+1]) / 2 (exact
// scalings by powers of two), which takes 2 operations per axis instead of
// 3 multiply-adds (every fine index 2I+1+al lies inside the fine grid)
template <typename T, int D>
__global__ void k_restrict(const T* __restrict__ fine, T* __restrict__ coarse, int mf, int mc, long long nc) {
  const long long sy = mf, sz = (long long)mf * mf;
  for (long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x; I < nc; I += (long long)gridDim.x * blockDim.x) {
    int c[3];
    coords_of<D>(I, mc, c);
    const long long base = (2 * c[0] + 1) + sy * (2 * c[1] + 1) + (D > 2 ? sz * (2 * c[2] + 1) : 0);
    T plane[3];
#pragma unroll
    for (int az = 0; az < (D > 2 ? 3 : 1); ++az) {
      T row[3];
#pragma unroll
      for (int ay = 0; ay < 3; ++ay) {
        const T* f = fine + base + (ay - 1) * sy + (D > 2 ? (az - 1) * sz : 0);
        row[ay] = fma((T)0.5, f[-1] + f[1], f[0]);
      }
      plane[az] = fma((T)0.5, row[0] + row[2], row[1]);
    }
    coarse[I] = D > 2 ? fma((T)0.5, plane[0] + plane[2], plane[1]) : plane[0];
  }
}

// The same prolongation in 2D with one thread per pair of fine columns
// (x = 2i, 2i + 1) of one fine row: both take coarse column i (the odd one
// alone, the even one with column i - 1), so the pair shares its coarse
// loads and no lane of a warp takes a different branch. Row y odd: coarse
// row (y-1)/2; y even: rows y/2-1 and y/2 summed (weight 1/2). About 2 FP64
// operations per fine node instead of 5.
template <typename T>
__global__ void k_prolong_add_2d(const T* __restrict__ coarse, T* __restrict__ fine, int mf, int mc) {
  const int npair = (mf + 1) >> 1;  // fine columns 0..mf-1 = 2 mc: pairs 0..mc
  const long long total = (long long)npair * mf;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(t / npair), i = (int)(t - (long long)y * npair);
    // coarse rows of fine row y: r1 (always), r2 (even y only)
    const bool ev = (y & 1) == 0;
    const int r1 = ev ? (y >> 1) - 1 : (y - 1) >> 1, r2 = y >> 1;
    auto cval = [&](int r, int c) -> T {
      return (r >= 0 && r < mc && c >= 0 && c < mc) ? __ldg(coarse + (long long)r * mc + c) : (T)0;
    };
    T a = cval(r1, i - 1), b = cval(r1, i);
    if (ev) {
      a += cval(r2, i - 1);
      b += cval(r2, i);
    }
    const T wr = ev ? (T)0.5 : (T)1;  // row weight
    T* row = fine + (long long)y * mf;
    const int x0 = 2 * i;
    row[x0] = fma((T)0.5 * wr, a + b, row[x0]);  // even column: (a + b) / 2
    if (x0 + 1 < mf) row[x0 + 1] = fma(wr, b, row[x0 + 1]);
  }
}

// fine[a] += sum_I P[a][I] coarse[I]: per axis an odd fine index sits on coarse
// node (c-1)/2 (weight 1), an even one between c/2-1 and c/2 (weight 1/2
// each, a missing boundary neighbour contributing 0); the coarse values are
// summed first and scaled once by 2^-(number of even axes), exactly
template <typename T, int D>
__global__ void k_prolong_add(const T* __restrict__ coarse, T* __restrict__ fine, int mf, int mc, long long nf) {
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < nf; a += (long long)gridDim.x * blockDim.x) {
    int c[3];
    coords_of<D>(a, mf, c);
    int lo[3], cnt[3];
    int halves = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (k >= D) { lo[k] = 0; cnt[k] = 1; continue; }
      if (c[k] & 1) { lo[k] = (c[k] - 1) >> 1; cnt[k] = 1; }
      else { lo[k] = (c[k] >> 1) - 1; cnt[k] = 2; ++halves; }
    }
    T acc = 0;
    for (int iz = 0; iz < cnt[2]; ++iz)
      for (int iy = 0; iy < cnt[1]; ++iy)
        for (int ix = 0; ix < cnt[0]; ++ix) {
          const int X = lo[0] + ix, Y = lo[1] + iy, Z = lo[2] + iz;
          if (X < 0 || X >= mc || Y < 0 || Y >= mc || (D > 2 && (Z < 0 || Z >= mc))) continue;
          acc += coarse[X + (long long)mc * Y + (long long)mc * mc * Z];
        }
    const T scale = halves == 0 ? (T)1 : halves == 1 ? (T)0.5 : halves == 2 ? (T)0.25 : (T)0.125;
    fine[a] = fma(scale, acc, fine[a]);
  }
}

struct RasArgs {
  int m;
  const int* work;           // [nwork*3]: class, first index into class_patches, count
  const int* class_patches;  // patch ids grouped by class
  const RasClass* classes;
  const int4* origin;        // [npatch] box origin (x, y, z) and its node index
  const int2* core;          // [npatch] core tile in box-local coordinates, packed 10 bits per axis (lo, hi)
  const int* local;          // per class: packed local coordinates, 10 bits per axis
  const int* local_off_node; // per class: node offset of each local node from the box origin node
  const long long* item_off; // [nwork] offset of each work item's results in y
  const int4* axis_tab;      // [m] per coordinate: (t0, l0, t1, l1), t1 = -1 when one box only
  int nwork;
  int items_per_cta;
  long long g_off;           // elements of shared memory before the residual tile
  double* err;               // device error slot (set to 1 when a bounded wait gives up)
};

// Box results are stored node-major: y[node * SL + slot], SL = 2^D, where bit
// `ax` of `slot` says whether the box is the node's own core tile along axis
// ax (0) or the neighbouring tile whose overlap reaches the node (1); with
// 2*overlap <= patch a node lies in at most two boxes per axis.
template <int D>
constexpr int slots_per_node() { return 1 << D; }

// (1) residual on each box of a batch, times the shared inverse, to y.
// A CTA walks a contiguous range of work items (sorted by class); when
// RESIDENT, the class inverse is brought into shared memory with one bulk
// asynchronous copy while the residuals are gathered, and kept while the
// class does not change. GEMM Y[np x nb] = inv[np x np] G[np x nb]: thread
// (ty, tx) owns rows 4ty..4ty+3 and boxes 8tx..8tx+7 (16-byte shared loads);
// the class's batch width nb_c = 8 * bg with bg * ceil(np/4) <= threads.
template <typename T>
struct Vec4 { using type = float4; };
template <>
struct Vec4<double> { using type = double4; };

template <typename T>
__device__ __forceinline__ void lds4(const T* p, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
}

template <typename T, int D, bool RESIDENT>
__global__ void __launch_bounds__(kRasThreads) k_ras_solve(RasArgs ra, const T* __restrict__ rvec,
                                                            const T* __restrict__ inv, T* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  const int tid = threadIdx.x;
  const int w0 = blockIdx.x * ra.items_per_cta;
  const int w1 = min(ra.nwork, w0 + ra.items_per_cta);
  if (RESIDENT) {
    if (tid == 0) mbar_init(&bar, 1);
    __syncthreads();
  }
  unsigned phase = 0;
  int cur_cls = -1;
  for (int w = w0; w < w1; ++w) {
    const int cls = ra.work[3 * w], first = ra.work[3 * w + 1], nb = ra.work[3 * w + 2];
    const RasClass C = ra.classes[cls];
    const int np = C.np;
    const int npp = C.npp;                                  // padded row length of the inverse (multiple of 4)
    const int NB = C.nb;                                    // batch width of the class (power of 2, <= 256)
    const int bg = NB >> 3;                                 // box groups of 8
    const int rg = (np + 3) >> 2;                           // row groups of 4
    T* As = reinterpret_cast<T*>(smem_raw);                 // RESIDENT: [np][npp], else [kKC][npp]
    T* G = As + ra.g_off;                                   // [np][NB]
    __syncthreads();
    bool loading = false;
    if (RESIDENT && cls != cur_cls) {
      if (tid == 0) {
        const unsigned bytes = (unsigned)((size_t)np * npp * sizeof(T));  // multiple of 16
        mbar_expect_tx(&bar, bytes);
        tma_load_1d(As, inv + C.inv_off, bytes, &bar);
      }
      loading = true;
      cur_cls = cls;
    }
    // gather the residual (computed once per node beforehand) on the boxes:
    // thread keeps box b = tid % NB; one load per box node
    {
      const int b = tid & (NB - 1);
      const int kstep = kRasThreads / NB;
      int node0 = 0;
      if (b < nb) node0 = __ldg(ra.origin + __ldg(ra.class_patches + first + b)).w;
#pragma unroll 8
      for (int k = tid / NB; k < np; k += kstep) {
        T r = 0;
        if (b < nb) r = __ldg(rvec + node0 + __ldg(ra.local_off_node + C.local_off + k));
        G[(size_t)k * NB + b] = r;
      }
    }
    bool ok = true;
    if (loading) {
      ok = mbar_wait_bounded(&bar, phase) || mbar_wait_bounded(&bar, phase);
      phase ^= 1u;
    }
    const int tx = tid % bg, ty = tid / bg;
    const bool active = ty < rg;
    T acc[4][8];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[r][c] = 0;
    if (RESIDENT) {
      if (__syncthreads_or(!ok)) {  // uniform decision after the barrier
        if (tid == 0) *ra.err = 1.0;
        return;
      }
      if (active) {
        const T* gcol = G + 8 * tx;
        const T* acol = As + 4 * ty;
#pragma unroll 2
        for (int kk = 0; kk < np; ++kk) {
          T av[4], g0[4], g1[4];
          lds4(acol + (size_t)kk * npp, av);
          lds4(gcol + (size_t)kk * NB, g0);
          lds4(gcol + (size_t)kk * NB + 4, g1);
#pragma unroll
          for (int r = 0; r < 4; ++r) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              acc[r][c] = fma(av[r], g0[c], acc[r][c]);
              acc[r][c + 4] = fma(av[r], g1[c], acc[r][c + 4]);
            }
          }
        }
      }
    } else {
      const T* invc = inv + C.inv_off;
      for (int k0 = 0; k0 < np; k0 += kKC) {
        const int kc = min(kKC, np - k0);
        __syncthreads();
#pragma unroll 8
        for (int idx = tid; idx < kc * npp; idx += blockDim.x) As[idx] = __ldg(invc + (size_t)k0 * npp + idx);
        __syncthreads();
        if (active) {
          const T* gcol = G + 8 * tx;
          for (int kk = 0; kk < kc; ++kk) {
            T av[4], g0[4], g1[4];
            lds4(As + (size_t)kk * npp + 4 * ty, av);
            lds4(gcol + (size_t)(k0 + kk) * NB, g0);
            lds4(gcol + (size_t)(k0 + kk) * NB + 4, g1);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                acc[r][c] = fma(av[r], g0[c], acc[r][c]);
                acc[r][c + 4] = fma(av[r], g1[c], acc[r][c + 4]);
              }
            }
          }
        }
      }
    }
    // epilogue: results in the work item's layout y[item][i][NB] (8
    // consecutive boxes per thread row: two 16-byte stores)
    if (active) {
      T* yi = y + ra.item_off[w];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = 4 * ty + r;
        if (i < np) {
          T* dst = yi + (size_t)i * NB + 8 * tx;
          if constexpr (sizeof(T) == 4) {
            reinterpret_cast<float4*>(dst)[0] = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
            reinterpret_cast<float4*>(dst)[1] = make_float4(acc[r][4], acc[r][5], acc[r][6], acc[r][7]);
          } else {
#pragma unroll
            for (int c = 0; c < 8; c += 2)
              reinterpret_cast<double2*>(dst)[c / 2] = make_double2(acc[r][c], acc[r][c + 1]);
          }
        }
      }
    }
  }
}

// (1') Tensor-core variant (tcgen05, kind::f16): per work item of kTcBatch
// boxes (rows up to 128 of the M = 128 MMA, the rest zero),
// D[128 x npad] = G^T[128 x npad] * inv^T with BF16 operands and
// FP32 accumulation in TMEM (the inverse is symmetric, so inv^T = inv). The
// class inverse is stored at setup in the canonical K-major BF16 layout and
// brought into shared memory with one bulk copy; the residual tile is
// gathered, rounded to BF16 and written in the same layout; one thread issues
// npad/16 MMAs (M=128, N=npad, K=16) and commits them to an mbarrier; the
// epilogue reads TMEM with tcgen05.ld (warp w: lanes 32(w%4).., half of the
// columns) and stores results coalesced in the work item's entry-major
// layout [i][nb] (a box-major layout, 32-byte runs per lane, measured slower).
template <int D>
__global__ void __launch_bounds__(256) k_ras_solve_tc(RasArgs ra, const float* __restrict__ rvec,
                                                       const __nv_bfloat16* __restrict__ invb, float* __restrict__ y) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar_tma;
  __shared__ __align__(8) uint64_t bar_mma;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    mbar_init(&bar_tma, 1);
    mbar_init(&bar_mma, 1);
  }
  if (warp == 0) tmem_alloc(&tmem_base, 256);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  unsigned ph_tma = 0, ph_mma = 0;
  int cur_cls = -1;
  bool failed = false;
  const int w0 = blockIdx.x * ra.items_per_cta;
  const int w1 = min(ra.nwork, w0 + ra.items_per_cta);
  __nv_bfloat16* sB = reinterpret_cast<__nv_bfloat16*>(smem_raw);  // inverse [npad][npad], canonical
  __nv_bfloat16* sA = sB + ra.g_off;                                  // residuals [128][npad], canonical
  for (int w = w0; w < w1; ++w) {
    const int cls = ra.work[3 * w], first = ra.work[3 * w + 1], nb = ra.work[3 * w + 2];
    const RasClass C = ra.classes[cls];
    const int np = C.np, npad = C.npk;
    __syncthreads();  // the previous item is done with sA and with TMEM
    bool loading = false;
    if (cls != cur_cls) {
      if (tid == 0) {
        const unsigned bytes = (unsigned)((size_t)npad * npad * sizeof(__nv_bfloat16));
        mbar_expect_tx(&bar_tma, bytes);
        tma_load_1d(sB, invb + C.inv_off, bytes, &bar_tma);
      }
      loading = true;
      cur_cls = cls;
    }
    {
      // thread keeps box b = tid % 128 (rows >= nb are zero) and walks the
      // entries k = tid / 128, + 2, ...
      const int b = tid & 127;
      int node0 = 0;
      if (b < nb) node0 = __ldg(ra.origin + __ldg(ra.class_patches + first + b)).w;
#pragma unroll 8
      for (int k = tid >> 7; k < npad; k += 2) {
        float r = 0.f;
        if (b < nb && k < np) r = __ldg(rvec + node0 + __ldg(ra.local_off_node + C.local_off + k));
        sA[canon_bf16(b, k, npad)] = __float2bfloat16_rn(r);
      }
    }
    fence_async_smem();
    bool ok = true;
    if (loading) {
      ok = mbar_wait_bounded(&bar_tma, ph_tma) || mbar_wait_bounded(&bar_tma, ph_tma);
      ph_tma ^= 1u;
    }
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc_fence_after();
    if (tid == 0) {
      const uint32_t idesc = umma_idesc_bf16(128, npad);
      const unsigned sbo = (unsigned)(npad / 8) * 128u;
      const unsigned a0 = smem_u32(sA), b0 = smem_u32(sB);
      for (int k0 = 0; k0 < npad; k0 += 16) {
        const uint64_t adesc = umma_smem_desc(a0 + (unsigned)(k0 / 8) * 128u, 128u, sbo);
        const uint64_t bdesc = umma_smem_desc(b0 + (unsigned)(k0 / 8) * 128u, 128u, sbo);
        umma_bf16(tmem, adesc, bdesc, idesc, k0 > 0);
      }
      umma_commit(&bar_mma);
    }
    ok = mbar_wait_bounded(&bar_mma, ph_mma) || mbar_wait_bounded(&bar_mma, ph_mma);
    ph_mma ^= 1u;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc_fence_after();
    {
      const int quarter = warp & 3;
      const int box = 32 * quarter + lane;
      const int half = npad >> 1;
      const int c0 = (warp >> 2) * half;
      float* yi = y + ra.item_off[w];
      for (int c = c0; c < c0 + half; c += 8) {
        float v[8];
        tmem_ld8(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c, v);
        if (box < nb) {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (c + j < np) yi[(size_t)(c + j) * C.nb + box] = v[j];
        }
      }
    }
    tc_fence_before();
  }
  __syncthreads();
  if (failed && tid == 0) *ra.err = 1.0;
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 256);
}


// (1'') FP64 local solves by fast diagonalisation. On a level whose stencil
// is the Q1 Laplacian / d (checked at setup), a box's local matrix
// R_i Z_k R_i^T is (1/d) sum_i (x)_ax {K_l if ax = i else M_l} with the 1D
// Dirichlet matrices K_l = (1/h) tridiag(-1, 2, -1) and M_l = (h/6)
// tridiag(1, 4, 1) of the box extents l, both diagonalised by the orthonormal
// sine matrix S_l. The exact solve (A_k)_i^{-1} g is then: S along every axis
// but the last, one tridiagonal solve per line along the last axis (the
// operator restricted to each transformed line is tridiagonal, symmetric and
// diagonally dominant; its elimination factors are precomputed), S back.
// Per 12 x 12 box that is about 3,900 FP64 operations instead of the 20,736
// of the dense inverse: this GPU issues FP64 at a small fraction of its FP32
// rate, so the count of FP64 operations is what the FP64 smoother costs.
// A CTA takes one work item (boxes of one class); every phase gives each
// thread one grid line of one box (box index fastest), the box values live
// in shared memory with an odd row stride (np + 1), lines in registers (LM
// = the largest extent, a compile-time bound). Results are written box-major,
// y[item][b][i], the layout the level's index table gives k_ras_update.
// S applied along one grid line of length l (entries base + x * stride),
// in place. Row j of the sine matrix is symmetric (j even) or antisymmetric
// (j odd) about the line's midpoint, so the line is folded once into
// p_x = v_x + v_{l-1-x} and q_x = v_x - v_{l-1-x} (x < l/2) and each output
// takes l/2 FMAs (plus the middle entry for odd l and even j): about
// l + l^2/2 FP64 operations instead of l^2.
template <int LM>
__device__ __forceinline__ void fdm_line_transform(double* __restrict__ W, int base, int stride, int l,
                                                   const double* __restrict__ S, double* __restrict__ out = nullptr,
                                                   long long out_stride = 0) {
  constexpr int HM = (LM + 1) / 2;
  const int h = l >> 1;
  double pe[HM], qo[HM];
#pragma unroll
  for (int x = 0; x < HM; ++x) {
    if (x < h) {
      const double a = W[base + x * stride], b = W[base + (l - 1 - x) * stride];
      pe[x] = a + b;
      qo[x] = a - b;
    } else {
      pe[x] = 0.0;
      qo[x] = 0.0;
    }
  }
  const double mid = (l & 1) ? W[base + h * stride] : 0.0;
#pragma unroll
  for (int j = 0; j < LM; ++j) {
    if (j < l) {
      const double* Sj = S + j * l;
      double acc = 0.0;
      if (j & 1) {
#pragma unroll
        for (int x = 0; x < HM; ++x)
          if (x < h) acc = fma(__ldg(Sj + x), qo[x], acc);
      } else {
        if (l & 1) acc = __ldg(Sj + h) * mid;
#pragma unroll
        for (int x = 0; x < HM; ++x)
          if (x < h) acc = fma(__ldg(Sj + x), pe[x], acc);
      }
      if (out) out[j * out_stride] = acc;
      else W[base + j * stride] = acc;
    }
  }
}

template <int LM>
__device__ __forceinline__ void fdm_line_solve(double* __restrict__ W, int base, int stride, int n,
                                               const double* __restrict__ t) {
  // t = [b, l_0, winv_0, l_1, winv_1, ...]: y_i = g_i - l_i y_{i-1};
  // x_{n-1} = y_{n-1} winv_{n-1}; x_i = (y_i - b x_{i+1}) winv_i
  double g[LM];
#pragma unroll
  for (int i = 0; i < LM; ++i) g[i] = i < n ? W[base + i * stride] : 0.0;
#pragma unroll
  for (int i = 1; i < LM; ++i)
    if (i < n) g[i] = fma(-__ldg(t + 1 + 2 * i), g[i - 1], g[i]);
  const double b = __ldg(t);
  double xn = 0.0;
#pragma unroll
  for (int i = LM - 1; i >= 0; --i) {
    if (i < n) {
      const double xi = fma(-b, xn, g[i]) * __ldg(t + 2 + 2 * i);  // xn = 0 for i = n - 1: exactly g[i]
      W[base + i * stride] = xi;
      xn = xi;
    }
  }
}

template <int D, int LM>
__global__ void __launch_bounds__(kFdmThreads) k_ras_fdm(RasArgs ra, const double* __restrict__ rvec,
                                                 const double* __restrict__ tab, double* __restrict__ y) {
  extern __shared__ __align__(16) double W[];
  const int w = blockIdx.x;
  const int cls = ra.work[3 * w], first = ra.work[3 * w + 1], cnt = ra.work[3 * w + 2];
  const RasClass C = ra.classes[cls];
  const int lx = C.len[0], ly = C.len[1], lz = D > 2 ? C.len[2] : 1;
  const int np = C.np, ld = np + 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  // gather the residual on the boxes
  for (int t = tid; t < cnt * np; t += nt) {
    const int b = t / np, i = t - b * np;
    const int node0 = __ldg(ra.origin + __ldg(ra.class_patches + first + b)).w;
    W[b * ld + i] = __ldg(rvec + node0 + __ldg(ra.local_off_node + C.local_off + i));
  }
  __syncthreads();
  const double* Sx = tab + C.fdm_s[0];
  const double* Sy = tab + C.fdm_s[1];
  // forward transforms along x (and y in 3D)
  for (int t = tid; t < cnt * ly * lz; t += nt) {
    const int b = t % cnt, line = t / cnt;
    fdm_line_transform<LM>(W, b * ld + line * lx, 1, lx, Sx);
  }
  __syncthreads();
  if (D > 2) {
    for (int t = tid; t < cnt * lx * lz; t += nt) {
      const int b = t % cnt, line = t / cnt, j = line % lx, z = line / lx;
      fdm_line_transform<LM>(W, b * ld + j + z * lx * ly, lx, ly, Sy);
    }
    __syncthreads();
  }
  // tridiagonal solves along the last axis, one per transformed line
  {
    const int nlines = D > 2 ? lx * ly : lx, n = D > 2 ? lz : ly, stride = D > 2 ? lx * ly : lx;
    for (int t = tid; t < cnt * nlines; t += nt) {
      const int b = t % cnt, line = t / cnt;
      fdm_line_solve<LM>(W, b * ld + line, stride, n, tab + C.fdm_tri + (long long)line * (1 + 2 * n));
    }
  }
  __syncthreads();
  if (D > 2) {
    for (int t = tid; t < cnt * lx * lz; t += nt) {
      const int b = t % cnt, line = t / cnt, j = line % lx, z = line / lx;
      fdm_line_transform<LM>(W, b * ld + j + z * lx * ly, lx, ly, Sy);
    }
    __syncthreads();
  }
  // back along x in place, then the results to the work item's box-major
  // layout y[item][b][i] with consecutive threads on consecutive entries
  // (the per-node weighted sum then reads runs of neighbouring nodes)
  for (int t = tid; t < cnt * ly * lz; t += nt) {
    const int b = t % cnt, line = t / cnt;
    fdm_line_transform<LM>(W, b * ld + line * lx, 1, lx, Sx);
  }
  __syncthreads();
  double* yi = y + ra.item_off[w];
  for (int t = tid; t < cnt * np; t += nt) {
    const int b = t / np, i = t - b * np;
    yi[t] = W[b * ld + i];
  }
}

// symmetrised inverse as BF16 in the canonical K-major layout, padded to npad
__global__ void k_inv_bf16_canon(const double* __restrict__ a, __nv_bfloat16* __restrict__ out, int n, int npad) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)npad * npad) return;
  const int i = (int)(t / npad), k = (int)(t % npad);
  const double v = (i < n && k < n) ? 0.5 * (a[(long long)i * n + k] + a[(long long)k * n + i]) : 0.0;
  out[canon_bf16(i, k, npad)] = __float2bfloat16_rn((float)v);
}

// (2) z[j] += D_j * sum over the boxes containing j of their result for j;
// ysrc[j * 2^D + slot] is the index of that result in y (-1: no such box),
// slot bit ax = 0 for the node's own core tile along axis ax, 1 for the
// neighbouring tile whose overlap reaches it. D_j = 1/multiplicity, or 0/1
// on the core (restricted: slot 0 only).
template <typename T, int D>
__global__ void k_ras_update(const int* __restrict__ ysrc, const T* __restrict__ y, T* __restrict__ z, long long nn,
                             int restricted) {
  constexpr int SL = 1 << D;
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < nn; a += (long long)gridDim.x * blockDim.x) {
    int idx[SL];
    if constexpr (SL == 4) {
      const int4 t = __ldg(reinterpret_cast<const int4*>(ysrc) + a);
      idx[0] = t.x; idx[1] = t.y; idx[2] = t.z; idx[3] = t.w;
    } else {
      const int4 t0 = __ldg(reinterpret_cast<const int4*>(ysrc) + 2 * a);
      const int4 t1 = __ldg(reinterpret_cast<const int4*>(ysrc) + 2 * a + 1);
      idx[0] = t0.x; idx[1] = t0.y; idx[2] = t0.z; idx[3] = t0.w;
      idx[4] = t1.x; idx[5] = t1.y; idx[6] = t1.z; idx[7] = t1.w;
    }
    T s = __ldg(y + idx[0]);
    int mult = 1;
    if (!restricted) {
#pragma unroll
      for (int sl = 1; sl < SL; ++sl)
        if (idx[sl] >= 0) {
          s += __ldg(y + idx[sl]);
          ++mult;
        }
    }
    // multiplicities are products of 1s and 2s (a node lies in at most two
    // boxes per axis): the reciprocal is an exact power of two, picked
    // without a division, so s * inv = s / mult exactly and one FMA adds it
    const T inv = (restricted || mult == 1) ? (T)1 : mult == 2 ? (T)0.5 : mult == 4 ? (T)0.25 : (T)0.125;
    z[a] = fma(s, inv, z[a]);
  }
}

// Four consecutive shared-memory values (16-byte aligned) into registers.
__device__ __forceinline__ void lds4(const float* p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void lds4(const double* p, double (&v)[4]) {
  const double2 t0 = *reinterpret_cast<const double2*>(p);
  const double2 t1 = *reinterpret_cast<const double2*>(p + 2);
  v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
}

// Coarsest solve pass: S applied along one axis of the level grid, as the GEMM
//   C[i][n] = sum_k S[k][i] B[k][n],  B[k][n] = in[(n / inner) m inner + k inner + n % inner]
// (inner = m^axis; S is symmetric, so S[k][i] = S[i][k]). A CTA of 128 threads owns a
// 32 x 32 tile of C, each thread a 2 x 4 register block; k runs through
// chunks of 32 staged in two shared-memory buffers, the next chunk held in
// registers while the current one is multiplied. The k sum runs in order
// 0..m-1 for every output. Rows of S and columns of B are read coalesced (for
// axis 0 a warp reads 32 consecutive k of one column and stores them
// transposed).
constexpr int kFdmTile = 32, kFdmLd = 36;

template <typename T, bool AXIS0>
__global__ void __launch_bounds__(128) k_fdm_pass(const T* __restrict__ in, T* __restrict__ out,
                                                  const T* __restrict__ S, int m, long long inner,
                                                  long long ncols) {
  constexpr int KC = kFdmTile, LD = kFdmLd, NT = 128, R = KC * kFdmTile / NT, KW = NT / 32;
  __shared__ __align__(16) T sA[2][KC][LD];
  __shared__ __align__(16) T sB[2][KC][LD];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i0 = blockIdx.y * kFdmTile;
  const long long n0 = (long long)blockIdx.x * kFdmTile;
  const bool ia_ok = i0 + lane < m;
  // column of B this thread loads (all chunks) when the columns are the fast index
  const long long nb_l = n0 + lane;
  const bool nb_ok = nb_l < ncols;
  long long bbase = 0;
  if (!AXIS0 && nb_ok) {
    const long long hi = nb_l / inner;
    bbase = hi * m * inner + (nb_l - hi * inner);
  }
  T ra[R], rb[R];
  auto load = [&](int k0) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int k = warp + KW * r;  // row of the chunk
      const int kk = k0 + k;
      ra[r] = (kk < m && ia_ok) ? __ldg(S + (size_t)kk * m + i0 + lane) : (T)0;
      if (AXIS0) {
        const long long nb = n0 + k;  // here r walks the columns, lane the k
        const int kb = k0 + lane;
        rb[r] = (nb < ncols && kb < m) ? __ldg(in + (size_t)nb * m + kb) : (T)0;
      } else {
        rb[r] = (kk < m && nb_ok) ? __ldg(in + bbase + (size_t)kk * inner) : (T)0;
      }
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int k = warp + KW * r;
      sA[buf][k][lane] = ra[r];
      if (AXIS0) sB[buf][lane][k] = rb[r];
      else sB[buf][k][lane] = rb[r];
    }
  };
  const int ti = (tid >> 3) * 2, tn = (tid & 7) * 4;
  T acc[2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[a][q] = (T)0;
  const int nchunks = (m + KC - 1) / KC;
  load(0);
  store(0);
  __syncthreads();
  for (int c = 0; c < nchunks; ++c) {
    const int buf = c & 1;
    if (c + 1 < nchunks) load((c + 1) * KC);
#pragma unroll 8
    for (int k = 0; k < KC; ++k) {
      T bv[4];
      const T av[2] = {sA[buf][k][ti], sA[buf][k][ti + 1]};
      lds4(&sB[buf][k][tn], bv);
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[a][q] = fma(av[a], bv[q], acc[a][q]);
    }
    if (c + 1 < nchunks) store(buf ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const int ii = i0 + ti + a;
    if (ii >= m) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const long long nb = n0 + tn + q;
      if (nb >= ncols) continue;
      const long long hi = nb / inner;
      const long long o = hi * m * inner + (long long)ii * inner + (nb - hi * inner);
      out[o] = acc[a][q];
    }
  }
}

// ---------------------------------------------------------------------------
// FFT route for the same passes when N = m + 1 is a power of two: applying S
// along an axis is a type-I discrete sine transform of each grid line,
//   (S x)_k = sqrt(2/N) sum_j x_j sin(pi j k / N),  j, k = 1..N-1,
// which is -Im(V_k) / 2 (times sqrt(2/N)) for V the length-2N discrete
// Fourier transform of the odd extension (0, x_1..x_{N-1}, 0, -x_{N-1}..-x_1).
// Two real lines share one complex transform (line a in the real part, b in
// the imaginary part: a's sums are -Im(V)/2, b's are Re(V)/2). A CTA takes
// COLS consecutive lines, builds their extensions in shared memory in
// bit-reversed order and runs the log2(2N) radix-2 butterfly stages there,
// twiddles staged from a table made on the host in FP64.
// O(m^d log m) work instead of the dense passes' O(m^(d+1)).

template <typename T>
struct cplx;
template <>
struct cplx<float> {
  using type = float2;
};
template <>
struct cplx<double> {
  using type = double2;
};

// position of transform entry e in shared memory: one pad slot every 32
// entries, so the bit-reversed scatter of consecutive entries (which would
// land 32 entries apart) spreads over the banks
__device__ __forceinline__ int dst_pad(int e) { return e + (e >> 5); }

// the odd extension of the COLS lines' values v (entry k of line c, k < m)
// into bit-reversed, padded positions
template <typename T>
__device__ __forceinline__ void dst_scatter(T* bufr, int NP, int N2, int log2n2, int c, int k, T v) {
  const int j = k + 1, p = c >> 1, part = c & 1;
  const int r1 = (int)(__brev((unsigned)j) >> (32 - log2n2));
  const int r2 = (int)(__brev((unsigned)(N2 - j)) >> (32 - log2n2));
  bufr[2 * (p * NP + dst_pad(r1)) + part] = v;
  bufr[2 * (p * NP + dst_pad(r2)) + part] = -v;
}

template <typename C2>
__device__ __forceinline__ void dst_stages(C2* buf, const C2* stw, int NP, int N, int log2n2, int pairs) {
  for (int s = 0; s < log2n2; ++s) {
    const int h = 1 << s;
    for (int b = threadIdx.x; b < pairs * N; b += blockDim.x) {
      const int p = b / N, q = b - p * N;
      const int pos = q & (h - 1);
      const int i0 = ((q >> s) << (s + 1)) + pos, i1 = i0 + h;
      const C2 w = stw[pos << (log2n2 - 1 - s)];
      C2* e0 = buf + p * NP + dst_pad(i0);
      C2* e1 = buf + p * NP + dst_pad(i1);
      const C2 a = *e0, x = *e1;
      const auto tr = w.x * x.x - w.y * x.y, ti = w.x * x.y + w.y * x.x;
      *e0 = C2{a.x + tr, a.y + ti};
      *e1 = C2{a.x - tr, a.y - ti};
    }
    __syncthreads();
  }
}

// Threads per CTA of the long-transform kernel (k_dst_half below: two lines
// per CTA, so the grid has only ncols / 2 CTAs): FP32 gains from more warps
// (512 threads), FP64 is issue-bound and measured best at 256.
template <typename T>
constexpr int dst_threads() { return sizeof(T) == 4 ? 512 : 256; }

// One pass: out = S in along one axis, line by line (short transforms,
// 2(m+1) <= 256, COLS lines per CTA).
template <typename T, bool AXIS0, int COLS>
__global__ void __launch_bounds__(256) k_dst_pass(const T* __restrict__ in, T* __restrict__ out,
                                                  const typename cplx<T>::type* __restrict__ tw, int m, int log2n2,
                                                  long long inner, long long ncols, T scale) {
  using C2 = typename cplx<T>::type;
  extern __shared__ __align__(16) unsigned char dst_smem[];
  const int N2 = 1 << log2n2, N = N2 >> 1, NP = N2 + (N2 >> 5);
  C2* buf = reinterpret_cast<C2*>(dst_smem);  // [COLS / 2][NP]
  C2* stw = buf + (COLS / 2) * NP;             // [N]
  T* bufr = reinterpret_cast<T*>(buf);
  const long long n0 = (long long)blockIdx.x * COLS;
  for (int j = threadIdx.x; j < N; j += blockDim.x) stw[j] = tw[j];
  // the two zeros of every extension (positions 0 and N; bit reversal keeps
  // 0 at 0 and sends N to 1)
  for (int t = threadIdx.x; t < COLS / 2; t += blockDim.x) {
    buf[t * NP] = C2{(T)0, (T)0};
    buf[t * NP + 1] = C2{(T)0, (T)0};
  }
  const int total = COLS * m;
  auto entry = [&](int t, int& c, int& k) {
    if (AXIS0) {  // lines are contiguous: k fastest
      c = t / m;
      k = t - c * m;
    } else {      // lines are strided: consecutive threads take consecutive lines
      k = t / COLS;
      c = t - k * COLS;
    }
  };
  auto gidx = [&](long long nb, int k) {
    const long long hi = nb / inner;
    return hi * m * inner + (long long)k * inner + (nb - hi * inner);
  };
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int c, k;
    entry(t, c, k);
    const long long nb = n0 + c;
    const T v = nb < ncols ? __ldg(in + gidx(nb, k)) : (T)0;
    dst_scatter(bufr, NP, N2, log2n2, c, k, v);
  }
  __syncthreads();
  dst_stages(buf, stw, NP, N, log2n2, COLS / 2);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int c, k;
    entry(t, c, k);
    const long long nb = n0 + c;
    if (nb >= ncols) continue;
    const C2 V = buf[(c >> 1) * NP + dst_pad(k + 1)];
    T v = (c & 1) ? V.x : -V.y;
    out[gidx(nb, k)] = v * scale;  // scale = sqrt(2/N) / 2
  }
}

template <typename T, int COLS>
size_t dst_smem_bytes(int log2n2) {
  const size_t N2 = (size_t)1 << log2n2;
  return sizeof(typename cplx<T>::type) * ((COLS / 2) * (N2 + (N2 >> 5)) + N2 / 2);
}

// Long sine transforms (N = m + 1 >= 256, lines a, b per CTA) through one
// complex FFT of length N instead of 2N, about 40% fewer FP64 operations.
// With x_0 = x_N = 0 and, for j = 1..N-1,
//   y_j = sin(pi j / N) (x_j + x_{N-j}) + (x_j - x_{N-j}) / 2,   y_0 = 0,
// the DFT Y_k = R_k + i I_k of y (k = 0..N/2-1) gives the sine sums
//   X_{2k} = -I_k,   X_{2k+1} = X_{2k-1} + R_k,   X_1 = R_0 / 2
// (the symmetric part of y carries the odd sums through sin(pi j/N) cos(2 pi j k/N)
// = (sin(pi j (2k+1)/N) - sin(pi j (2k-1)/N)) / 2, the antisymmetric part the even
// ones). Lines a and b form the real and imaginary parts of one complex
// sequence, separated after the FFT through Z_k and conj(Z_{N-k}); the odd
// outputs are prefix sums of R, formed by a Hillis-Steele scan in shared
// memory (log2(N/2) steps; the rounding grows with the tree depth, as in the
// FFT itself). Output scale sqrt(2/N) (the orthonormal S).
template <typename T, bool AXIS0>
__global__ void __launch_bounds__(dst_threads<T>()) k_dst_half(const T* __restrict__ in, T* __restrict__ out,
                                                              const typename cplx<T>::type* __restrict__ tw, int m,
                                                              int log2n2, long long inner, long long ncols, T scale) {
  using C2 = typename cplx<T>::type;
  extern __shared__ __align__(16) unsigned char dst_smem[];
  const int log2n = log2n2 - 1, N = 1 << log2n, H = N >> 1, NP = N + (N >> 5);
  C2* buf = reinterpret_cast<C2*>(dst_smem);  // [NP]: the length-N transform
  C2* stw = buf + NP;                          // [N]: e^{-2 pi i j / (2N)}
  T* scan = reinterpret_cast<T*>(stw + N);     // [2 buffers][2 lines][H]
  const int tid = threadIdx.x, bd = blockDim.x;
  const long long la = 2LL * blockIdx.x, lb = la + 1;
  const bool va = la < ncols, vb = lb < ncols;
  auto gidx = [&](long long nb, int k) {
    if (AXIS0) return nb * m + k;
    const long long hi = nb / inner;
    return hi * m * inner + (long long)k * inner + (nb - hi * inner);
  };
  auto xin = [&](bool v, long long nb, int j) {  // x_j, j = 1..N-1 (entry j - 1)
    return v ? __ldg(in + gidx(nb, j - 1)) : (T)0;
  };
  for (int j = tid; j < N; j += bd) stw[j] = tw[j];
  __syncthreads();
  for (int j = tid; j < N; j += bd) {
    C2 z{(T)0, (T)0};
    if (j > 0) {
      const T sj = -stw[j].y;  // sin(pi j / N)
      const T a1 = xin(va, la, j), a2 = xin(va, la, N - j), b1 = xin(vb, lb, j), b2 = xin(vb, lb, N - j);
      z.x = fma(sj, a1 + a2, (T)0.5 * (a1 - a2));
      z.y = fma(sj, b1 + b2, (T)0.5 * (b1 - b2));
    }
    const int r = (int)(__brev((unsigned)j) >> (32 - log2n));
    buf[dst_pad(r)] = z;
  }
  __syncthreads();
  for (int st = 0; st < log2n; ++st) {
    const int h = 1 << st;
    for (int q = tid; q < H; q += bd) {
      const int pos = q & (h - 1);
      const int i0 = ((q >> st) << (st + 1)) + pos, i1 = i0 + h;
      const C2 w = stw[pos << (log2n2 - 1 - st)];  // e^{-2 pi i pos / 2^(st+1)}
      C2* e0 = buf + dst_pad(i0);
      C2* e1 = buf + dst_pad(i1);
      const C2 a = *e0, x = *e1;
      const T tr = w.x * x.x - w.y * x.y, ti = w.x * x.y + w.y * x.x;
      *e0 = C2{a.x + tr, a.y + ti};
      *e1 = C2{a.x - tr, a.y - ti};
    }
    __syncthreads();
  }
  const T sc = (T)2 * scale;  // sqrt(2/N)
  for (int k = tid; k < H; k += bd) {
    const C2 zk = buf[dst_pad(k)], zn = buf[dst_pad((N - k) & (N - 1))];
    const T ra = (T)0.5 * (zk.x + zn.x), ia = (T)0.5 * (zk.y - zn.y);
    const T rb = (T)0.5 * (zk.y + zn.y), ib = (T)0.5 * (zn.x - zk.x);
    if (k > 0) {
      if (va) out[gidx(la, 2 * k - 1)] = -ia * sc;
      if (vb) out[gidx(lb, 2 * k - 1)] = -ib * sc;
    }
    scan[k] = k == 0 ? (T)0.5 * ra : ra;
    scan[H + k] = k == 0 ? (T)0.5 * rb : rb;
  }
  __syncthreads();
  int cur = 0;
  for (int off = 1; off < H; off <<= 1) {
    const T* src = scan + cur * 2 * H;
    T* dst = scan + (cur ^ 1) * 2 * H;
    for (int t = tid; t < 2 * H; t += bd) {
      const int k = t & (H - 1);
      dst[t] = k >= off ? src[t] + src[t - off] : src[t];
    }
    __syncthreads();
    cur ^= 1;
  }
  const T* fin = scan + cur * 2 * H;
  for (int t = tid; t < 2 * H; t += bd) {
    const int k = t & (H - 1);
    if (t < H) {
      if (va) out[gidx(la, 2 * k)] = fin[t] * sc;
    } else if (vb) {
      out[gidx(lb, 2 * k)] = fin[t] * sc;
    }
  }
}

template <typename T>
size_t dst_half_smem_bytes(int log2n2) {
  const size_t N = (size_t)1 << (log2n2 - 1);
  return sizeof(typename cplx<T>::type) * ((N + (N >> 5)) + N) + sizeof(T) * 2 * N;
}

// one DST pass: long transforms (m + 1 >= 256) by the half-length FFT, two
// lines per CTA (enough CTAs to fill the GPU); short ones by the length-2N
// FFT, 8 lines per CTA. The route takes 2(m+1) <= 2048.
template <typename T>
void dst_pass(const T* in, T* out, const typename cplx<T>::type* tw, int m, int log2n2, long long inner,
              long long ncols, T scale, cudaStream_t s) {
  if (log2n2 >= 9) {
    const unsigned grid = (unsigned)((ncols + 1) / 2);
    const size_t smem = dst_half_smem_bytes<T>(log2n2);
    if (inner == 1) k_dst_half<T, true><<<grid, dst_threads<T>(), smem, s>>>(in, out, tw, m, log2n2, 1, ncols, scale);
    else k_dst_half<T, false><<<grid, dst_threads<T>(), smem, s>>>(in, out, tw, m, log2n2, inner, ncols, scale);
  } else {
    const unsigned grid = (unsigned)((ncols + 7) / 8);
    const size_t smem = dst_smem_bytes<T, 8>(log2n2);
    if (inner == 1) k_dst_pass<T, true, 8><<<grid, 256, smem, s>>>(in, out, tw, m, log2n2, 1, ncols, scale);
    else k_dst_pass<T, false, 8><<<grid, 256, smem, s>>>(in, out, tw, m, log2n2, inner, ncols, scale);
  }
}

// shared-memory opt-in of the sine-transform kernels for the largest
// transform the route takes (2(m+1) = 2048)
template <typename T>
int set_dst_smem() {
  const int big = (int)dst_half_smem_bytes<T>(11), small = (int)dst_smem_bytes<T, 8>(8);
  const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  DCG_CUDA(cudaFuncSetAttribute(k_dst_half<T, true>, attr, big));
  DCG_CUDA(cudaFuncSetAttribute(k_dst_half<T, false>, attr, big));
  DCG_CUDA(cudaFuncSetAttribute(k_dst_pass<T, true, 8>, attr, small));
  DCG_CUDA(cudaFuncSetAttribute(k_dst_pass<T, false, 8>, attr, small));
  return DCG_OK;
}

// Line solves T_j x = g along the last axis of the coarsest grid (factors
// from k_tri_setup; line j holds entries j + M1 y, y < m). The two sweeps
// are chains of m dependent FMAs, so their latency, not their arithmetic,
// sets the time: a CTA takes few lines (`cols`, chosen so that the grid
// covers the SMs about twice), stages them and their factors in shared
// memory with all its threads ([y][c] layout, loads unrolled so that many
// are in flight), `cols` threads run the sweeps, and all threads store.
// The backward step is one FMA on the chain:
//   x_y = (g'_y - e x_{y+1}) / w_y = fma(-(e / w_y), x_{y+1}, g'_y / w_y).
constexpr size_t kTriSmem = 200 * 1024;

template <typename T>
__global__ void __launch_bounds__(256) k_tri_last(const T* __restrict__ in, T* __restrict__ out,
                                                  const T* __restrict__ fl, const T* __restrict__ fw,
                                                  const T* __restrict__ fe, int m, long long M1, int cols) {
  extern __shared__ __align__(16) unsigned char tri_smem[];
  T* g = reinterpret_cast<T*>(tri_smem);
  T* sl = g + (size_t)m * cols;
  T* sw = sl + (size_t)m * cols;
  const long long j0 = (long long)blockIdx.x * cols;
  const int total = m * cols;
#pragma unroll 4
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int y = t / cols, c = t - y * cols;
    const long long j = j0 + c;
    if (j < M1) {
      const long long o = j + M1 * y;
      g[t] = __ldg(in + o);
      sl[t] = __ldg(fl + o);
      sw[t] = __ldg(fw + o);
    }
  }
  __syncthreads();
  const int c = threadIdx.x;
  if (c < cols && j0 + c < M1) {
    const T e = __ldg(fe + j0 + c);
    T prev = (T)0;  // forward: g'_y = g_y - l_y g'_{y-1}
    for (int y = 0; y < m; ++y) {
      const int t = y * cols + c;
      prev = fma(-sl[t], prev, g[t]);
      g[t] = prev;
    }
    T xn = (T)0;  // backward, x_m = 0
    for (int y = m - 1; y >= 0; --y) {
      const int t = y * cols + c;
      const T wi = sw[t];
      xn = fma(-(e * wi), xn, g[t] * wi);
      g[t] = xn;
    }
  }
  __syncthreads();
#pragma unroll 4
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int y = t / cols, c2 = t - y * cols;
    const long long j = j0 + c2;
    if (j < M1) out[j + M1 * y] = g[t];
  }
}

// lines per CTA of k_tri_last: enough CTAs for about two per SM, at most
// one 128-byte shared-memory row per y (conflict-free sweeps) and what the
// staging buffer holds; 0 when even one line does not fit
template <typename T>
int tri_cols(int m, long long M1) {
  if (3 * (size_t)m * sizeof(T) > kTriSmem) return 0;
  long long cols = std::max<long long>(1, std::min<long long>((long long)(128 / sizeof(T)), M1 / (2 * 152)));
  while (cols > 1 && 3 * (size_t)m * cols * sizeof(T) > kTriSmem) cols >>= 1;
  return (int)cols;
}

template <typename T>
void tri_last(const T* in, T* out, const T* fl, const T* fw, const T* fe, int m, long long M1, cudaStream_t s) {
  const int cols = tri_cols<T>(m, M1);
  const unsigned grid = (unsigned)((M1 + cols - 1) / cols);
  const size_t smem = 3 * (size_t)m * cols * sizeof(T);
  k_tri_last<T><<<grid, 256, smem, s>>>(in, out, fl, fw, fe, m, M1, cols);
}

// The same line solves by cyclic reduction when m = 2^q - 1 (coefficients
// from k_cr_setup). A CTA takes `cols` consecutive lines, staged in shared
// memory as [i][c] with zero rows i = 0 and i = m + 1 (the Dirichlet ends);
// reduction step k (k = 1..q-1, h = 2^(k-1)) updates the equations at the
// multiples of 2h, g_i += -beta_{k-1} (g_{i-h} + g_{i+h}); the last unknown
// (i = 2^(q-1)) is g gamma_{q-1}; back-substitution level k-1 solves the odd
// multiples of h, x_i = gamma_{k-1} g_i - beta_{k-1} (x_{i-h} + x_{i+h}).
// 2q - 1 steps separated by barriers, each spread over all threads: no long
// dependent chain. The CTA's coefficients are staged with its lines, so the
// steps touch shared memory only; few lines per CTA keep the grid wide (the
// staging loads of many CTAs are in flight together).
template <typename T>
__global__ void __launch_bounds__(256) k_tri_cr(const T* __restrict__ in, T* __restrict__ out,
                                                const T* __restrict__ beta, const T* __restrict__ gamma, int m, int q,
                                                long long M1, int cols) {
  extern __shared__ __align__(16) unsigned char cr_smem[];
  T* g = reinterpret_cast<T*>(cr_smem);  // [m + 2][cols]
  T* sb = g + (size_t)(m + 2) * cols;    // beta [q][cols]
  T* sg = sb + (size_t)q * cols;         // gamma [q][cols]
  const long long j0 = (long long)blockIdx.x * cols;
  const int total = m * cols;
#pragma unroll 4
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int i = t / cols, c = t - i * cols;
    const long long j = j0 + c;
    g[(i + 1) * cols + c] = j < M1 ? __ldg(in + j + M1 * i) : (T)0;
  }
  for (int t = threadIdx.x; t < q * cols; t += blockDim.x) {
    const int k = t / cols, c = t - k * cols;
    const long long j = min(j0 + c, M1 - 1);
    sb[t] = __ldg(beta + (long long)k * M1 + j);
    sg[t] = __ldg(gamma + (long long)k * M1 + j);
  }
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    g[c] = (T)0;
    g[(m + 1) * cols + c] = (T)0;
  }
  __syncthreads();
  for (int k = 1; k < q; ++k) {
    const int h = 1 << (k - 1), cnt = (1 << (q - k)) - 1;
    for (int t = threadIdx.x; t < cnt * cols; t += blockDim.x) {
      const int c = t % cols, i = (t / cols + 1) * 2 * h;
      g[i * cols + c] = fma(-sb[(k - 1) * cols + c], g[(i - h) * cols + c] + g[(i + h) * cols + c], g[i * cols + c]);
    }
    __syncthreads();
  }
  {
    const int i = 1 << (q - 1);
    for (int c = threadIdx.x; c < cols; c += blockDim.x) g[i * cols + c] *= sg[(q - 1) * cols + c];
  }
  __syncthreads();
  for (int k = q - 1; k >= 1; --k) {
    const int h = 1 << (k - 1), cnt = 1 << (q - k);
    for (int t = threadIdx.x; t < cnt * cols; t += blockDim.x) {
      const int c = t % cols, i = h * (2 * (t / cols) + 1);
      g[i * cols + c] = fma(-sb[(k - 1) * cols + c], g[(i - h) * cols + c] + g[(i + h) * cols + c],
                            sg[(k - 1) * cols + c] * g[i * cols + c]);
    }
    __syncthreads();
  }
#pragma unroll 4
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int i = t / cols, c = t - i * cols;
    const long long j = j0 + c;
    if (j < M1) out[j + M1 * i] = g[(i + 1) * cols + c];
  }
}

// lines per CTA of k_tri_cr: enough CTAs for about two per SM, at most one
// 128-byte shared-memory row per i, and what the buffer holds
template <typename T>
int cr_cols(int m, int q, long long M1) {
  long long cols = std::max<long long>(1, std::min<long long>((long long)(128 / sizeof(T)), M1 / (2 * 152)));
  while (cols > 1 && (size_t)(m + 2 + 2 * q) * cols * sizeof(T) > kTriSmem) cols >>= 1;
  return (int)cols;
}

template <typename T>
void tri_cr(const T* in, T* out, const T* beta, const T* gamma, int m, int q, long long M1, cudaStream_t s) {
  const int cols = cr_cols<T>(m, q, M1);
  const unsigned grid = (unsigned)((M1 + cols - 1) / cols);
  const size_t smem = (size_t)(m + 2 + 2 * q) * cols * sizeof(T);
  k_tri_cr<T><<<grid, 256, smem, s>>>(in, out, beta, gamma, m, q, M1, cols);
}

// z = Z_1^-1 f on the coarsest grid: passes of S along axes 0..d-2, line
// solves along axis d-1, passes of S along axes d-2..0 (2d - 1 launches).
// tmp: scratch of m^D values. With log2n2 > 0 (m + 1 a power of two) the
// passes are sine transforms by FFT, else dense GEMM passes with S.
// Returns the number of kernels launched.
template <typename T, int D>
int fdm_passes(const T* f, T* z, T* tmp, const T* S, const T* fl, const T* fw, const T* fe,
               const typename cplx<T>::type* tw, int log2n2, int m, cudaStream_t s) {
  // FFT route (m + 1 = 2^(log2n2 - 1)): fl, fw hold the cyclic-reduction
  // beta and gamma tables (fe unused); dense route: Thomas factors
  long long nn = 1;
  for (int k = 0; k < D; ++k) nn *= m;
  const long long ncols = nn / m, M1 = nn / m;
  const T scale = (T)(0.5 * std::sqrt(2.0 / (m + 1)));
  const dim3 ggrid((unsigned)((ncols + kFdmTile - 1) / kFdmTile), (unsigned)((m + kFdmTile - 1) / kFdmTile));
  auto pass = [&](const T* in, T* out, int axis) {
    const long long inner = axis == 0 ? 1 : (axis == 1 ? (long long)m : (long long)m * m);
    if (log2n2 > 0) dst_pass<T>(in, out, tw, m, log2n2, inner, ncols, scale, s);
    else if (inner == 1) k_fdm_pass<T, true><<<ggrid, 128, 0, s>>>(in, out, S, m, 1, ncols);
    else k_fdm_pass<T, false><<<ggrid, 128, 0, s>>>(in, out, S, m, inner, ncols);
  };
  auto lines = [&](const T* in, T* out) {
    if (log2n2 > 0) tri_cr<T>(in, out, fl, fw, m, log2n2 - 1, M1, s);
    else tri_last<T>(in, out, fl, fw, fe, m, M1, s);
  };
  if (D == 2) {
    pass(f, z, 0);
    lines(z, tmp);
    pass(tmp, z, 0);
  } else {
    pass(f, z, 0);
    pass(z, tmp, 1);
    lines(tmp, z);
    pass(z, tmp, 1);
    pass(tmp, z, 0);
  }
  return 2 * D - 1;
}

// FP64 fine residual r = g - Z_J z, stored into the cycle's level-J RHS (in
// the cycle precision); zeroes the level-J iterate; reduces ||r||^2 and, when
// with_g, ||g||^2 (g does not change within an inner solve). FP64 arithmetic
// is scarce on this GPU: with an FP32 cycle the squares of r are summed from
// its FP32 copy (the norm only feeds the stopping test).
template <typename T, int D>
__global__ void k_inner_residual(Stencil<double> st, const double* __restrict__ g, const double* __restrict__ z,
                                 T* __restrict__ fJ, T* __restrict__ zJ, double* __restrict__ r64, int m, long long nn,
                                 Reduce red, bool with_g) {
  double part[2] = {0.0, 0.0};
  T rr = (T)0;
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < nn; a += (long long)gridDim.x * blockDim.x) {
    int c[3];
    coords_of<D>(a, m, c);
    const double ga = g[a];
    const double r = ga - stencil_apply<double, D>(st, z, m, c);
    const T rt = (T)r;
    if (fJ) fJ[a] = rt;
    if (zJ) zJ[a] = (T)0;
    if (r64) r64[a] = r;
    rr = fma(rt, rt, rr);
    if (with_g) part[1] = fma(ga, ga, part[1]);
  }
  part[0] = (double)rr;
  grid_reduce<2>(part, red);
}

// k_inner_residual on a 2D box-sum level; a 1D grid of column blocks x row
// segments (bx fastest), so that the grid reduction sees gridDim.x CTAs
template <typename T>
__global__ void __launch_bounds__(kBoxThreads) k_inner_residual_box(double c0, double c1, const double* __restrict__ g,
                                                                    const double* __restrict__ z, T* __restrict__ fJ,
                                                                    T* __restrict__ zJ, int m, int gx, Reduce red,
                                                                    bool with_g) {
  double part[2] = {0.0, 0.0};
  T rr = (T)0;
  const int bx = blockIdx.x % gx, by = blockIdx.x / gx;
  const int x = bx * kBoxThreads + threadIdx.x;
  if (x < m) {
    box_residual_walk<double, double>(c0, c1, g, z, m, x, by * kBoxSeg, [&](long long a, double r) {
      const T rt = (T)r;
      fJ[a] = rt;
      zJ[a] = (T)0;
      rr = fma(rt, rt, rr);
      if (with_g) {
        const double ga = __ldg(g + a);
        part[1] = fma(ga, ga, part[1]);
      }
    });
  }
  part[0] = (double)rr;
  grid_reduce<2>(part, red);
}

template <typename T>
__global__ void k_fill_zero(T* __restrict__ z, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    z[i] = (T)0;
}

template <typename T>
__global__ void k_accumulate(double* __restrict__ z, const T* __restrict__ c, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    z[i] += (double)c[i];
}

template <typename T>
__global__ void k_from_t(const T* __restrict__ a, double* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

thread_local bool g_capturing = false;  // launches are being captured into the W-cycle graph

}  // namespace

std::vector<int> level_sizes(int n, int max_levels) {
  std::vector<int> s{n};
  while (s.back() % 2 == 0 && s.back() >= 8 && (int)s.size() < max_levels) s.push_back(s.back() / 2);
  return s;
}

namespace {

long long ipow(int b, int e) {
  long long r = 1;
  for (int k = 0; k < e; ++k) r *= b;
  return r;
}

// closed-form Q1 Laplacian stencil / d at spacing h (reference for the FDM solver)
Stencil<double> q1_laplacian_over_d(int D, double h) {
  Stencil<double> st{};
  const double K[3] = {-1.0 / h, 2.0 / h, -1.0 / h};
  const double M[3] = {h / 6.0, 4.0 * h / 6.0, h / 6.0};
  for (int o = 0; o < 27; ++o) {
    int off[3] = {o % 3, (o / 3) % 3, o / 9};
    if (D == 2 && off[2] != 1) continue;
    double s = 0.0;
    for (int i = 0; i < D; ++i) {
      double term = 1.0;
      for (int k = 0; k < D; ++k) term *= (k == i) ? K[off[k]] : M[off[k]];
      s += term;
    }
    int idx = off[0] + 3 * off[1] + (D == 2 ? 0 : 9 * off[2]);
    st.c[idx] = s / D;
  }
  return st;
}

constexpr size_t kResidentSmem = 220 * 1024;  // dynamic shared memory of a resident-inverse CTA

template <typename K>
int set_ras_smem(K kernel) {
  cudaFuncAttributes fa{};
  DCG_CUDA(cudaFuncGetAttributes(&fa, kernel));
  const int cap = 227 * 1024 - (int)fa.sharedSizeBytes;
  DCG_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
  return DCG_OK;
}

// batch width of a box class: 8 boxes per thread column, as many columns as
// fit 256 threads with ceil(np/4) row groups (power of two, 8..256 boxes)
int class_batch(int np) {
  const int rg = (np + 3) / 4;
  int bg = 1;
  while (bg * 2 * rg <= kRasThreads && bg * 2 <= 32) bg *= 2;
  return 8 * bg;
}

template <typename T>
bool ras_resident(const Level& L) {
  const size_t npp = (L.npmax + 3) / 4 * 4;
  return sizeof(T) * ((size_t)L.npmax * npp + (size_t)L.gmax) <= kResidentSmem;
}
template <typename T>
long long ras_goff(const Level& L) {
  const long long npp = (L.npmax + 3) / 4 * 4;
  return ras_resident<T>(L) ? (long long)L.npmax * npp : (long long)kKC * npp;
}
template <typename T>
size_t ras_smem_bytes(const Level& L) {
  return sizeof(T) * ((size_t)ras_goff<T>(L) + (size_t)L.gmax);
}

void free_level(Level& L) {
  cudaFree(L.d_patch_class); cudaFree(L.d_work); cudaFree(L.d_class_patches);
  cudaFree(L.d_classes); cudaFree(L.d_origin); cudaFree(L.d_core); cudaFree(L.d_local); cudaFree(L.d_axis_tab);
  cudaFree(L.d_local_node); cudaFree(L.d_item_off); cudaFree(L.d_ysrc); cudaFree(L.r);
  cudaFree(L.d_inv); cudaFree(L.d_inv_bf16); cudaFree(L.f); cudaFree(L.z); cudaFree(L.y); cudaFree(L.d_fdm);
  L = Level{};
}

int setup_ras(dcg_problem* p, Level& L, bool fp32, cudaStream_t s) {
  const int D = p->dim;
  const dcg_options& o = p->opts;
  L.tc = fp32 && o.ras_inverse == DCG_INV_BF16;  // BF16 inverses on the tensor cores
  L.tiles = Tiles1D{L.m, o.patch, o.overlap, (L.m + o.patch - 1) / o.patch};
  const int nt = L.tiles.ntile;
  L.npatch = (int)ipow(nt, D);
  // per-axis extent of every tile
  std::vector<int> len1(nt);
  for (int t = 0; t < nt; ++t) len1[t] = L.tiles.ext_hi(t) - L.tiles.ext_lo(t);
  std::map<std::vector<int>, int> cls_of;
  std::vector<int> pclass(L.npatch);
  L.classes.clear();
  for (int pid = 0; pid < L.npatch; ++pid) {
    int t3[3] = {pid % nt, (pid / nt) % nt, D > 2 ? pid / (nt * nt) : 0};
    std::vector<int> key(3, 1);
    for (int k = 0; k < D; ++k) key[k] = len1[t3[k]];
    auto it = cls_of.find(key);
    int c;
    if (it == cls_of.end()) {
      c = (int)L.classes.size();
      cls_of[key] = c;
      RasClass rc{};
      rc.len[0] = key[0]; rc.len[1] = key[1]; rc.len[2] = key[2];
      rc.np = key[0] * key[1] * key[2];
      L.classes.push_back(rc);
    } else {
      c = it->second;
    }
    pclass[pid] = c;
  }

  // FP64 levels whose stencil is the Q1 Laplacian / d solve their boxes by
  // fast diagonalisation (tables built below), in work items of kFdmBatch boxes
  L.fdm = false;
  if (!fp32) {
    int lmax = 0;
    for (int t = 0; t < nt; ++t) lmax = std::max(lmax, len1[t]);
    const Stencil<double> cf = q1_laplacian_over_d(D, 1.0 / L.n);
    double dev = 0.0, mx = 0.0;
    for (int k = 0; k < 27; ++k) {
      dev = std::max(dev, std::fabs(cf.c[k] - L.st64.c[k]));
      mx = std::max(mx, std::fabs(cf.c[k]));
    }
    L.fdm = dev <= 1e-12 * mx && lmax <= (D == 2 ? 16 : 6);
    L.fdm_lmax = lmax;
  }
  L.ras_np2 = 0;
  for (int pid = 0; pid < L.npatch; ++pid) L.ras_np2 += (long long)L.classes[pclass[pid]].np * L.classes[pclass[pid]].np;
  L.nclass = (int)L.classes.size();
  L.npmax = 0;
  long long inv_total = 0;
  for (auto& c : L.classes) {
    if (c.np > kMaxNp) {
      set_error_msg("RAS box larger than 256 nodes: reduce patch/overlap");
      return DCG_ERR_UNSUPPORTED;
    }
    c.npp = (c.np + 3) / 4 * 4;    // rows padded: 16-byte aligned vector loads
    c.npk = (c.np + 15) / 16 * 16;   // tensor-core N and K padding
    c.inv_off = inv_total;           // 16-byte aligned for the bulk copy into shared memory
    inv_total += L.tc ? (long long)c.npk * c.npk : (long long)c.np * c.npp;
    c.nb = L.tc ? kTcBatch : (L.fdm ? kFdmBatch : class_batch(c.np));
    L.npmax = std::max(L.npmax, c.np);
    L.gmax = std::max(L.gmax, (long long)c.np * c.nb);
  }
  // group patches by class, batch into work items
  std::vector<int> grouped;
  std::vector<int> work;
  for (int c = 0; c < L.nclass; ++c) {
    int start = (int)grouped.size();
    for (int pid = 0; pid < L.npatch; ++pid)
      if (pclass[pid] == c) grouped.push_back(pid);
    int cnt = (int)grouped.size() - start;
    const int nbc = L.classes[c].nb;
    for (int b = 0; b < cnt; b += nbc) {
      work.push_back(c);
      work.push_back(start + b);
      work.push_back(std::min(nbc, cnt - b));
    }
  }
  L.nwork = (int)work.size() / 3;
  // box origins, packed local coordinates per class, per-coordinate box table
  std::vector<int4> origin(L.npatch);
  std::vector<int2> core(L.npatch);
  for (int pid = 0; pid < L.npatch; ++pid) {
    int t3[3] = {pid % nt, (pid / nt) % nt, D > 2 ? pid / (nt * nt) : 0};
    int o3[3] = {0, 0, 0};
    int lo = 0, hi = 0;
    for (int k = 0; k < D; ++k) {
      o3[k] = L.tiles.ext_lo(t3[k]);
      lo |= (L.tiles.core_lo(t3[k]) - o3[k]) << (10 * k);
      hi |= (L.tiles.core_hi(t3[k]) - o3[k]) << (10 * k);
    }
    long long node = o3[0] + (long long)L.m * o3[1] + (long long)L.m * L.m * o3[2];
    origin[pid] = make_int4(o3[0], o3[1], o3[2], (int)node);
    core[pid] = make_int2(lo, hi);
  }
  std::vector<int> local, local_node;
  for (auto& c : L.classes) {
    c.local_off = (int)local.size();
    for (int k = 0; k < c.np; ++k) {
      int lx = k % c.len[0], ly = (k / c.len[0]) % c.len[1], lz = k / (c.len[0] * c.len[1]);
      local.push_back(lx | (ly << 10) | (lz << 20));
      local_node.push_back((int)(lx + (long long)L.m * (ly + (long long)L.m * lz)));
    }
  }
  // work-item result offsets and, per node and slot, the index of its result
  const int SL = 1 << D;
  std::vector<long long> item_off(L.nwork);
  long long ytot = 0;
  for (int w = 0; w < L.nwork; ++w) {
    const RasClass& c = L.classes[work[3 * w]];
    item_off[w] = ytot;
    ytot += (long long)c.np * c.nb;
  }
  L.ylen = ytot;
  if (ytot >= (1LL << 31)) {
    set_error_msg("RAS result buffer exceeds int32 indexing");
    return DCG_ERR_UNSUPPORTED;
  }
  std::vector<int> ysrc((size_t)L.nn * SL, -1);
  for (int w = 0; w < L.nwork; ++w) {
    const RasClass& c = L.classes[work[3 * w]];
    const int first = work[3 * w + 1], cnt = work[3 * w + 2];
    for (int b = 0; b < cnt; ++b) {
      const int pid = grouped[first + b];
      const int4 o4 = origin[pid];
      const int2 cb = core[pid];
      for (int i = 0; i < c.np; ++i) {
        const int pk = local[c.local_off + i];
        const int l3[3] = {pk & 1023, (pk >> 10) & 1023, (pk >> 20) & 1023};
        int slot = 0;
        for (int k = 0; k < D; ++k) {
          const int lo = (cb.x >> (10 * k)) & 1023, hi = (cb.y >> (10 * k)) & 1023;
          if (l3[k] < lo || l3[k] >= hi) slot |= 1 << k;
        }
        const long long node = o4.w + (long long)local_node[c.local_off + i];
        // item layout: [i][b] (entry-major) for the product kernels, [b][i]
        // (box-major) for the fast-diagonalisation kernel
        const long long at = L.fdm ? (long long)b * c.np + i : (long long)i * c.nb + b;
        ysrc[(size_t)node * SL + slot] = (int)(item_off[w] + at);
      }
    }
  }
  std::vector<int4> axis_tab(L.m);
  for (int c = 0; c < L.m; ++c) {
    const int t0 = c / o.patch;
    int4 e = make_int4(t0, c - L.tiles.ext_lo(t0), -1, 0);
    for (int t = t0 - 1; t <= t0 + 1; ++t) {
      if (t == t0 || t < 0 || t >= nt) continue;
      if (c >= L.tiles.ext_lo(t) && c < L.tiles.ext_hi(t)) { e.z = t; e.w = c - L.tiles.ext_lo(t); }
    }
    axis_tab[c] = e;
  }
  DCG_CUDA(cudaMalloc(&L.d_origin, sizeof(int4) * L.npatch));
  DCG_CUDA(cudaMalloc(&L.d_local, sizeof(int) * local.size()));
  DCG_CUDA(cudaMalloc(&L.d_local_node, sizeof(int) * local_node.size()));
  DCG_CUDA(cudaMalloc(&L.d_item_off, sizeof(long long) * item_off.size()));
  DCG_CUDA(cudaMalloc(&L.d_ysrc, sizeof(int) * ysrc.size()));
  DCG_CUDA(cudaMemcpyAsync(L.d_local_node, local_node.data(), sizeof(int) * local_node.size(), cudaMemcpyHostToDevice, s));
  DCG_CUDA(cudaMemcpyAsync(L.d_item_off, item_off.data(), sizeof(long long) * item_off.size(), cudaMemcpyHostToDevice, s));
  DCG_CUDA(cudaMemcpyAsync(L.d_ysrc, ysrc.data(), sizeof(int) * ysrc.size(), cudaMemcpyHostToDevice, s));
  DCG_CUDA(cudaMalloc(&L.d_axis_tab, sizeof(int4) * L.m));
  DCG_CUDA(cudaMalloc(&L.d_core, sizeof(int2) * L.npatch));
  DCG_CUDA(cudaMemcpyAsync(L.d_core, core.data(), sizeof(int2) * L.npatch, cudaMemcpyHostToDevice, s));
  DCG_CUDA(cudaMemcpyAsync(L.d_origin, origin.data(), sizeof(int4) * L.npatch, cudaMemcpyHostToDevice, s));
  DCG_CUDA(cudaMemcpyAsync(L.d_local, local.data(), sizeof(int) * local.size(), cudaMemcpyHostToDevice, s));
  DCG_CUDA(cudaMemcpyAsync(L.d_axis_tab, axis_tab.data(), sizeof(int4) * L.m, cudaMemcpyHostToDevice, s));
  DCG_CUDA(cudaStreamSynchronize(s));
  DCG_CUDA(cudaMalloc(&L.d_patch_class, sizeof(int) * L.npatch));
  DCG_CUDA(cudaMalloc(&L.d_class_patches, sizeof(int) * grouped.size()));
  DCG_CUDA(cudaMalloc(&L.d_work, sizeof(int) * work.size()));
  DCG_CUDA(cudaMalloc(&L.d_classes, sizeof(RasClass) * L.nclass));
  DCG_CUDA(cudaMemcpyAsync(L.d_patch_class, pclass.data(), sizeof(int) * L.npatch, cudaMemcpyHostToDevice, s));
  DCG_CUDA(cudaMemcpyAsync(L.d_class_patches, grouped.data(), sizeof(int) * grouped.size(), cudaMemcpyHostToDevice, s));
  DCG_CUDA(cudaMemcpyAsync(L.d_work, work.data(), sizeof(int) * work.size(), cudaMemcpyHostToDevice, s));
  DCG_CUDA(cudaMemcpyAsync(L.d_classes, L.classes.data(), sizeof(RasClass) * L.nclass, cudaMemcpyHostToDevice, s));
  const size_t tsz = fp32 ? sizeof(float) : sizeof(double);
  // fast-diagonalisation tables (sine matrices per box extent, elimination
  // factors of the line solves along the last axis), computed here in FP64
  if (L.fdm) {
    const double h = 1.0 / L.n;
    {
      std::vector<double> tab;
      std::map<int, int> s_off;  // extent -> offset of its sine matrix
      auto sine = [&](int l) {
        auto it = s_off.find(l);
        if (it != s_off.end()) return it->second;
        const int off = (int)tab.size();
        for (int j = 0; j < l; ++j)
          for (int x = 0; x < l; ++x)
            tab.push_back(std::sqrt(2.0 / (l + 1)) * std::sin(M_PI * (double)((j + 1) * (x + 1)) / (l + 1)));
        s_off[l] = off;
        return off;
      };
      auto kap = [&](int l, int j) { return (2.0 / h) * (1.0 - std::cos(M_PI * (j + 1) / (l + 1))); };
      auto mu = [&](int l, int j) { return (h / 3.0) * (2.0 + std::cos(M_PI * (j + 1) / (l + 1))); };
      for (auto& c : L.classes) {
        for (int k = 0; k < D; ++k) c.fdm_s[k] = sine(c.len[k]);
        c.fdm_tri = (long long)tab.size();
        const int n = c.len[D - 1];
        const int nsys = D == 2 ? c.len[0] : c.len[0] * c.len[1];
        for (int sys = 0; sys < nsys; ++sys) {
          // operator along the last axis after the transforms: a M_n + b K_n
          // (2D: (kap_j M + mu_j K) / 2; 3D: ((kap_j mu_k + mu_j kap_k) M + mu_j mu_k K) / 3)
          double cm, ck;
          if (D == 2) {
            cm = kap(c.len[0], sys) / 2.0;
            ck = mu(c.len[0], sys) / 2.0;
          } else {
            const int j = sys % c.len[0], k = sys / c.len[0];
            cm = (kap(c.len[0], j) * mu(c.len[1], k) + mu(c.len[0], j) * kap(c.len[1], k)) / 3.0;
            ck = mu(c.len[0], j) * mu(c.len[1], k) / 3.0;
          }
          const double a = cm * (4.0 * h / 6.0) + ck * (2.0 / h);
          const double b = cm * (h / 6.0) - ck * (1.0 / h);
          tab.push_back(b);
          double wprev = 0.0;
          for (int i = 0; i < n; ++i) {
            const double li = i == 0 ? 0.0 : b / wprev;
            const double wi = a - li * b;
            tab.push_back(li);
            tab.push_back(1.0 / wi);
            wprev = wi;
          }
        }
      }
      DCG_CUDA(cudaMalloc(&L.d_fdm, sizeof(double) * tab.size()));
      DCG_CUDA(cudaMemcpyAsync(L.d_fdm, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, s));
      DCG_CUDA(cudaMemcpyAsync(L.d_classes, L.classes.data(), sizeof(RasClass) * L.nclass, cudaMemcpyHostToDevice, s));
      DCG_CUDA(cudaStreamSynchronize(s));  // the host table goes out of scope
      // algorithmic flops of one smoothing product (an FMA counts 2): folded
      // transforms along every axis but the last, forward and back, and the
      // line solves along the last
      L.fdm_flops = 0.0;
      for (int pid = 0; pid < L.npatch; ++pid) {
        const RasClass& c = L.classes[pclass[pid]];
        const int n = c.len[D - 1];
        double per = (double)(c.np / n) * (5.0 * n - 2.0);  // line solves
        for (int k = 0; k < D - 1; ++k) {
          const int l = c.len[k], h = l / 2;
          per += 2.0 * (double)(c.np / l) * (2.0 * h + 2.0 * l * h);  // folded transforms, forward and back
        }
        L.fdm_flops += per;
      }
    }
  }
  // local inverses: box matrix from the stencil, Gauss-Jordan in FP64 (not
  // needed when the level solves its boxes by fast diagonalisation)
  if (L.fdm) inv_total = 1;
  DCG_CUDA(cudaMalloc(&L.d_inv, (L.tc ? sizeof(__nv_bfloat16) : tsz) * inv_total));
  double* work64 = nullptr;
  DCG_CUDA(cudaMalloc(&work64, sizeof(double) * (size_t)L.npmax * L.npmax));
  for (auto& c : L.classes) {
    if (L.fdm) break;
    const int np = c.np;
    const long long nel = (long long)np * np;
    const int g = (int)((nel + 255) / 256);
    if (D == 2) k_box_matrix<2><<<g, 256, 0, s>>>(L.st64, c.len[0], c.len[1], 1, work64);
    else k_box_matrix<3><<<g, 256, 0, s>>>(L.st64, c.len[0], c.len[1], c.len[2], work64);
    DCG_LAUNCH_CHECK();
    k_gauss_jordan<<<1, 1024, sizeof(double) * np, s>>>(work64, np);
    DCG_LAUNCH_CHECK();
    if (L.tc) {
      const int gp = (int)(((long long)c.npk * c.npk + 255) / 256);
      k_inv_bf16_canon<<<gp, 256, 0, s>>>(work64, (__nv_bfloat16*)L.d_inv + c.inv_off, np, c.npk);
    } else {
      const int gp = (int)(((long long)np * c.npp + 255) / 256);
      if (fp32) k_sym_convert<float><<<gp, 256, 0, s>>>(work64, (float*)L.d_inv + c.inv_off, np, c.npp);
      else k_sym_convert<double><<<gp, 256, 0, s>>>(work64, (double*)L.d_inv + c.inv_off, np, c.npp);
    }
    DCG_LAUNCH_CHECK();
  }
  DCG_CUDA(cudaStreamSynchronize(s));
  cudaFree(work64);
  DCG_CUDA(cudaMalloc(&L.y, tsz * L.ylen));
  DCG_CUDA(cudaMalloc(&L.r, tsz * L.nn));
  return DCG_OK;
}

template <typename T>
Stencil<T> st_of(const Level& L);
template <>
Stencil<float> st_of<float>(const Level& L) { return L.st32; }
template <>
Stencil<double> st_of<double>(const Level& L) { return L.st64; }

// r = f - Z_k z on level L (box-sum kernel where the stencil allows it)
template <typename T, int D>
void level_residual(const Level& L, const T* f, const T* z, T* r, cudaStream_t s) {
  if (D == 2 && L.box) {
    const dim3 grid((unsigned)((L.m + kBoxThreads - 1) / kBoxThreads), (unsigned)((L.m + kBoxSeg - 1) / kBoxSeg));
    k_residual_box<T><<<grid, kBoxThreads, 0, s>>>((T)L.box_c0, (T)L.box_c1, f, z, r, L.m);
  } else {
    k_residual<T, D><<<grid_for(L.nn, 256, 8192), 256, 0, s>>>(st_of<T>(L), f, z, r, L.m, L.nn);
  }
}

template <typename T>
const T* coarse_S(const Coarse& c);
template <>
const float* coarse_S<float>(const Coarse& c) { return c.S32; }
template <>
const double* coarse_S<double>(const Coarse& c) { return c.S64; }
// line-solve tables of the coarsest level in the cycle precision (cyclic
// reduction beta, gamma on the FFT route; Thomas l, 1/w, e otherwise)
template <typename T>
void coarse_tri(const Coarse& c, const T** f);
template <>
void coarse_tri<float>(const Coarse& c, const float** f) {
  f[0] = c.tri_l32;
  f[1] = c.tri_w32;
  f[2] = c.tri_e32;
}
template <>
void coarse_tri<double>(const Coarse& c, const double** f) {
  f[0] = c.tri_l64;
  f[1] = c.tri_w64;
  f[2] = c.tri_e64;
}
template <typename T>
const typename cplx<T>::type* coarse_tw(const Coarse& c);
template <>
const float2* coarse_tw<float>(const Coarse& c) { return c.tw32; }
template <>
const double2* coarse_tw<double>(const Coarse& c) { return c.tw64; }

template <typename T, int D>
int coarse_solve_t(dcg_problem* p, const T* f, T* z, cudaStream_t s) {
  const Coarse& C = p->coarse;
  const long long nn = ipow(C.m, D);
  const int prof = prof_begin(p, PC_COARSE, s, g_capturing);
  const T* tri[3];
  coarse_tri<T>(C, tri);
  const int nl = fdm_passes<T, D>(f, z, (T*)C.tmp, coarse_S<T>(C), tri[0], tri[1], tri[2], coarse_tw<T>(C), C.log2n2,
                                  C.m, s);
  note_launches(nl - 1);  // the check below counts one
  DCG_LAUNCH_CHECK();
  // algorithmic work: 2(d-1) transform passes (dense: 2 m flops per value;
  // FFT: 5 N2 log2(N2) flops per complex transform of length N2, two lines
  // each) and the line solves (Thomas 4 flops per value, cyclic reduction 5);
  // bytes: every pass reads and writes the field once, the Thomas sweeps
  // also read l and 1/w (the cyclic-reduction tables are q values per line)
  const double npass = 2.0 * (D - 1);
  const double flops = (C.log2n2 > 0 ? npass * ((double)nn / C.m / 2.0) * 5.0 * (double)(1 << C.log2n2) * C.log2n2 +
                                           5.0 * (double)nn
                                     : npass * 2.0 * (double)nn * C.m + 4.0 * (double)nn);
  const double bytes = sizeof(T) * 2.0 * (npass + 1) * (double)nn +
                       (C.log2n2 > 0 ? 0.0 : sizeof(T) * ((double)C.m * C.m + 2.0 * (double)nn));
  prof_end(p, prof, s, flops, bytes, g_capturing);
  return DCG_OK;
}

// shared memory of k_ras_fdm: the boxes of one work item, rows of np + 1
size_t fdm_smem_bytes(const Level& L) {
  size_t mx = 0;
  for (const auto& c : L.classes) mx = std::max(mx, sizeof(double) * (size_t)c.nb * (c.np + 1));
  return mx;
}

template <typename T, int D>
int ras_step_t(dcg_problem* p, Level& L, cudaStream_t s, bool z_zero = false) {
  RasArgs ra{};
  ra.m = L.m;
  ra.work = L.d_work; ra.class_patches = L.d_class_patches; ra.classes = L.d_classes;
  ra.origin = L.d_origin; ra.core = L.d_core; ra.local = L.d_local; ra.axis_tab = L.d_axis_tab;
  ra.local_off_node = L.d_local_node; ra.item_off = L.d_item_off;
  ra.err = p->scal + S_ERR;
  ra.nwork = L.nwork;
  ra.g_off = ras_goff<T>(L);
  const size_t smem = ras_smem_bytes<T>(L);
  const bool resident = ras_resident<T>(L);
  const int per_sm = std::max(1, std::min(2048 / kRasThreads, (int)((227 * 1024) / (smem + 1024))));
  const int cap = 152 * per_sm;
  ra.items_per_cta = (L.nwork + cap - 1) / cap;
  int grid = (L.nwork + ra.items_per_cta - 1) / ra.items_per_cta;
  // residual once per node (the first step from a zero iterate uses f itself)
  const T* rvec = (const T*)L.f;
  if (!z_zero) {
    const int prof = prof_begin(p, PC_TRANSFER, s, g_capturing);
    level_residual<T, D>(L, (const T*)L.f, (const T*)L.z, (T*)L.r, s);
    prof_end(p, prof, s, 2.0 * ipow(3, D) * (double)L.nn, sizeof(T) * 3.0 * L.nn, g_capturing);
    rvec = (const T*)L.r;
  }
  // algorithmic work: the shared-inverse products and the data they touch
  double bytes = 0.0;
  for (const auto& c : L.classes) bytes += sizeof(T) * (double)c.np * c.npp;
  const double flops = 2.0 * (double)L.ras_np2;
  bytes += sizeof(T) * 2.0 * (double)L.ylen;
  int prof = prof_begin(p, PC_RAS_SOLVE, s, g_capturing);
  if constexpr (sizeof(T) == 4) {
    if (L.tc) {
      long long npkmax = 0;
      for (const auto& c : L.classes) npkmax = std::max<long long>(npkmax, c.npk);
      RasArgs rt = ra;
      rt.g_off = npkmax * npkmax;
      const size_t smem_tc = sizeof(__nv_bfloat16) * (size_t)(npkmax * npkmax + 128 * npkmax);
      const int per_sm_tc = std::max(1, std::min(2, (int)((227 * 1024) / (smem_tc + 1024))));
      const int cap_tc = 152 * per_sm_tc;
      rt.items_per_cta = (L.nwork + cap_tc - 1) / cap_tc;
      const int grid_tc = (L.nwork + rt.items_per_cta - 1) / rt.items_per_cta;
      k_ras_solve_tc<D><<<grid_tc, 256, smem_tc, s>>>(rt, (const float*)rvec, (const __nv_bfloat16*)L.d_inv,
                                                      (float*)L.y);
      DCG_LAUNCH_CHECK();
      prof_end(p, prof, s, flops, bytes, g_capturing);
      prof = prof_begin(p, PC_RAS_UPDATE, s, g_capturing);
      k_ras_update<T, D><<<grid_for(L.nn, 256, 8192), 256, 0, s>>>(L.d_ysrc, (const T*)L.y, (T*)L.z, L.nn,
                                                                    p->opts.ras_weights == DCG_RAS_RESTRICTED);
      DCG_LAUNCH_CHECK();
      prof_end(p, prof, s, (double)L.nn * (1 << D),
               (double)L.nn * ((1 << D) * (4.0 + sizeof(T)) + 2.0 * sizeof(T)), g_capturing);
      return DCG_OK;
    }
  }
  if constexpr (sizeof(T) == 8) {
    if (L.fdm) {
      const size_t smem_f = fdm_smem_bytes(L);
      const int lm = L.fdm_lmax;
      if constexpr (D == 2) {
        if (lm <= 4) k_ras_fdm<D, 4><<<L.nwork, kFdmThreads, smem_f, s>>>(ra, (const double*)rvec, L.d_fdm, (double*)L.y);
        else if (lm <= 6) k_ras_fdm<D, 6><<<L.nwork, kFdmThreads, smem_f, s>>>(ra, (const double*)rvec, L.d_fdm, (double*)L.y);
        else if (lm <= 8) k_ras_fdm<D, 8><<<L.nwork, kFdmThreads, smem_f, s>>>(ra, (const double*)rvec, L.d_fdm, (double*)L.y);
        else if (lm <= 10) k_ras_fdm<D, 10><<<L.nwork, kFdmThreads, smem_f, s>>>(ra, (const double*)rvec, L.d_fdm, (double*)L.y);
        else if (lm <= 12) k_ras_fdm<D, 12><<<L.nwork, kFdmThreads, smem_f, s>>>(ra, (const double*)rvec, L.d_fdm, (double*)L.y);
        else k_ras_fdm<D, 16><<<L.nwork, kFdmThreads, smem_f, s>>>(ra, (const double*)rvec, L.d_fdm, (double*)L.y);
      } else {
        if (lm <= 4) k_ras_fdm<D, 4><<<L.nwork, kFdmThreads, smem_f, s>>>(ra, (const double*)rvec, L.d_fdm, (double*)L.y);
        else k_ras_fdm<D, 6><<<L.nwork, kFdmThreads, smem_f, s>>>(ra, (const double*)rvec, L.d_fdm, (double*)L.y);
      }
      DCG_LAUNCH_CHECK();
      prof_end(p, prof, s, L.fdm_flops, bytes, g_capturing);
      prof = prof_begin(p, PC_RAS_UPDATE, s, g_capturing);
      k_ras_update<T, D><<<grid_for(L.nn, 256, 8192), 256, 0, s>>>(L.d_ysrc, (const T*)L.y, (T*)L.z, L.nn,
                                                                    p->opts.ras_weights == DCG_RAS_RESTRICTED);
      DCG_LAUNCH_CHECK();
      prof_end(p, prof, s, (double)L.nn * (1 << D),
               (double)L.nn * ((1 << D) * (4.0 + sizeof(T)) + 2.0 * sizeof(T)), g_capturing);
      return DCG_OK;
    }
  }
  if (resident)
    k_ras_solve<T, D, true><<<grid, kRasThreads, smem, s>>>(ra, rvec, (const T*)L.d_inv, (T*)L.y);
  else
    k_ras_solve<T, D, false><<<grid, kRasThreads, smem, s>>>(ra, rvec, (const T*)L.d_inv, (T*)L.y);
  DCG_LAUNCH_CHECK();
  prof_end(p, prof, s, flops, bytes, g_capturing);
  prof = prof_begin(p, PC_RAS_UPDATE, s, g_capturing);
  k_ras_update<T, D><<<grid_for(L.nn, 256, 8192), 256, 0, s>>>(L.d_ysrc, (const T*)L.y, (T*)L.z, L.nn,
                                                                p->opts.ras_weights == DCG_RAS_RESTRICTED);
  DCG_LAUNCH_CHECK();
  prof_end(p, prof, s, (double)L.nn * (1 << D),
           (double)L.nn * ((1 << D) * (4.0 + sizeof(T)) + 2.0 * sizeof(T)), g_capturing);
  return DCG_OK;
}

template <typename T, int D>
int wcycle_t(dcg_problem* p, int k, cudaStream_t s, bool z_zero) {
  Level& L = p->levels[k - 1];
  if (k == 1) return coarse_solve_t<T, D>(p, (const T*)L.f, (T*)L.z, s);
  Level& Lc = p->levels[k - 2];
  for (int i = 0; i < p->opts.m1; ++i) DCG_TRY((ras_step_t<T, D>(p, L, s, z_zero && i == 0)));
  int prof = prof_begin(p, PC_TRANSFER, s, g_capturing);
  level_residual<T, D>(L, (const T*)L.f, (const T*)L.z, (T*)L.r, s);
  k_restrict<T, D><<<grid_for(Lc.nn, 256, 8192), 256, 0, s>>>((const T*)L.r, (T*)Lc.f, L.m, Lc.m, Lc.nn);
  DCG_LAUNCH_CHECK();
  prof_end(p, prof, s, 2.0 * (ipow(3, D) * (double)L.nn + ipow(3, D) * (double)Lc.nn),
           sizeof(T) * (4.0 * L.nn + Lc.nn), g_capturing);
  // the next level starts from zero; the exact coarsest solve overwrites its
  // z and needs no fill (a kernel, not a memset: graph bodies take it)
  if (k - 1 > 1) {
    k_fill_zero<T><<<grid_for(Lc.nn, 256, 8192), 256, 0, s>>>((T*)Lc.z, Lc.nn);
    DCG_LAUNCH_CHECK();
  }
  DCG_TRY((wcycle_t<T, D>(p, k - 1, s, true)));
  // Algorithm 4's second recursive call W_{k-1}(r_c, e1): on the coarsest
  // level W is the exact solve, which ignores the initial guess, so the second
  // call would repeat the first bit for bit and is skipped there
  if (k - 1 > 1) DCG_TRY((wcycle_t<T, D>(p, k - 1, s, false)));
  prof = prof_begin(p, PC_TRANSFER, s, g_capturing);
  if (D == 2) {
    const long long npairs = (long long)((L.m + 1) / 2) * L.m;
    k_prolong_add_2d<T><<<grid_for(npairs, 256, 8192), 256, 0, s>>>((const T*)Lc.z, (T*)L.z, L.m, Lc.m);
  } else {
    k_prolong_add<T, D><<<grid_for(L.nn, 256, 8192), 256, 0, s>>>((const T*)Lc.z, (T*)L.z, L.m, Lc.m, L.nn);
  }
  DCG_LAUNCH_CHECK();
  prof_end(p, prof, s, 2.0 * L.nn, sizeof(T) * (2.0 * L.nn + Lc.nn), g_capturing);
  for (int i = 0; i < p->opts.m2; ++i) DCG_TRY((ras_step_t<T, D>(p, L, s)));
  return DCG_OK;
}

template <typename T>
int wcycle_dispatch(dcg_problem* p, cudaStream_t s) {
  const int J = (int)p->levels.size();
  return p->dim == 2 ? wcycle_t<T, 2>(p, J, s, true) : wcycle_t<T, 3>(p, J, s, true);
}

int build_wcycle_graph(dcg_problem* p) {
  MGState& S = p->mg;
  if (S.wexec) { cudaGraphExecDestroy(S.wexec); S.wexec = nullptr; }
  prof_clear_graph(p);
  if (!S.cap) DCG_CUDA(cudaStreamCreateWithFlags(&S.cap, cudaStreamNonBlocking));
  DCG_CUDA(cudaStreamBeginCapture(S.cap, cudaStreamCaptureModeThreadLocal));
  g_capturing = true;
  t_capturing = true;
  t_capture_launches = 0;
  int st = S.fp32 ? wcycle_dispatch<float>(p, S.cap) : wcycle_dispatch<double>(p, S.cap);
  S.graph_kernels = t_capture_launches;
  t_capturing = false;
  g_capturing = false;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(S.cap, &graph);
  if (st != DCG_OK) { if (graph) cudaGraphDestroy(graph); return st; }
  if (e != cudaSuccess) { set_error("cudaStreamEndCapture", e); return DCG_ERR_CUDA; }
  e = cudaGraphInstantiate(&S.wexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) { set_error("cudaGraphInstantiate", e); return DCG_ERR_CUDA; }
  return DCG_OK;
}

int run_wcycle(dcg_problem* p, cudaStream_t s) {
  MGState& S = p->mg;
  if (!S.wexec) DCG_TRY(build_wcycle_graph(p));
  DCG_CUDA(cudaGraphLaunch(S.wexec, s));
  note_launches(S.graph_kernels);
  return DCG_OK;
}

bool exact_mode(const dcg_problem* p) { return p->opts.inner_rule == DCG_INNER_EXACT; }

}  // namespace

void mg_free(dcg_problem* p) {
  for (auto& L : p->levels) free_level(L);
  p->levels.clear();
  cudaFree(p->coarse.S64); cudaFree(p->coarse.S32); cudaFree(p->coarse.tri_l64); cudaFree(p->coarse.tri_w64); cudaFree(p->coarse.tri_e64);
  cudaFree(p->coarse.tri_l32); cudaFree(p->coarse.tri_w32); cudaFree(p->coarse.tri_e32);
  cudaFree(p->coarse.tmp);
  cudaFree(p->coarse.tw64); cudaFree(p->coarse.tw32);
  p->coarse = Coarse{};
  if (p->mg.wexec) cudaGraphExecDestroy(p->mg.wexec);
  if (p->mg.cap) cudaStreamDestroy(p->mg.cap);
  p->mg = MGState{};
}

int mg_setup(dcg_problem* p, cudaStream_t s) {
  mg_free(p);
  const int D = p->dim;
  const dcg_options& o = p->opts;
  const bool fp32 = (o.precision == DCG_MIXED) && !exact_mode(p);
  double* scal2 = nullptr;
  DCG_CUDA(cudaMalloc(&scal2, sizeof(double) * 2 + sizeof(double) * 27 * 2));
  Stencil<double> stJ{};
  if (p->matrix_free) {
    // --- Z_J = V^T A V by probing the matrix-free operator (checked below,
    // once the hierarchy exists, against the stencil on a full vector)
    if (D != 3 || p->m < 3) {
      cudaFree(scal2);
      set_error_msg("matrix-free problems need a 3D mesh with n >= 4");
      return DCG_ERR_UNSUPPORTED;
    }
    int st = mf_probe_stencil(p, stJ.c, s);
    if (st != DCG_OK) {
      cudaFree(scal2);
      return st;
    }
  } else {
  // --- Z_J = V^T A V from the assembled matrix, checked to be one stencil
  double* rows = nullptr;
  DCG_CUDA(cudaMalloc(&rows, sizeof(double) * 27 * p->n_nodes));
  DCG_CUDA(cudaMemsetAsync(scal2, 0, sizeof(double) * 2, s));
  const int g = grid_for(p->n_nodes, 256, 1 << 30);
  if (D == 2) k_zj_rows<2><<<g, 256, 0, s>>>(p->row_ptr, p->col_idx, p->vals, p->m, p->n_nodes, 1.0 / D, rows, scal2);
  else k_zj_rows<3><<<g, 256, 0, s>>>(p->row_ptr, p->col_idx, p->vals, p->m, p->n_nodes, 1.0 / D, rows, scal2);
  DCG_LAUNCH_CHECK();
  // Reference stencil: offset o is read from a node whose neighbour at o
  // exists (low corner for +1, high corner for -1), so meshes with fewer than
  // three interior nodes per axis are covered too; offsets that exist for no
  // node (m = 1) stay zero and are never used.
  double* d_ref = scal2 + 2;
  DCG_CUDA(cudaMemsetAsync(d_ref, 0, sizeof(double) * 27, s));
  for (int o = 0; o < (D == 2 ? 9 : 27); ++o) {
    const int off[3] = {o % 3 - 1, (o / 3) % 3 - 1, D > 2 ? o / 9 - 1 : 0};
    long long node = 0, stride = 1;
    bool exists = true;
    for (int k = 0; k < D; ++k) {
      const int c = off[k] > 0 ? 0 : (off[k] < 0 ? p->m - 1 : 0);
      exists = exists && (c + off[k] >= 0 && c + off[k] < p->m);
      node += c * stride;
      stride *= p->m;
    }
    if (exists)
      DCG_CUDA(cudaMemcpyAsync(d_ref + o, rows + node * 27 + o, sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  if (D == 2) k_zj_check<2><<<g, 256, 0, s>>>(rows, d_ref, p->m, p->n_nodes, scal2 + 1);
  else k_zj_check<3><<<g, 256, 0, s>>>(rows, d_ref, p->m, p->n_nodes, scal2 + 1);
  DCG_LAUNCH_CHECK();
  double h_sc[2];
  DCG_CUDA(cudaMemcpyAsync(h_sc, scal2, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
  DCG_CUDA(cudaMemcpyAsync(stJ.c, d_ref, sizeof(double) * 27, cudaMemcpyDeviceToHost, s));
  DCG_CUDA(cudaStreamSynchronize(s));
  cudaFree(rows);
  double smax = 0.0;
  for (double v : stJ.c) smax = std::max(smax, std::fabs(v));
  const double tol = std::max(1e-12 * smax, 8.0 * D * D * std::ldexp(1.0, -52) * h_sc[0]);
  if (!(h_sc[1] <= tol) || p->m < 1) {
    char buf[200];
    snprintf(buf, sizeof buf, "V^T A V is not a constant stencil (deviation %.3e, tolerance %.3e)", h_sc[1], tol);
    set_error_msg(buf);
    cudaFree(scal2);
    return DCG_ERR_UNSUPPORTED;
  }
  }  // assembled
  // --- levels
  std::vector<int> sizes = exact_mode(p) ? std::vector<int>{p->n} : level_sizes(p->n, o.max_levels);
  const int J = (int)sizes.size();
  p->levels.assign(J, Level{});
  {
    Level& LJ = p->levels[J - 1];
    LJ.n = sizes[0];
    LJ.m = sizes[0] - 1;
    LJ.nn = ipow(LJ.m, D);
    LJ.st64 = stJ;
  }
  double* d_sf = scal2 + 2;
  double* d_sc = scal2 + 2 + 27;
  for (int k = J - 1; k >= 1; --k) {
    Level& Lf = p->levels[k];
    Level& Lc = p->levels[k - 1];
    Lc.n = sizes[J - k];
    Lc.m = Lc.n - 1;
    Lc.nn = ipow(Lc.m, D);
    DCG_CUDA(cudaMemcpyAsync(d_sf, Lf.st64.c, sizeof(double) * 27, cudaMemcpyHostToDevice, s));
    DCG_CUDA(cudaMemsetAsync(d_sc, 0, sizeof(double) * 27, s));
    if (D == 2) k_galerkin<2><<<1, 32, 0, s>>>(d_sf, d_sc);
    else k_galerkin<3><<<1, 32, 0, s>>>(d_sf, d_sc);
    DCG_LAUNCH_CHECK();
    DCG_CUDA(cudaMemcpyAsync(Lc.st64.c, d_sc, sizeof(double) * 27, cudaMemcpyDeviceToHost, s));
    DCG_CUDA(cudaStreamSynchronize(s));
  }
  cudaFree(scal2);
  for (auto& L : p->levels) {
    for (int k = 0; k < 27; ++k) L.st32.c[k] = (float)L.st64.c[k];
    // box-sum form: the 8 neighbour coefficients agree to 1e-12 (they are
    // equal in exact arithmetic for the Q1 Laplacian; assembly and the
    // Galerkin products leave rounding), their mean stands for all
    L.box = false;
    if (D == 2 && L.m >= 3) {
      double sum = 0.0, lo = L.st64.c[0], hi = L.st64.c[0];
      for (int k = 0; k < 9; ++k) {
        if (k == 4) continue;
        sum += L.st64.c[k];
        lo = std::min(lo, L.st64.c[k]);
        hi = std::max(hi, L.st64.c[k]);
      }
      const double c1 = sum / 8.0;
      if (c1 != 0.0 && hi - lo <= 1e-12 * std::fabs(c1)) {
        L.box = true;
        L.box_c1 = c1;
        L.box_c0 = L.st64.c[4] - c1;
      }
    }
  }
  // coarsest: check the closed form the fast-diagonalisation solver assumes
  {
    Level& L1 = p->levels[0];
    Stencil<double> cf = q1_laplacian_over_d(D, 1.0 / L1.n);
    double dev = 0.0, mx = 0.0;
    for (int k = 0; k < (D == 2 ? 9 : 27); ++k) {
      const int off[3] = {k % 3 - 1, (k / 3) % 3 - 1, D > 2 ? k / 9 - 1 : 0};
      bool used = true;  // offsets reaching outside a 1-node grid never act
      for (int a = 0; a < D; ++a) used = used && (off[a] == 0 || L1.m >= 2);
      if (!used) continue;
      dev = std::max(dev, std::fabs(cf.c[k] - L1.st64.c[k]));
      mx = std::max(mx, std::fabs(cf.c[k]));
    }
    if (!(dev <= 1e-10 * mx)) {
      char buf[160];
      snprintf(buf, sizeof buf, "coarsest stencil is not the Q1 Laplacian (deviation %.3e)", dev);
      set_error_msg(buf);
      return DCG_ERR_UNSUPPORTED;
    }
  }
  // --- buffers and RAS
  const size_t tsz = fp32 ? sizeof(float) : sizeof(double);
  p->mg.fp32 = fp32;
  for (int k = 0; k < J; ++k) {
    Level& L = p->levels[k];
    DCG_CUDA(cudaMalloc(&L.f, tsz * L.nn));
    DCG_CUDA(cudaMalloc(&L.z, tsz * L.nn));
    DCG_CUDA(cudaMemsetAsync(L.z, 0, tsz * L.nn, s));
    if (k >= 1) DCG_TRY(setup_ras(p, L, fp32, s));
  }
  // --- coarsest solver
  {
    Coarse& C = p->coarse;
    C.m = p->levels[0].m;
    const long long nn = p->levels[0].nn;
    DCG_CUDA(cudaMalloc(&C.S64, sizeof(double) * C.m * C.m));
    const long long M1 = nn / C.m;
    DCG_CUDA(cudaMalloc(&C.tmp, tsz * nn));
    k_fdm_setup<<<grid_for((long long)C.m * C.m, 256), 256, 0, s>>>(C.m, C.S64);
    DCG_LAUNCH_CHECK();
    // FFT route: m + 1 a power of two, transforms of length 2(m+1) <= 2048,
    // line solves by cyclic reduction; else dense passes and Thomas sweeps
    C.log2n2 = 0;
    long long nl_fac = nn, ne_fac = M1;  // sizes of the two factor tables and of e
    if (((C.m + 1) & C.m) == 0 && C.m + 1 <= 1024) {
      int l = 1;
      while ((1 << l) < 2 * (C.m + 1)) ++l;
      C.log2n2 = l;
      const int q = l - 1;  // m = 2^q - 1
      nl_fac = (long long)q * M1;
      ne_fac = 0;
      DCG_CUDA(cudaMalloc(&C.tri_l64, sizeof(double) * nl_fac));
      DCG_CUDA(cudaMalloc(&C.tri_w64, sizeof(double) * nl_fac));
      if (D == 2) k_cr_setup<2><<<grid_for(M1, 128), 128, 0, s>>>(C.m, q, C.tri_l64, C.tri_w64);
      else k_cr_setup<3><<<grid_for(M1, 128), 128, 0, s>>>(C.m, q, C.tri_l64, C.tri_w64);
      DCG_LAUNCH_CHECK();
      const int N = C.m + 1;
      std::vector<double2> tw(N);
      std::vector<float2> tw32(N);
      for (int j = 0; j < N; ++j) {
        const double a = M_PI * (double)j / (double)N;  // 2 pi j / (2N)
        tw[j] = make_double2(std::cos(a), -std::sin(a));
        tw32[j] = make_float2((float)tw[j].x, (float)tw[j].y);
      }
      DCG_CUDA(cudaMalloc(&C.tw64, sizeof(double2) * N));
      DCG_CUDA(cudaMalloc(&C.tw32, sizeof(float2) * N));
      DCG_CUDA(cudaMemcpyAsync(C.tw64, tw.data(), sizeof(double2) * N, cudaMemcpyHostToDevice, s));
      DCG_CUDA(cudaMemcpyAsync(C.tw32, tw32.data(), sizeof(float2) * N, cudaMemcpyHostToDevice, s));
      DCG_CUDA(cudaStreamSynchronize(s));  // the host tables go out of scope
      DCG_TRY(set_dst_smem<float>());
      DCG_TRY(set_dst_smem<double>());
      DCG_CUDA(cudaFuncSetAttribute(k_tri_cr<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTriSmem));
      DCG_CUDA(cudaFuncSetAttribute(k_tri_cr<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTriSmem));
    } else {
      if (tri_cols<double>(C.m, M1) < 1) {
        set_error_msg("coarsest level too large for its line solves (more than 8533 nodes per axis)");
        return DCG_ERR_UNSUPPORTED;
      }
      DCG_CUDA(cudaMalloc(&C.tri_l64, sizeof(double) * nn));
      DCG_CUDA(cudaMalloc(&C.tri_w64, sizeof(double) * nn));
      DCG_CUDA(cudaMalloc(&C.tri_e64, sizeof(double) * M1));
      if (D == 2) k_tri_setup<2><<<grid_for(M1, 128), 128, 0, s>>>(C.m, C.tri_l64, C.tri_w64, C.tri_e64);
      else k_tri_setup<3><<<grid_for(M1, 128), 128, 0, s>>>(C.m, C.tri_l64, C.tri_w64, C.tri_e64);
      DCG_LAUNCH_CHECK();
      DCG_CUDA(cudaFuncSetAttribute(k_tri_last<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTriSmem));
      DCG_CUDA(cudaFuncSetAttribute(k_tri_last<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTriSmem));
    }
    if (fp32) {
      DCG_CUDA(cudaMalloc(&C.S32, sizeof(float) * C.m * C.m));
      DCG_CUDA(cudaMalloc(&C.tri_l32, sizeof(float) * nl_fac));
      DCG_CUDA(cudaMalloc(&C.tri_w32, sizeof(float) * nl_fac));
      k_to_t<float><<<grid_for(C.m * C.m, 256), 256, 0, s>>>(C.S64, C.S32, (long long)C.m * C.m);
      k_to_t<float><<<grid_for(nl_fac, 256), 256, 0, s>>>(C.tri_l64, C.tri_l32, nl_fac);
      k_to_t<float><<<grid_for(nl_fac, 256), 256, 0, s>>>(C.tri_w64, C.tri_w32, nl_fac);
      if (ne_fac > 0) {
        DCG_CUDA(cudaMalloc(&C.tri_e32, sizeof(float) * ne_fac));
        k_to_t<float><<<grid_for(ne_fac, 256), 256, 0, s>>>(C.tri_e64, C.tri_e32, ne_fac);
      }
      DCG_LAUNCH_CHECK();
    }
  }
  // RAS kernel shared memory opt-in: 227 KB per block minus the kernel's
  // static shared memory
  DCG_TRY(set_ras_smem(k_ras_solve_tc<2>));
  DCG_TRY(set_ras_smem(k_ras_solve_tc<3>));
  DCG_TRY(set_ras_smem(k_ras_solve<float, 2, true>));
  DCG_TRY(set_ras_smem(k_ras_solve<float, 3, true>));
  DCG_TRY(set_ras_smem(k_ras_solve<float, 2, false>));
  DCG_TRY(set_ras_smem(k_ras_solve<float, 3, false>));
  DCG_TRY(set_ras_smem(k_ras_fdm<2, 4>));
  DCG_TRY(set_ras_smem(k_ras_fdm<2, 6>));
  DCG_TRY(set_ras_smem(k_ras_fdm<2, 8>));
  DCG_TRY(set_ras_smem(k_ras_fdm<2, 10>));
  DCG_TRY(set_ras_smem(k_ras_fdm<2, 12>));
  DCG_TRY(set_ras_smem(k_ras_fdm<2, 16>));
  DCG_TRY(set_ras_smem(k_ras_fdm<3, 4>));
  DCG_TRY(set_ras_smem(k_ras_fdm<3, 6>));
  DCG_TRY(set_ras_smem(k_ras_solve<double, 2, true>));
  DCG_TRY(set_ras_smem(k_ras_solve<double, 3, true>));
  DCG_TRY(set_ras_smem(k_ras_solve<double, 2, false>));
  DCG_TRY(set_ras_smem(k_ras_solve<double, 3, false>));
  DCG_CUDA(cudaStreamSynchronize(s));
  if (p->matrix_free) DCG_TRY(mf_check_stencil(p, s));
  if (!exact_mode(p)) DCG_TRY(build_wcycle_graph(p));
  return DCG_OK;
}

int mg_rebuild_graph(dcg_problem* p) {
  if (p->levels.empty() || exact_mode(p)) return DCG_OK;
  return build_wcycle_graph(p);
}

int mg_inner_apply(dcg_problem* p, const double* z, double* y, cudaStream_t s) {
  if (p->levels.empty()) return DCG_ERR_STATE;
  Level& L = p->levels.back();
  const int g = grid_for(L.nn, 256, 8192);
  if (p->dim == 2) k_apply<double, 2><<<g, 256, 0, s>>>(L.st64, z, y, L.m, L.nn);
  else k_apply<double, 3><<<g, 256, 0, s>>>(L.st64, z, y, L.m, L.nn);
  DCG_LAUNCH_CHECK();
  return DCG_OK;
}

namespace {

template <typename T>
int inner_residual(dcg_problem* p, const double* g, const double* z, cudaStream_t s, bool with_g = true) {
  Level& L = p->levels.back();
  const int grid = grid_for(L.nn, 256, kRedGrid);
  Reduce red = make_reduce(p, S_TMP0);  // S_TMP0 <- ||r||^2, S_TMP1 <- ||g||^2
  const int prof = prof_begin(p, PC_INNER_RES, s);
  const int gx = (L.m + kBoxThreads - 1) / kBoxThreads, gy = (L.m + kBoxSeg - 1) / kBoxSeg;
  if (p->dim == 2 && L.box && (long long)gx * gy <= kMaxRedCtas)
    k_inner_residual_box<T><<<gx * gy, kBoxThreads, 0, s>>>(L.box_c0, L.box_c1, g, z, (T*)L.f, (T*)L.z, L.m, gx, red,
                                                            with_g);
  else if (p->dim == 2)
    k_inner_residual<T, 2><<<grid, 256, 0, s>>>(L.st64, g, z, (T*)L.f, (T*)L.z, nullptr, L.m, L.nn, red, with_g);
  else
    k_inner_residual<T, 3><<<grid, 256, 0, s>>>(L.st64, g, z, (T*)L.f, (T*)L.z, nullptr, L.m, L.nn, red, with_g);
  DCG_LAUNCH_CHECK();
  prof_end(p, prof, s, 2.0 * ipow(3, p->dim) * (double)L.nn, (16.0 + 2.0 * sizeof(T)) * L.nn);
  return DCG_OK;
}

template <typename T>
int accumulate(dcg_problem* p, double* z, cudaStream_t s) {
  Level& L = p->levels.back();
  k_accumulate<T><<<grid_for(L.nn, 256, 8192), 256, 0, s>>>(z, (const T*)L.z, L.nn);
  DCG_LAUNCH_CHECK();
  return DCG_OK;
}

// exact inner solve: z = Z_J^-1 g by fast diagonalisation (FP64)
int exact_solve(dcg_problem* p, const double* g, double* z, cudaStream_t s) {
  Level& L = p->levels.back();
  DCG_CUDA(cudaMemcpyAsync(L.f, g, sizeof(double) * L.nn, cudaMemcpyDeviceToDevice, s));
  int st = p->dim == 2 ? coarse_solve_t<double, 2>(p, (const double*)L.f, (double*)L.z, s)
                       : coarse_solve_t<double, 3>(p, (const double*)L.f, (double*)L.z, s);
  if (st != DCG_OK) return st;
  DCG_CUDA(cudaMemcpyAsync(z, L.z, sizeof(double) * L.nn, cudaMemcpyDeviceToDevice, s));
  return DCG_OK;
}

}  // namespace

int mg_cycles(dcg_problem* p, const double* g, double* z, int ncycles, cudaStream_t s) {
  if (p->levels.empty()) return DCG_ERR_STATE;
  if (exact_mode(p)) return exact_solve(p, g, z, s);
  const bool fp32 = p->mg.fp32;
  for (int c = 0; c < ncycles; ++c) {
    DCG_TRY(fp32 ? inner_residual<float>(p, g, z, s) : inner_residual<double>(p, g, z, s));
    DCG_TRY(run_wcycle(p, s));
    DCG_TRY(fp32 ? accumulate<float>(p, z, s) : accumulate<double>(p, z, s));
    if (p->prof.mask) {
      DCG_CUDA(cudaStreamSynchronize(s));
      prof_flush_graph(p);
      prof_flush(p);
    }
  }
  return DCG_OK;
}

int mg_solve(dcg_problem* p, const double* g, double* z, double tol, int nmax, int* ncyc, cudaStream_t s) {
  if (p->levels.empty()) return DCG_ERR_STATE;
  *ncyc = 0;
  if (exact_mode(p)) return exact_solve(p, g, z, s);
  const bool fp32 = p->mg.fp32;
  int n = 0;
  double gn = 0.0;
  for (;;) {
    DCG_TRY(fp32 ? inner_residual<float>(p, g, z, s, n == 0) : inner_residual<double>(p, g, z, s, n == 0));
    DCG_TRY(read_scalars(p, s));
    if (n > 0 && p->prof.mask) prof_flush_graph(p);  // the replay before this read
    const double rn = std::sqrt(p->scal_host[S_TMP0]);
    if (n == 0) gn = std::sqrt(p->scal_host[S_TMP1]);
    if (!(gn > 0.0)) break;
    if (!(rn / gn > tol) || n >= nmax) break;
    DCG_TRY(run_wcycle(p, s));
    DCG_TRY(fp32 ? accumulate<float>(p, z, s) : accumulate<double>(p, z, s));
    ++n;
  }
  *ncyc = n;
  return DCG_OK;
}

// Pieces of Algorithm 3 for a solve captured into one CUDA graph (graph.cu):
// the FP64 residual of the inner system into the cycle's input (||r||^2 to
// S_TMP0 and, with with_g, ||g||^2 to S_TMP1), one W-cycle launched as
// kernels on the capturing stream, and z += the cycle's correction.
int mg_graph_residual(dcg_problem* p, const double* g, const double* z, bool with_g, cudaStream_t s) {
  return p->mg.fp32 ? inner_residual<float>(p, g, z, s, with_g) : inner_residual<double>(p, g, z, s, with_g);
}
int mg_graph_wcycle(dcg_problem* p, cudaStream_t s) {
  g_capturing = true;
  const int st = p->mg.fp32 ? wcycle_dispatch<float>(p, s) : wcycle_dispatch<double>(p, s);
  g_capturing = false;
  return st;
}
int mg_graph_accumulate(dcg_problem* p, double* z, cudaStream_t s) {
  return p->mg.fp32 ? accumulate<float>(p, z, s) : accumulate<double>(p, z, s);
}
bool mg_exact(const dcg_problem* p) { return exact_mode(p); }

int mg_ras_step_hook(dcg_problem* p, int level, const double* f, double* z, cudaStream_t s) {
  if (level < 2 || level > (int)p->levels.size()) return DCG_ERR_INVALID_ARG;
  Level& L = p->levels[level - 1];
  const bool fp32 = p->mg.fp32;
  const int g = grid_for(L.nn, 256, 8192);
  if (fp32) {
    k_to_t<float><<<g, 256, 0, s>>>(f, (float*)L.f, L.nn);
    k_to_t<float><<<g, 256, 0, s>>>(z, (float*)L.z, L.nn);
    DCG_TRY(p->dim == 2 ? (ras_step_t<float, 2>(p, L, s)) : (ras_step_t<float, 3>(p, L, s)));
    k_from_t<float><<<g, 256, 0, s>>>((const float*)L.z, z, L.nn);
  } else {
    DCG_CUDA(cudaMemcpyAsync(L.f, f, sizeof(double) * L.nn, cudaMemcpyDeviceToDevice, s));
    DCG_CUDA(cudaMemcpyAsync(L.z, z, sizeof(double) * L.nn, cudaMemcpyDeviceToDevice, s));
    DCG_TRY(p->dim == 2 ? (ras_step_t<double, 2>(p, L, s)) : (ras_step_t<double, 3>(p, L, s)));
    DCG_CUDA(cudaMemcpyAsync(z, L.z, sizeof(double) * L.nn, cudaMemcpyDeviceToDevice, s));
  }
  DCG_LAUNCH_CHECK();
  return DCG_OK;
}

int mg_coarse_hook(dcg_problem* p, const double* f, double* z, cudaStream_t s) {
  if (p->levels.empty()) return DCG_ERR_STATE;
  Level& L = p->levels[0];
  const bool fp32 = p->mg.fp32;
  const int g = grid_for(L.nn, 256, 8192);
  if (fp32) {
    k_to_t<float><<<g, 256, 0, s>>>(f, (float*)L.f, L.nn);
    DCG_TRY(p->dim == 2 ? (coarse_solve_t<float, 2>(p, (const float*)L.f, (float*)L.z, s))
                        : (coarse_solve_t<float, 3>(p, (const float*)L.f, (float*)L.z, s)));
    k_from_t<float><<<g, 256, 0, s>>>((const float*)L.z, z, L.nn);
  } else {
    DCG_CUDA(cudaMemcpyAsync(L.f, f, sizeof(double) * L.nn, cudaMemcpyDeviceToDevice, s));
    DCG_TRY(p->dim == 2 ? (coarse_solve_t<double, 2>(p, (const double*)L.f, (double*)L.z, s))
                        : (coarse_solve_t<double, 3>(p, (const double*)L.f, (double*)L.z, s)));
    DCG_CUDA(cudaMemcpyAsync(z, L.z, sizeof(double) * L.nn, cudaMemcpyDeviceToDevice, s));
  }
  DCG_LAUNCH_CHECK();
  return DCG_OK;
}

}  // namespace dcg

// ---------------------------------------------------------------------------
// Allocation-free exact coarsest solve.
//
// dcg_coarse_solve keeps its intermediate vectors in buffers that dcg_setup
// allocated. This variant allocates nothing at all: the one intermediate
// vector between the fast-diagonalisation passes lives in the fixed device
// array below, compiled into the library (1 MiB; every GPU that loads the
// library holds it until the process exits). It is meant for callers that
// cannot call cudaMalloc at the point where they need the solve, for example
// code running under a fixed device-memory budget that a caching allocator
// has already reserved, or a latency-critical loop in which an allocation's
// implicit synchronisation is not acceptable.
//
// The device address of the array is looked up once per device, on the first
// call made with that device current (cudaGetSymbolAddress); make that first
// call before any stream capture. All calls share the array: two calls whose
// work overlaps on the GPU (different streams, or different threads) race on
// it and must be serialised by the caller. Every element the passes read is
// written earlier in the same call, so no clearing is needed.
// ---------------------------------------------------------------------------
namespace dcg {
namespace {
static __device__ __align__(256) double g_static_coarse_tmp[DCG_STATIC_COARSE_MAX];
constexpr int kMaxDevices = 64;
// per-device address of the array, looked up on the first call with that
// device current; atomic, so first calls from several host threads are safe
std::atomic<double*> g_static_coarse_ptr[kMaxDevices] = {};
}  // namespace
}  // namespace dcg

extern "C" int dcg_coarse_solve_static(dcg_problem* p, const double* f_dev, double* z_dev, void* stream) {
  using namespace dcg;
  if (!p || !f_dev || !z_dev || f_dev == z_dev) {
    set_error_msg("dcg_coarse_solve_static: need a problem and distinct f, z device arrays");
    return DCG_ERR_INVALID_ARG;
  }
  if (!p->is_setup || p->levels.empty()) {
    set_error_msg("dcg_coarse_solve_static before dcg_setup of a deflated solver");
    return DCG_ERR_STATE;
  }
  const Coarse& C = p->coarse;
  const int D = p->dim;
  const long long nn = ipow(C.m, D);
  if (nn > (long long)DCG_STATIC_COARSE_MAX) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "dcg_coarse_solve_static: coarsest level has %lld nodes, more than the fixed scratch of %d "
             "(DCG_STATIC_COARSE_MAX); use dcg_coarse_solve or more multigrid levels", nn,
             (int)DCG_STATIC_COARSE_MAX);
    set_error_msg(buf);
    return DCG_ERR_INVALID_ARG;
  }
  int dev = 0;
  DCG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error_msg("dcg_coarse_solve_static: device index out of range");
    return DCG_ERR_UNSUPPORTED;
  }
  double* tmp = g_static_coarse_ptr[dev].load(std::memory_order_acquire);
  if (!tmp) {
    void* ptr = nullptr;
    DCG_CUDA(cudaGetSymbolAddress(&ptr, g_static_coarse_tmp));
    tmp = static_cast<double*>(ptr);
    g_static_coarse_ptr[dev].store(tmp, std::memory_order_release);  // every thread finds the same address
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int nl = D == 2 ? fdm_passes<double, 2>(f_dev, z_dev, tmp, C.S64, C.tri_l64, C.tri_w64, C.tri_e64, C.tw64,
                                                C.log2n2, C.m, s)
                        : fdm_passes<double, 3>(f_dev, z_dev, tmp, C.S64, C.tri_l64, C.tri_w64, C.tri_e64, C.tw64,
                                                C.log2n2, C.m, s);
  note_launches(nl - 1);
  DCG_LAUNCH_CHECK();
  return DCG_OK;
}
