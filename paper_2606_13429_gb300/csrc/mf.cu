// Matrix-free product with the 3D pseudo-stress operator
//
//   y = sum_e P_e^T [ (1/(nu_e dt)) M_e (x) D_3 + G_e ] P_e x
//
// (Section 3.1 block structure, forms of Section 3.2.1 on Q1 hexahedra; the
// element matrix couples the 8 nodes x 9 components of an element: the mass
// part M_e (x) D_3 scaled by the element's 1/nu, and the divergence part, in
// which component (k, p) of node a meets component (k, q) of node b through
// int d_p phi_a d_q phi_b.)
//
// The element sum is regrouped per output node (a gather: each node adds the
// contributions of its 8 elements, no atomics, deterministic):
//   * mass: y_a += D_3 (sum_o c_o x_{a+o}) / dt, c_o = W_o prod_ax (h/3 | h/6),
//     W_o = sum of 1/nu over the elements that hold both a and a+o;
//   * divergence: nu-independent, so its element sum is a constant 27-point
//     stencil per (p, q); the p != q stencils vanish where o_p = 0 or o_q = 0
//     (the two elements on either side cancel), and are skipped there.
// Nothing of A is stored: the kernel reads x, the per-element 1/nu and writes y.
//
// Layout: a CTA owns a 32 x 8 column of nodes and marches along z, keeping
// three z-planes of the operand (halo included, zero outside the interior
// grid) in shared memory, one array per component; each thread produces one
// node per plane. T is the arithmetic type (float for the FP32 variant, whose
// input and output stay FP64 in memory; double for the FP64 one). The
// operand, output and dot-product variants are those of the BSR product.
#include "common.cuh"

namespace dcg {
namespace {

// tile: 32 x MY nodes per CTA, MY = 8 for FP32 and 4 for FP64 (the three
// halo planes then take 37 KB and 44 KB of shared memory)
constexpr int kMX = 32, kPX = kMX + 2;
template <typename T>
__host__ __device__ constexpr int mf_my() {
  return sizeof(T) == 8 ? 4 : 8;
}

enum MfX { MX_X = 0, MX_X_MINUS_VZ = 1, MX_VZ = 2 };
enum MfO { MO_Y = 0, MO_FMY = 1, MO_VT = 2 };

struct MfArgs {
  const double* x;
  const double* zh;
  const double* f;
  double* y;
  const double* dvec;
  const double* inv_nu;  // per element (n^3), or null: inv_nu_const
  double inv_nu_const;
  double isd;
  int m, n;
  int tiles_x, tiles_y, zchunk;
  Reduce red;
  double mc64[27];      // h^3 prod(1/3 | 1/6) / dt per offset
  float mc32[27];
  double gs64[9][27];   // divergence stencil [p*3+q][offset]
  float gs32[9][27];
};

template <typename T>
__device__ __forceinline__ T mc_of(const MfArgs& A, int o);
template <>
__device__ __forceinline__ float mc_of<float>(const MfArgs& A, int o) { return A.mc32[o]; }
template <>
__device__ __forceinline__ double mc_of<double>(const MfArgs& A, int o) { return A.mc64[o]; }
template <typename T>
__device__ __forceinline__ T gs_of(const MfArgs& A, int pq, int o);
template <>
__device__ __forceinline__ float gs_of<float>(const MfArgs& A, int pq, int o) { return A.gs32[pq][o]; }
template <>
__device__ __forceinline__ double gs_of<double>(const MfArgs& A, int pq, int o) { return A.gs64[pq][o]; }

template <int XM>
__device__ __forceinline__ double operand(const MfArgs& A, long long a, int c) {
  const bool diag = (c & 3) == 0;  // components 0, 4, 8
  if (XM == MX_X) return __ldg(A.x + a * 9 + c);
  if (XM == MX_VZ) return diag ? A.isd * __ldg(A.zh + a) : 0.0;
  const double v = __ldg(A.x + a * 9 + c);
  return diag ? v - A.isd * __ldg(A.zh + a) : v;
}

template <typename T, int XM, int OM, bool DOT>
__global__ void __launch_bounds__(kMX * mf_my<T>()) k_mf(MfArgs A) {
  constexpr int kMY = mf_my<T>(), kMT = kMX * kMY, kPY = kMY + 2;
  __shared__ T pl[3][9][kPY][kPX];
  const int tx = threadIdx.x & (kMX - 1), ty = threadIdx.x / kMX;
  const int m = A.m;
  int b = blockIdx.x;
  const int bx = b % A.tiles_x;
  b /= A.tiles_x;
  const int by = b % A.tiles_y;
  const int bz = b / A.tiles_y;
  const int x0 = bx * kMX, y0 = by * kMY, z0 = bz * A.zchunk;
  const int z1 = min(m, z0 + A.zchunk);
  const int x = x0 + tx, y = y0 + ty;
  const bool own = x < m && y < m;
  // plane z of the operand into slot (z - z0 + 1) % 3; zero outside the grid
  auto load_plane = [&](int z) {
    const int slot = (z - z0 + 1) % 3;
    for (int t = threadIdx.x; t < kPY * kPX * 9; t += kMT) {
      const int row = t / (kPX * 9);
      const int j = t - row * (kPX * 9);
      const int node = j / 9, c = j - node * 9;
      const int gx = x0 - 1 + node, gy = y0 - 1 + row;
      T v = (T)0;
      if (z >= 0 && z < m && gx >= 0 && gx < m && gy >= 0 && gy < m)
        v = (T)operand<XM>(A, gx + (long long)m * (gy + (long long)m * z), c);
      pl[slot][c][row][node] = v;
    }
  };
  double part[1] = {0.0};
  load_plane(z0 - 1);
  load_plane(z0);
  for (int z = z0; z < z1; ++z) {
    load_plane(z + 1);
    __syncthreads();
    if (own) {
      // 1/nu of the 8 elements around the node: w[sz][sy][sx], element lower
      // corner at grid coordinate (interior index + s)
      T w[2][2][2];
#pragma unroll
      for (int sz = 0; sz < 2; ++sz)
#pragma unroll
        for (int sy = 0; sy < 2; ++sy)
#pragma unroll
          for (int sx = 0; sx < 2; ++sx) {
            const long long e = (x + sx) + (long long)A.n * ((y + sy) + (long long)A.n * (z + sz));
            w[sz][sy][sx] = A.inv_nu ? (T)__ldg(A.inv_nu + e) : (T)A.inv_nu_const;
          }
      // W over offsets: -1 -> element s = 0 only, 0 -> both, +1 -> s = 1 only
      T wx[2][2][3], wy[2][3][3], W[3][3][3];
#pragma unroll
      for (int sz = 0; sz < 2; ++sz)
#pragma unroll
        for (int sy = 0; sy < 2; ++sy) {
          wx[sz][sy][0] = w[sz][sy][0];
          wx[sz][sy][1] = w[sz][sy][0] + w[sz][sy][1];
          wx[sz][sy][2] = w[sz][sy][1];
        }
#pragma unroll
      for (int sz = 0; sz < 2; ++sz)
#pragma unroll
        for (int ox = 0; ox < 3; ++ox) {
          wy[sz][0][ox] = wx[sz][0][ox];
          wy[sz][1][ox] = wx[sz][0][ox] + wx[sz][1][ox];
          wy[sz][2][ox] = wx[sz][1][ox];
        }
#pragma unroll
      for (int oy = 0; oy < 3; ++oy)
#pragma unroll
        for (int ox = 0; ox < 3; ++ox) {
          W[0][oy][ox] = wy[0][oy][ox];
          W[1][oy][ox] = wy[0][oy][ox] + wy[1][oy][ox];
          W[2][oy][ox] = wy[1][oy][ox];
        }
      T ym[9], yg[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) ym[c] = yg[c] = (T)0;
#pragma unroll
      for (int oz = 0; oz < 3; ++oz) {
        const int slot = (z - z0 + oz) % 3;
#pragma unroll
        for (int oy = 0; oy < 3; ++oy)
#pragma unroll
          for (int ox = 0; ox < 3; ++ox) {
            const int o = ox + 3 * (oy + 3 * oz);
            const int oc[3] = {ox, oy, oz};
            T xn[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) xn[c] = pl[slot][c][ty + oy][tx + ox];
            const T cm = W[oz][oy][ox] * mc_of<T>(A, o);
#pragma unroll
            for (int c = 0; c < 9; ++c) ym[c] = fma(cm, xn[c], ym[c]);
#pragma unroll
            for (int p = 0; p < 3; ++p) {
              const T gpp = gs_of<T>(A, p * 3 + p, o);
#pragma unroll
              for (int k = 0; k < 3; ++k) yg[k * 3 + p] = fma(gpp, xn[k * 3 + p], yg[k * 3 + p]);
#pragma unroll
              for (int q = 0; q < 3; ++q) {
                if (q == p || oc[p] == 1 || oc[q] == 1) continue;  // cross stencil is zero there
                const T gpq = gs_of<T>(A, p * 3 + q, o);
#pragma unroll
                for (int k = 0; k < 3; ++k) yg[k * 3 + p] = fma(gpq, xn[k * 3 + q], yg[k * 3 + p]);
              }
            }
          }
      }
      // y = D_3 (mass sum) + divergence part; D_3 removes a third of the trace
      // from the diagonal components
      const T tr3 = (ym[0] + ym[4] + ym[8]) / (T)3;
      double out[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) out[c] = (double)(((c & 3) == 0 ? ym[c] - tr3 : ym[c]) + yg[c]);
      const long long a = x + (long long)m * (y + (long long)m * z);
      if (OM == MO_VT) {
        const double g = A.isd * (out[0] + out[4] + out[8]);
        A.y[a] = g;
        if (DOT) part[0] = fma(g, g, part[0]);
      } else {
#pragma unroll
        for (int c = 0; c < 9; ++c) {
          double v = out[c];
          if (OM == MO_FMY) v = A.f[a * 9 + c] - v;
          A.y[a * 9 + c] = v;
          if (DOT) part[0] = (OM == MO_FMY) ? fma(v, v, part[0]) : fma(A.dvec[a * 9 + c], v, part[0]);
        }
      }
    }
    __syncthreads();  // the next plane load overwrites slot (z - 1)
  }
  if (DOT) grid_reduce<1>(part, A.red);
}

// Host tables: divergence stencil and mass weights for mesh width h, step dt.
void build_tables(MfArgs& a, int n, double dt) {
  const double h = 1.0 / n;
  for (int o = 0; o < 27; ++o) {
    const int off[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
    double mc = 1.0 / dt;
    for (int ax = 0; ax < 3; ++ax) mc *= off[ax] == 0 ? h / 3.0 : h / 6.0;
    a.mc64[o] = mc;
    a.mc32[o] = (float)mc;
  }
  div_stencil(3, n, a.gs64);
  for (int pq = 0; pq < 9; ++pq)
    for (int o = 0; o < 27; ++o) a.gs32[pq][o] = (float)a.gs64[pq][o];
}

__global__ void k_unit(double* v, long long i) { v[i] = 1.0; }


// deterministic test pattern in [-1, 1)
__global__ void k_pattern_vec(double* v, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    v[i] = (double)((unsigned long long)(i * 2654435761ULL) % 1000ULL) / 500.0 - 1.0;
}

__global__ void k_sub_inplace(double* a, const double* b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    a[i] -= b[i];
}

template <typename T, int XM, int OM, bool DOT>
void launch_mf(MfArgs a, cudaStream_t s) {
  // z chunks: enough CTAs for every SM to hold several (two halo planes per chunk)
  a.tiles_x = (a.m + kMX - 1) / kMX;
  a.tiles_y = (a.m + mf_my<T>() - 1) / mf_my<T>();
  const long long cols = (long long)a.tiles_x * a.tiles_y;
  long long nzc = (4 * 152 + cols - 1) / cols;
  nzc = std::max(1LL, std::min(nzc, (long long)(a.m + 7) / 8));
  a.zchunk = (int)((a.m + nzc - 1) / nzc);
  nzc = (a.m + a.zchunk - 1) / a.zchunk;
  k_mf<T, XM, OM, DOT><<<(unsigned)(cols * nzc), kMX * mf_my<T>(), 0, s>>>(a);
}

}  // namespace

int mf_product(dcg_problem* p, int xm, int om, bool dot, bool lowp, const double* x, const double* zh,
               const double* f, double* y, const double* dvec, Reduce red, cudaStream_t s) {
  if (p->dim != 3) {
    set_error_msg("matrix-free product is implemented for 3D meshes");
    return DCG_ERR_UNSUPPORTED;
  }
  MfArgs a;
  a.x = x;
  a.zh = zh;
  a.f = f;
  a.y = y;
  a.dvec = dvec;
  a.inv_nu = p->inv_nu_elem;
  a.inv_nu_const = 1.0 / p->nu;
  a.isd = 1.0 / std::sqrt(3.0);
  a.m = p->m;
  a.n = p->n;
  a.red = red;
  build_tables(a, p->n, p->dt);
  // the fused reduction takes one partial per CTA; the grid has fewer than
  // (tile columns + 608) CTAs, tile columns at most ceil(m/32) ceil(m/4)
  const long long cols_max = (long long)((p->m + kMX - 1) / kMX) * ((p->m + 3) / 4);
  if (dot && cols_max + 608 > kMaxRedCtas) {
    set_error_msg("matrix-free product: grid too large for the fused reduction");
    return DCG_ERR_UNSUPPORTED;
  }
  // algorithmic work per node: 27 x 9 mass FMAs, 27 x 9 diagonal and
  // 6 x 12 x 3 cross divergence FMAs; bytes: operand, 1/nu (one element per
  // node), output, and f or dvec when read
  const double nn = (double)p->n_nodes;
  const double flops = 2.0 * (243 + 243 + 216) * nn;
  double bytes = (xm == MX_VZ ? 8.0 : 72.0) * nn + (xm == MX_X_MINUS_VZ ? 8.0 : 0.0) * nn;
  bytes += (p->inv_nu_elem ? 8.0 : 0.0) * nn + (om == MO_VT ? 8.0 : 72.0) * nn;
  if (om == MO_FMY || (dot && om == MO_Y)) bytes += 72.0 * nn;
  const int prof = prof_begin(p, PC_SPMV, s);
#define DCG_MF(T, XMV, OMV, DT) launch_mf<T, XMV, OMV, DT>(a, s)
#define DCG_MF_T(XMV, OMV, DT) \
  do {                          \
    if (lowp) DCG_MF(float, XMV, OMV, DT); \
    else DCG_MF(double, XMV, OMV, DT);     \
  } while (0)
  if (xm == MX_X && om == MO_Y && !dot) DCG_MF_T(MX_X, MO_Y, false);
  else if (xm == MX_X && om == MO_Y && dot) DCG_MF_T(MX_X, MO_Y, true);
  else if (xm == MX_X && om == MO_FMY) DCG_MF_T(MX_X, MO_FMY, true);
  else if (xm == MX_X && om == MO_VT) DCG_MF_T(MX_X, MO_VT, true);
  else if (xm == MX_VZ && om == MO_Y) DCG_MF_T(MX_VZ, MO_Y, false);
  else if (xm == MX_VZ && om == MO_FMY) DCG_MF_T(MX_VZ, MO_FMY, true);
  else if (xm == MX_VZ && om == MO_VT) DCG_MF_T(MX_VZ, MO_VT, true);
  else if (xm == MX_X_MINUS_VZ && om == MO_Y) DCG_MF_T(MX_X_MINUS_VZ, MO_Y, true);
  else {
    set_error_msg("matrix-free product: unsupported operand/output combination");
    return DCG_ERR_UNSUPPORTED;
  }
#undef DCG_MF_T
#undef DCG_MF
  DCG_LAUNCH_CHECK();
  prof_end(p, prof, s, flops, bytes);
  return DCG_OK;
}

// Z_J = V^T A V read off the operator: the column of a unit vector at an
// interior node whose 27 neighbours are all interior (Z_J is symmetric, so the
// column is the row's stencil).
int mf_probe_stencil(dcg_problem* p, double* stencil, cudaStream_t s) {
  const long long nn = p->n_nodes, m = p->m;
  double *e = nullptr, *g = nullptr;
  if (cudaMalloc(&e, sizeof(double) * nn) != cudaSuccess || cudaMalloc(&g, sizeof(double) * nn) != cudaSuccess) {
    cudaFree(e);
    set_error_msg("matrix-free setup: probe allocation failed");
    return DCG_ERR_OOM;
  }
  const long long c = 1 + m * (1 + m);
  int st = DCG_OK;
  if (cudaMemsetAsync(e, 0, sizeof(double) * nn, s) != cudaSuccess) st = DCG_ERR_CUDA;
  if (st == DCG_OK) {
    k_unit<<<1, 1, 0, s>>>(e, c);
    st = mf_product(p, MX_VZ, MO_VT, true, false, nullptr, e, nullptr, g, nullptr, make_reduce(p, S_TMP0), s);
  }
  for (int o = 0; o < 27 && st == DCG_OK; ++o) {
    const long long nb = c + (o % 3 - 1) + m * ((o / 3) % 3 - 1) + m * m * (o / 9 - 1);
    if (cudaMemcpyAsync(stencil + o, g + nb, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      st = DCG_ERR_CUDA;
  }
  if (st == DCG_OK && cudaStreamSynchronize(s) != cudaSuccess) st = DCG_ERR_CUDA;
  if (st == DCG_ERR_CUDA) set_error("matrix-free stencil probe", cudaGetLastError());
  cudaFree(e);
  cudaFree(g);
  return st;
}

// V^T A V z (matrix-free, FP64) against the level-J stencil on a full test
// vector: the probe's stencil must hold for every row (boundary rows too).
int mf_check_stencil(dcg_problem* p, cudaStream_t s) {
  const long long nn = p->n_nodes;
  double *z = nullptr, *y1 = nullptr, *y2 = nullptr;
  if (cudaMalloc(&z, sizeof(double) * nn) != cudaSuccess || cudaMalloc(&y1, sizeof(double) * nn) != cudaSuccess ||
      cudaMalloc(&y2, sizeof(double) * nn) != cudaSuccess) {
    cudaFree(z);
    cudaFree(y1);
    set_error_msg("matrix-free setup: check allocation failed");
    return DCG_ERR_OOM;
  }
  const int g = grid_for(nn, 256, 4096);
  k_pattern_vec<<<g, 256, 0, s>>>(z, nn);
  int st = mf_product(p, MX_VZ, MO_VT, true, false, nullptr, z, nullptr, y1, nullptr, make_reduce(p, S_TMP0), s);
  if (st == DCG_OK) st = mg_inner_apply(p, z, y2, s);
  if (st == DCG_OK) {
    k_sub_inplace<<<g, 256, 0, s>>>(y1, y2, nn);
    st = vec_dot(p, y1, y1, nn, S_TMP0, s);
  }
  if (st == DCG_OK) st = vec_dot(p, y2, y2, nn, S_TMP1, s);
  if (st == DCG_OK) st = read_scalars(p, s);
  cudaFree(z);
  cudaFree(y1);
  cudaFree(y2);
  if (st != DCG_OK) return st;
  const double dev = std::sqrt(p->scal_host[S_TMP0]), ref = std::sqrt(p->scal_host[S_TMP1]);
  if (!(dev <= 1e-12 * ref)) {
    char buf[160];
    snprintf(buf, sizeof buf, "matrix-free V^T A V differs from its probed stencil (relative %.3e)", dev / ref);
    set_error_msg(buf);
    return DCG_ERR_UNSUPPORTED;
  }
  return DCG_OK;
}

}  // namespace dcg
