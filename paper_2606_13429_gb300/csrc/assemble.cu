// Assembly of A = (1/dt) M_dev + K_div in BSR form on the device.
//
// Forms: Section 2.3 Eq. component_form with the conforming scalar forms of
// Section 3.2.1 (m(s,t) = int s t, a_ij(s,t) = int d_i s d_j t) on Q1 nodal
// elements; block structure of Section 3.1 (M = D_d kron M1, A_div = I_d kron
// C_d). Block between interior nodes a (row) and c (column):
//   A_ac = (1/dt) mt_ac D_d + kron(I_d, G_ac),
//   mt_ac = sum_e nu_e^-1 int_e phi_a phi_c,  (G_ac)_pq = int d_p phi_a d_q phi_c.
// The mass part is formed as off = -(mt/dt)/d, diag = -(d-1) off so that
// M_dev V = 0 holds exactly in floating point.
//
// Pattern: one block per pair of nodes sharing an element (3^d neighbourhood
// clipped at the eliminated boundary), columns ascending. Element sums run
// over the shared elements in ascending element index with explicit
// round-to-nearest multiplies and adds (no contraction), so values are
// reproducible bit for bit.
#include "common.cuh"

namespace dcg {
namespace {

template <int D>
__device__ __forceinline__ void node_coords(long long a, int m, int (&c)[3]) {
  c[0] = (int)(a % m);
  c[1] = D > 1 ? (int)((a / m) % m) : 0;
  c[2] = D > 2 ? (int)(a / ((long long)m * m)) : 0;
}

// number of valid neighbour offsets along an axis for coordinate i
__device__ __forceinline__ int axis_count(int i, int m) {
  return 1 + (i > 0) + (i < m - 1);
}
// prefix of axis_count over indices < i
__device__ __forceinline__ long long axis_prefix(int i, int m) {
  if (i == 0) return 0;
  // index 0 has (m > 1 ? 2 : 1); indices 1..i-1 have 3 (if < m-1)
  long long first = (m > 1) ? 2 : 1;
  return first + 3LL * (i - 1);
}

template <int D>
__global__ void k_pattern(int m, long long n_nodes, int* __restrict__ row_ptr, int* __restrict__ col_idx) {
  long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (a >= n_nodes) return;
  int c[3];
  node_coords<D>(a, m, c);
  const long long T = 3LL * m - 2;  // blocks per axis line total
  long long start;
  if (D == 2) {
    start = axis_prefix(c[1], m) * T + axis_count(c[1], m) * axis_prefix(c[0], m);
  } else {
    start = axis_prefix(c[2], m) * T * T +
            axis_count(c[2], m) * (axis_prefix(c[1], m) * T + axis_count(c[1], m) * axis_prefix(c[0], m));
  }
  row_ptr[a] = (int)start;
  if (a == n_nodes - 1) {
    long long tot = 1;
    for (int k = 0; k < D; ++k) tot *= T;
    row_ptr[n_nodes] = (int)tot;
  }
  long long s = start;
  for (int dz = (D > 2 ? -1 : 0); dz <= (D > 2 ? 1 : 0); ++dz) {
    int z = c[2] + dz;
    if (D > 2 && (z < 0 || z >= m)) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      int y = c[1] + dy;
      if (y < 0 || y >= m) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        int x = c[0] + dx;
        if (x < 0 || x >= m) continue;
        long long lin = x + (long long)m * y + (D > 2 ? (long long)m * m * z : 0);
        col_idx[s++] = (int)lin;
      }
    }
  }
}

struct Elem1D {
  double M[2][2];  // int psi_a psi_b
  double K[2][2];  // int psi_a' psi_b'
  double C[2][2];  // int psi_a' psi_b
};

__device__ __forceinline__ Elem1D elem1d(int n) {
  Elem1D e;
  const double h = 1.0 / (double)n;
  const double hs = h / 6.0;
  const double ih = 1.0 / h;
  e.M[0][0] = __dmul_rn(hs, 2.0); e.M[1][1] = e.M[0][0];
  e.M[0][1] = hs; e.M[1][0] = hs;
  e.K[0][0] = ih; e.K[1][1] = ih; e.K[0][1] = -ih; e.K[1][0] = -ih;
  e.C[0][0] = -0.5; e.C[0][1] = -0.5; e.C[1][0] = 0.5; e.C[1][1] = 0.5;
  return e;
}

// One thread per (node, neighbour offset); writes the b*b block values.
template <int D>
__global__ void k_values(int n, int m, long long n_nodes, double dt, double inv_nu_const,
                         const double* __restrict__ inv_nu_elem, const int* __restrict__ row_ptr,
                         double* __restrict__ vals) {
  constexpr int NOFF = D == 2 ? 9 : 27;
  constexpr int B = D * D;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n_nodes * NOFF) return;
  const long long a = t / NOFF;
  const int o = (int)(t % NOFF);
  int off[3] = {o % 3 - 1, (o / 3) % 3 - 1, D > 2 ? o / 9 - 1 : 0};
  int ca[3];
  node_coords<D>(a, m, ca);
  int cc[3];
  for (int k = 0; k < 3; ++k) cc[k] = ca[k] + off[k];
  for (int k = 0; k < D; ++k)
    if (cc[k] < 0 || cc[k] >= m) return;
  // slot = row_ptr[a] + rank of this offset among the valid ones (ascending)
  int rank = 0;
  for (int q = 0; q < o; ++q) {
    int qo[3] = {q % 3 - 1, (q / 3) % 3 - 1, D > 2 ? q / 9 - 1 : 0};
    bool ok = true;
    for (int k = 0; k < D; ++k) {
      int v = ca[k] + qo[k];
      ok = ok && (v >= 0 && v < m);
    }
    rank += ok;
  }
  const long long slot = (long long)row_ptr[a] + rank;

  const Elem1D e1 = elem1d(n);
  // grid coordinates (1..m) of the two nodes
  int ga[3], gc[3], elo[3], ehi[3];
  for (int k = 0; k < 3; ++k) {
    ga[k] = ca[k] + 1;
    gc[k] = cc[k] + 1;
    int hi = ga[k] < gc[k] ? ga[k] : gc[k];
    int lo = (ga[k] > gc[k] ? ga[k] : gc[k]) - 1;
    elo[k] = lo;
    ehi[k] = hi;
  }
  if (D == 2) { elo[2] = 0; ehi[2] = 0; ga[2] = gc[2] = 0; }
  double mt = 0.0;
  double G[D][D];
#pragma unroll
  for (int p = 0; p < D; ++p)
#pragma unroll
    for (int q = 0; q < D; ++q) G[p][q] = 0.0;

  for (int ez = elo[2]; ez <= ehi[2]; ++ez)
    for (int ey = elo[1]; ey <= ehi[1]; ++ey)
      for (int ex = elo[0]; ex <= ehi[0]; ++ex) {
        int ec[3] = {ex, ey, ez};
        int la[3], lc[3];
        for (int k = 0; k < 3; ++k) { la[k] = ga[k] - ec[k]; lc[k] = gc[k] - ec[k]; }
        long long elin = ex + (long long)n * ey + (D > 2 ? (long long)n * n * ez : 0);
        const double w = inv_nu_elem ? inv_nu_elem[elin] : inv_nu_const;
        // element mass: product of 1D factors in axis order
        double me = e1.M[la[0]][lc[0]];
#pragma unroll
        for (int k = 1; k < D; ++k) me = __dmul_rn(me, e1.M[la[k]][lc[k]]);
        mt = __dadd_rn(mt, __dmul_rn(w, me));
#pragma unroll
        for (int p = 0; p < D; ++p)
#pragma unroll
          for (int q = 0; q < D; ++q) {
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
              double f;
              if (k == p && k == q) f = e1.K[la[k]][lc[k]];
              else if (k == p) f = e1.C[la[k]][lc[k]];
              else if (k == q) f = e1.C[lc[k]][la[k]];
              else f = e1.M[la[k]][lc[k]];
              v = (k == 0) ? f : __dmul_rn(v, f);
            }
            G[p][q] = __dadd_rn(G[p][q], v);
          }
      }
  // block values
  const double c = mt / dt;
  const double offv = -c / (double)D;
  const double dg = __dmul_rn(-(double)(D - 1), offv);
  double* blk = vals + slot * (long long)(B * B);
#pragma unroll
  for (int r = 0; r < B; ++r) {
    const int k = r / D, i = r % D;
#pragma unroll
    for (int col = 0; col < B; ++col) {
      const int l = col / D, j = col % D;
      double mv = 0.0;
      if (k == i) {
        if (l == j) mv = (l == k) ? dg : offv;
      } else if (col == r) {
        mv = c;
      }
      double v = mv;
      if (k == l) v = __dadd_rn(mv, G[i][j]);
      blk[r * B + col] = v;
    }
  }
}

}  // namespace

int assemble_device(dcg_problem* p, const double* nu_elem_host, cudaStream_t s) {
  const int D = p->dim;
  const long long nn = p->n_nodes;
  const int threads = 256;
  long long n_elem = 1;
  for (int k = 0; k < D; ++k) n_elem *= p->n;
  if (nu_elem_host) {
    DCG_CUDA(cudaMalloc(&p->inv_nu_elem, sizeof(double) * n_elem));
    std::vector<double> inv(n_elem);
    for (long long e = 0; e < n_elem; ++e) inv[e] = 1.0 / nu_elem_host[e];
    DCG_CUDA(cudaMemcpyAsync(p->inv_nu_elem, inv.data(), sizeof(double) * n_elem, cudaMemcpyHostToDevice, s));
    DCG_CUDA(cudaStreamSynchronize(s));
  }
  if (p->matrix_free) return DCG_OK;
  DCG_CUDA(cudaMalloc(&p->row_ptr, sizeof(int) * (nn + 1)));
  // four spare entries: bulk copies of a column range start and end on
  // 16-byte boundaries and may read up to three entries past the last one
  DCG_CUDA(cudaMalloc(&p->col_idx, sizeof(int) * (p->nnzb + 4)));
  DCG_CUDA(cudaMemsetAsync(p->col_idx + p->nnzb, 0, sizeof(int) * 4, s));
  DCG_CUDA(cudaMalloc(&p->vals, sizeof(double) * p->nnzb * p->b * p->b));
  int g = (int)((nn + threads - 1) / threads);
  if (D == 2) k_pattern<2><<<g, threads, 0, s>>>(p->m, nn, p->row_ptr, p->col_idx);
  else k_pattern<3><<<g, threads, 0, s>>>(p->m, nn, p->row_ptr, p->col_idx);
  DCG_LAUNCH_CHECK();
  const int noff = D == 2 ? 9 : 27;
  long long work = nn * noff;
  long long gv = (work + threads - 1) / threads;
  const double inv_nu = 1.0 / p->nu;
  if (D == 2)
    k_values<2><<<(unsigned)gv, threads, 0, s>>>(p->n, p->m, nn, p->dt, inv_nu, p->inv_nu_elem, p->row_ptr, p->vals);
  else
    k_values<3><<<(unsigned)gv, threads, 0, s>>>(p->n, p->m, nn, p->dt, inv_nu, p->inv_nu_elem, p->row_ptr, p->vals);
  DCG_LAUNCH_CHECK();
  return DCG_OK;
}

}  // namespace dcg
