"""Q1 nodal discretisation of the pseudo-stress system (oracle, FP64).

Test infrastructure only (see the package docstring).

Problem (Section 2.3, Eq. weak_IE and Eq. component_form; Section 3, Eq.
pb_study): for one implicit-Euler step the matrix is ``A* = M + dt*A_div``.
This module assembles the same system divided by dt,

    A = (1/dt) * M_dev + K_div,

which has the same solution and the same CG iterates for a relative tolerance.
Each of the d*d tensor components is a continuous Q1 nodal field on the
uniform mesh of [0,1]^d with n elements per side; all boundary nodes are
eliminated (homogeneous Dirichlet), leaving m = n-1 interior nodes per axis.

Scalar forms (Section 3.2.1, conforming Galerkin): m(s,t) = int s*t and
a_ij(s,t) = int d_i s * d_j t. The viscosity enters M_dev only, as 1/nu
(Section 2.2, form M), elementwise when nu is given per element.

Unknown ordering: node-major. Interior nodes lexicographic with x fastest;
per node the d*d components in the paper's row-major order
[s11 s12 (s13) s21 s22 ... sdd] (Section 3.1, the vectors printed for d=2, 3).
The paper stacks component-major (kron(v, I)); node-major is a fixed
permutation of it.

Block of the matrix between interior nodes a (row) and b (column):

    A_ab = (1/dt) * mt_ab * D_d + kron(I_d, G_ab),
    mt_ab = sum_e nu_e^-1 int_e phi_a phi_b,
    (G_ab)_pq = int d_p phi_a d_q phi_b,
    D_d = I - (1/d) v v^T,  v = indicator of the diagonal components,

D_d being the matrices printed in Section 3.1 for d = 2 and d = 3. Blocks are
stored for every pair of nodes that share an element (the 3^d neighbourhood,
clipped at the boundary), columns ascending, numerical zeros kept.

Exactness rule (a reading; the paper is silent on rounding): the mass part of
a block is formed from c = mt_ab/dt as off = -c/d and diag = -(d-1)*off, so
that M_dev * V = 0 holds bit for bit.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

# ---------------------------------------------------------------------------
# 1D Q1 element integrals on [0, h]: psi_0 = 1 - x/h, psi_1 = x/h.
# ---------------------------------------------------------------------------


def mass_1d(h: float) -> np.ndarray:
    """int psi_a psi_b over [0,h]."""
    return (h / 6.0) * np.array([[2.0, 1.0], [1.0, 2.0]])


def stiff_1d(h: float) -> np.ndarray:
    """int psi_a' psi_b' over [0,h]."""
    return (1.0 / h) * np.array([[1.0, -1.0], [-1.0, 1.0]])


def mixed_1d(h: float) -> np.ndarray:
    """int psi_a' psi_b over [0,h] (row index carries the derivative)."""
    del h  # psi' = +-1/h, int psi = h/2: the product does not depend on h
    return np.array([[-0.5, -0.5], [0.5, 0.5]])


def local_bits(d: int) -> np.ndarray:
    """Local node a of a Q1 element has corner bits (a_0, ..., a_{d-1}),
    a = a_0 + 2 a_1 + 4 a_2. Returns array (2^d, d)."""
    return np.array([[(a >> ax) & 1 for ax in range(d)] for a in range(2 ** d)], dtype=np.int64)


def element_mass(d: int, h: float) -> np.ndarray:
    """Q1 element mass matrix int phi_a phi_b, closed form as a tensor product."""
    M1 = mass_1d(h)
    bits = local_bits(d)
    nl = 2 ** d
    out = np.ones((nl, nl))
    for a in range(nl):
        for b in range(nl):
            v = 1.0
            for ax in range(d):
                v = v * M1[bits[a, ax], bits[b, ax]]
            out[a, b] = v
    return out


def element_grad(d: int, h: float) -> np.ndarray:
    """G[p, q, a, b] = int d_p phi_a d_q phi_b on one element, closed form as
    a tensor product of 1D factors (factors multiplied in axis order)."""
    M1, K1, C1 = mass_1d(h), stiff_1d(h), mixed_1d(h)
    bits = local_bits(d)
    nl = 2 ** d
    out = np.zeros((d, d, nl, nl))
    for p in range(d):
        for q in range(d):
            for a in range(nl):
                for b in range(nl):
                    v = 1.0
                    for ax in range(d):
                        ia, ib = bits[a, ax], bits[b, ax]
                        if ax == p and ax == q:
                            f = K1[ia, ib]
                        elif ax == p:
                            f = C1[ia, ib]  # int psi_a' psi_b
                        elif ax == q:
                            f = C1[ib, ia]  # int psi_a psi_b'
                        else:
                            f = M1[ia, ib]
                        v = v * f
                    out[p, q, a, b] = v
    return out


def element_matrices_quadrature(d: int, h: float):
    """Same element integrals by 2-point Gauss quadrature per axis (exact for
    polynomials of degree <= 3 per axis; the integrands have degree <= 2).
    Independent of the tensor-product closed forms above."""
    g = 1.0 / math.sqrt(3.0)
    pts1 = np.array([0.5 * h * (1 - g), 0.5 * h * (1 + g)])
    w1 = np.array([0.5 * h, 0.5 * h])
    bits = local_bits(d)
    nl = 2 ** d
    mass = np.zeros((nl, nl))
    grad = np.zeros((d, d, nl, nl))
    for qi in np.ndindex(*([2] * d)):
        x = np.array([pts1[i] for i in qi])
        w = np.prod([w1[i] for i in qi])
        phi = np.zeros(nl)
        dphi = np.zeros((d, nl))
        for a in range(nl):
            vals = [(x[ax] / h) if bits[a, ax] else (1.0 - x[ax] / h) for ax in range(d)]
            ders = [(1.0 / h) if bits[a, ax] else (-1.0 / h) for ax in range(d)]
            phi[a] = np.prod(vals)
            for p in range(d):
                dphi[p, a] = np.prod([ders[ax] if ax == p else vals[ax] for ax in range(d)])
        mass += w * np.outer(phi, phi)
        for p in range(d):
            for q in range(d):
                grad[p, q] += w * np.outer(dphi[p], dphi[q])
    return mass, grad


# ---------------------------------------------------------------------------
# Deviatoric matrix D_d and deflation vector v (Section 3.1).
# ---------------------------------------------------------------------------


def diag_components(d: int) -> list[int]:
    """Positions j = (i-1)d + i (1-based) of sigma_ii in a node's block, 0-based."""
    return [i * d + i for i in range(d)]


def dev_matrix(d: int) -> np.ndarray:
    """D_d = I - (1/d) v v^T (the matrices printed in Section 3.1)."""
    v = np.zeros(d * d)
    v[diag_components(d)] = 1.0
    return np.eye(d * d) - np.outer(v, v) / d


# ---------------------------------------------------------------------------
# Mesh numbering and BSR pattern.
# ---------------------------------------------------------------------------


@dataclass
class Mesh:
    d: int
    n: int

    @property
    def m(self) -> int:
        return self.n - 1

    @property
    def h(self) -> float:
        return 1.0 / self.n

    @property
    def n_nodes(self) -> int:
        return self.m ** self.d

    @property
    def n_elem(self) -> int:
        return self.n ** self.d

    @property
    def b(self) -> int:
        return self.d * self.d

    @property
    def n_unknowns(self) -> int:
        return self.b * self.n_nodes


def node_coords(mesh: Mesh) -> np.ndarray:
    """(n_nodes, d) interior coordinates, x fastest."""
    m, d = mesh.m, mesh.d
    idx = np.arange(mesh.n_nodes, dtype=np.int64)
    return np.stack([(idx // (m ** ax)) % m for ax in range(d)], axis=1)


def bsr_pattern(mesh: Mesh):
    """Block pattern by the neighbour rule: node a couples node b iff
    |a_ax - b_ax| <= 1 on every axis. Columns ascending. int32 arrays."""
    d, m = mesh.d, mesh.m
    coords = node_coords(mesh)
    offsets = [np.array(o[::-1]) for o in np.ndindex(*([3] * d))]  # last axis slowest -> ascending
    cols = []
    for off in offsets:
        off = off - 1
        c = coords + off[None, :]
        ok = np.all((c >= 0) & (c < m), axis=1)
        lin = np.zeros(mesh.n_nodes, dtype=np.int64)
        for ax in range(d):
            lin += c[:, ax] * (m ** ax)
        cols.append(np.where(ok, lin, -1))
    cols = np.stack(cols, axis=1)  # (n_nodes, 3^d), ascending where valid
    valid = cols >= 0
    counts = valid.sum(axis=1)
    row_ptr = np.zeros(mesh.n_nodes + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col_idx = cols[valid]
    return row_ptr.astype(np.int32), col_idx.astype(np.int32)


def element_nodes(mesh: Mesh) -> np.ndarray:
    """(n_elem, 2^d) interior node index of each local node, -1 if the local
    node lies on the boundary (eliminated). Elements lexicographic, x fastest."""
    d, n, m = mesh.d, mesh.n, mesh.m
    e = np.arange(mesh.n_elem, dtype=np.int64)
    ecoord = np.stack([(e // (n ** ax)) % n for ax in range(d)], axis=1)
    bits = local_bits(d)
    out = np.empty((mesh.n_elem, 2 ** d), dtype=np.int64)
    for a in range(2 ** d):
        g = ecoord + bits[a][None, :]  # grid point in [0, n]
        inside = np.all((g >= 1) & (g <= n - 1), axis=1)
        lin = np.zeros(mesh.n_elem, dtype=np.int64)
        for ax in range(d):
            lin += (g[:, ax] - 1) * (m ** ax)
        out[:, a] = np.where(inside, lin, -1)
    return out


# ---------------------------------------------------------------------------
# Assembly.
# ---------------------------------------------------------------------------


@dataclass
class Assembled:
    mesh: Mesh
    dt: float
    row_ptr: np.ndarray  # int32 (n_nodes+1)
    col_idx: np.ndarray  # int32 (nnzb)
    values: np.ndarray   # float64 (nnzb, b, b), row-major blocks
    mt: np.ndarray       # float64 (nnzb): sum_e nu_e^-1 int phi_a phi_b
    G: np.ndarray        # float64 (nnzb, d, d): int d_p phi_a d_q phi_b

    def matrix(self) -> sp.bsr_matrix:
        b = self.mesh.b
        nb = self.mesh.n_nodes
        return sp.bsr_matrix((self.values, self.col_idx.astype(np.int64), self.row_ptr.astype(np.int64)),
                             shape=(nb * b, nb * b))


def _slot_of(row_ptr, col_idx, n_nodes, rows, cols):
    keys = np.repeat(np.arange(n_nodes, dtype=np.int64), np.diff(row_ptr.astype(np.int64))) * n_nodes \
        + col_idx.astype(np.int64)
    q = rows * n_nodes + cols
    s = np.searchsorted(keys, q)
    assert np.all(keys[s] == q), "contribution outside the neighbour pattern"
    return s


def assemble_scalar_forms(mesh: Mesh, nu: float = 1.0, nu_elem: np.ndarray | None = None):
    """Per pattern slot: mt (weighted mass) and G (gradient pairs), summing the
    element contributions in element order."""
    d = mesh.d
    row_ptr, col_idx = bsr_pattern(mesh)
    Me = element_mass(d, mesh.h)
    Ge = element_grad(d, mesh.h)
    en = element_nodes(mesh)  # (E, nl)
    nl = 2 ** d
    inv_nu = (1.0 / nu) * np.ones(mesh.n_elem) if nu_elem is None else 1.0 / np.asarray(nu_elem, dtype=np.float64)
    # contributions element-major: (E, nl, nl)
    A_idx = np.broadcast_to(en[:, :, None], (mesh.n_elem, nl, nl))
    B_idx = np.broadcast_to(en[:, None, :], (mesh.n_elem, nl, nl))
    keep = (A_idx >= 0) & (B_idx >= 0)
    rows = A_idx[keep]
    cols = B_idx[keep]
    slot = _slot_of(row_ptr, col_idx, mesh.n_nodes, rows, cols)
    nnzb = col_idx.shape[0]
    mcontrib = (inv_nu[:, None, None] * Me[None, :, :])
    mcontrib = np.broadcast_to(mcontrib, (mesh.n_elem, nl, nl))[keep]
    mt = np.bincount(slot, weights=mcontrib, minlength=nnzb)
    G = np.zeros((nnzb, d, d))
    for p in range(d):
        for q in range(d):
            gc = np.broadcast_to(Ge[p, q][None, :, :], (mesh.n_elem, nl, nl))[keep]
            G[:, p, q] = np.bincount(slot, weights=gc, minlength=nnzb)
    return row_ptr, col_idx, mt, G


def blocks_from_forms(d: int, dt: float, mt: np.ndarray, G: np.ndarray,
                      mass: bool = True, div: bool = True) -> np.ndarray:
    """A_ab = (1/dt) mt_ab D_d + kron(I_d, G_ab) per slot (exactness rule for
    the mass part; see module docstring)."""
    nnzb = mt.shape[0]
    b = d * d
    vals = np.zeros((nnzb, b, b))
    diagc = diag_components(d)
    if mass:
        c = mt / dt
        off = -c / d
        dg = -(d - 1) * off
        for k in range(d):
            for i in range(d):
                r = k * d + i
                if k == i:
                    for l in range(d):
                        col = diagc[l]
                        vals[:, r, col] = dg if l == k else off
                else:
                    vals[:, r, r] = c
    if div:
        for k in range(d):
            for p in range(d):
                for q in range(d):
                    vals[:, k * d + p, k * d + q] = vals[:, k * d + p, k * d + q] + G[:, p, q]
    return vals


def assemble(d: int, n: int, dt: float, nu: float = 1.0, nu_elem=None,
             mass: bool = True, div: bool = True) -> Assembled:
    """Assemble A = (1/dt) M_dev + K_div in BSR form."""
    if n < 2 or dt <= 0 or nu <= 0:
        raise ValueError("need n >= 2, dt > 0, nu > 0")
    mesh = Mesh(d, n)
    row_ptr, col_idx, mt, G = assemble_scalar_forms(mesh, nu, nu_elem)
    vals = blocks_from_forms(d, dt, mt, G, mass=mass, div=div)
    return Assembled(mesh, dt, row_ptr, col_idx, vals, mt, G)


def apply_elementwise(mesh: Mesh, dt: float, x: np.ndarray, nu: float = 1.0, nu_elem=None) -> np.ndarray:
    """y = sum_e P_e^T A_e P_e x, element by element (no assembled matrix):
    an independent route to A x, used to pin the assembled SpMV."""
    d, b = mesh.d, mesh.b
    Me = element_mass(d, mesh.h)
    Ge = element_grad(d, mesh.h)
    D = dev_matrix(d)
    en = element_nodes(mesh)
    inv_nu = (1.0 / nu) * np.ones(mesh.n_elem) if nu_elem is None else 1.0 / np.asarray(nu_elem)
    X = x.reshape(mesh.n_nodes, b)
    Y = np.zeros_like(X)
    nl = 2 ** d
    # element matrix (nl*b x nl*b) without nu: mass part and grad part
    Km = np.einsum("ab,rc->arbc", Me, D).reshape(nl * b, nl * b) / dt
    Kg = np.zeros((nl, b, nl, b))
    for k in range(d):
        for p in range(d):
            for q in range(d):
                Kg[:, k * d + p, :, k * d + q] = Ge[p, q]
    Kg = Kg.reshape(nl * b, nl * b)
    Xe = np.where(en[:, :, None] >= 0, X[np.maximum(en, 0)], 0.0).reshape(mesh.n_elem, nl * b)
    Ye = inv_nu[:, None] * (Xe @ Km.T) + Xe @ Kg.T
    Ye = Ye.reshape(mesh.n_elem, nl, b)
    for a in range(nl):
        ok = en[:, a] >= 0
        np.add.at(Y, en[ok, a], Ye[ok, a])
    return Y.reshape(-1)


def rows_of_Ax(mesh: Mesh, dt: float, x: np.ndarray, nodes: np.ndarray, nu: float = 1.0, nu_elem=None) -> np.ndarray:
    """Block rows `nodes` of A x, one node at a time from its (at most 2^d)
    elements: lets a full-size product be checked on sampled rows."""
    d, b, n, m = mesh.d, mesh.b, mesh.n, mesh.m
    Me = element_mass(d, mesh.h)
    Ge = element_grad(d, mesh.h)
    D = dev_matrix(d)
    bits = local_bits(d)
    X = x.reshape(mesh.n_nodes, b)
    out = np.zeros((len(nodes), b))
    for t, a_lin in enumerate(np.asarray(nodes, dtype=np.int64)):
        ac = np.array([(a_lin // (m ** ax)) % m for ax in range(d)]) + 1  # grid coords
        y = np.zeros(b)
        for la in range(2 ** d):
            ec = ac - bits[la]
            if np.any(ec < 0) or np.any(ec >= n):
                continue
            e_lin = int(sum(ec[ax] * n ** ax for ax in range(d)))
            w = (1.0 / nu) if nu_elem is None else 1.0 / nu_elem[e_lin]
            for lb in range(2 ** d):
                g = ec + bits[lb]
                if np.any(g < 1) or np.any(g > n - 1):
                    continue
                b_lin = int(sum((g[ax] - 1) * m ** ax for ax in range(d)))
                xb = X[b_lin]
                y += (w * Me[la, lb] / dt) * (D @ xb)
                for k in range(d):
                    for p in range(d):
                        for q in range(d):
                            y[k * d + p] += Ge[p, q, la, lb] * xb[k * d + q]
        out[t] = y
    return out


# ---------------------------------------------------------------------------
# Deflation space (Section 3.1, Eq. Vmatrix) and the independent Laplacian.
# ---------------------------------------------------------------------------


def V_matrix(mesh: Mesh) -> sp.csr_matrix:
    """V = (1/sqrt d)(v kron I) in node-major ordering: column a has 1/sqrt(d)
    in each sigma_ii slot of node a."""
    d, b, ns = mesh.d, mesh.b, mesh.n_nodes
    rows = (np.arange(ns)[:, None] * b + np.array(diag_components(d))[None, :]).reshape(-1)
    cols = np.repeat(np.arange(ns), d)
    vals = np.full(rows.shape[0], 1.0 / math.sqrt(d))
    return sp.csr_matrix((vals, (rows, cols)), shape=(ns * b, ns))


def embed(mesh: Mesh, q: np.ndarray) -> np.ndarray:
    """V q."""
    return V_matrix(mesh) @ q


def extract(mesh: Mesh, y: np.ndarray) -> np.ndarray:
    """V^T y."""
    return V_matrix(mesh).T @ y


def tridiag(m: int, lo: float, di: float, up: float) -> sp.csr_matrix:
    return sp.diags([np.full(m - 1, lo), np.full(m, di), np.full(m - 1, up)], [-1, 0, 1], format="csr")


def laplacian_kron(d: int, n: int) -> sp.csr_matrix:
    """Q1 Laplacian stiffness sum_i int d_i phi_a d_i phi_b on interior nodes,
    built from 1D interior matrices K1 = (1/h) tridiag(-1,2,-1) and
    M1 = (h/6) tridiag(1,4,1) by Kronecker products (x fastest ordering).
    Independent of the element assembly route."""
    m, h = n - 1, 1.0 / n
    K1 = tridiag(m, -1.0 / h, 2.0 / h, -1.0 / h)
    M1 = tridiag(m, h / 6.0, 4.0 * h / 6.0, h / 6.0)
    L = None
    for i in range(d):  # derivative along axis i
        factors = [K1 if ax == i else M1 for ax in range(d)]
        # kron ordering: slowest axis first
        T = factors[d - 1]
        for ax in range(d - 2, -1, -1):
            T = sp.kron(T, factors[ax], format="csr")
        L = T if L is None else L + T
    return L.tocsr()
