"""Multigrid for the inner (Laplacian) system, oracle in FP64.

Test infrastructure only (see the package docstring).

* Inner matrix Z_J = V^T A V (Algorithm 2, first setup line; Corollary 1 says
  it equals (1/d) times the Laplacian stiffness in the dt-scaled system).
* Hierarchy Z_{k-1} = R Z_k P (Algorithm 2 setup loop) with P the nodal
  bilinear/trilinear interpolation from the coarse interior nodes and R = P^T.
  Reading of Section 4.2: for nested Q1 spaces the L2-projection prolongation
  is the natural embedding, i.e. nodal interpolation; its L2 adjoint acting
  on residual (dual) vectors is P^T.
* Levels: coarsen while n_k is even, n_k >= 8 and fewer than ``max_levels``
  levels exist (the paper uses four levels in 2D, Section 5.1).
* RAS smoother (Section 4.2): blocks are core tiles of P nodes per axis,
  starting at index 0 (last tile may be short), extended by ``overlap`` nodes
  on each side and clipped to the interior; local matrix R_i Z_k R_i^T solved
  exactly; weights D_i = 1/multiplicity (the paper's partition of unity) or
  0/1 on the core ("restricted"). One smoothing step is
  z <- z + sum_i R_i^T D_i (Z_k)_i^{-1} R_i (f - Z_k z).
* W-cycle (Algorithm 4) and the multigrid driver (Algorithm 3), literally:
  coarsest level solved exactly, two recursive coarse solves, residual test
  before every cycle, cap n_max.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def level_sizes(n: int, max_levels: int = 4) -> list[int]:
    """Element counts per side, finest first."""
    sizes = [n]
    while sizes[-1] % 2 == 0 and sizes[-1] >= 8 and len(sizes) < max_levels:
        sizes.append(sizes[-1] // 2)
    return sizes


def prolongation_1d(m_c: int) -> sp.csr_matrix:
    """Coarse interior node i (0-based) sits at fine interior index 2i+1;
    fine nodes 2i and 2i+2 get weight 1/2 from it. Eliminated boundary nodes
    contribute nothing."""
    m_f = 2 * m_c + 1
    rows, cols, vals = [], [], []
    for i in range(m_c):
        rows += [2 * i, 2 * i + 1, 2 * i + 2]
        cols += [i, i, i]
        vals += [0.5, 1.0, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(m_f, m_c))


def prolongation(d: int, m_c: int) -> sp.csr_matrix:
    P1 = prolongation_1d(m_c)
    P = P1
    for _ in range(d - 1):
        P = sp.kron(P1, P, format="csr")  # slower axis on the left
    return P.tocsr()


@dataclass
class Patch:
    idx: np.ndarray       # global node indices of the extended block, x fastest
    core_mask: np.ndarray  # bool, node is in the core tile
    chol: tuple = None    # Cholesky factor of R_i Z R_i^T


def tiles_1d(m: int, P: int, o: int):
    """(core_lo, core_hi, ext_lo, ext_hi) per tile along one axis."""
    out = []
    for t in range(-(-m // P)):
        lo, hi = t * P, min((t + 1) * P, m)
        out.append((lo, hi, max(0, lo - o), min(m, hi + o)))
    return out


def build_patches(d: int, m: int, P: int, o: int) -> list[Patch]:
    t1 = tiles_1d(m, P, o)
    patches = []
    for tile in np.ndindex(*([len(t1)] * d)):
        tile = tile[::-1]  # axis 0 fastest
        ranges = [np.arange(t1[tile[ax]][2], t1[tile[ax]][3]) for ax in range(d)]
        cores = [(t1[tile[ax]][0], t1[tile[ax]][1]) for ax in range(d)]
        grids = np.meshgrid(*ranges[::-1], indexing="ij")  # slowest axis first
        coords = [g.reshape(-1) for g in grids[::-1]]        # coords[ax]
        idx = np.zeros(coords[0].shape[0], dtype=np.int64)
        core = np.ones(coords[0].shape[0], dtype=bool)
        for ax in range(d):
            idx += coords[ax] * (m ** ax)
            core &= (coords[ax] >= cores[ax][0]) & (coords[ax] < cores[ax][1])
        patches.append(Patch(idx=idx, core_mask=core))
    return patches


@dataclass
class Level:
    n: int
    m: int
    Z: sp.csr_matrix
    P: sp.csr_matrix | None = None      # prolongation from the next coarser level
    patches: list = field(default_factory=list)
    weights: list = field(default_factory=list)  # D_i diagonal per patch
    coarse_lu: object = None


@dataclass
class MGOptions:
    patch: int = 4
    overlap: int = 1
    m1: int = 2
    m2: int = 2
    max_levels: int = 4
    ras_weights: str = "multiplicity"  # or "restricted"


class Hierarchy:
    """Galerkin hierarchy Z_k, RAS patches and the coarsest factorisation."""

    def __init__(self, d: int, n: int, ZJ: sp.csr_matrix, opts: MGOptions):
        self.d, self.opts = d, opts
        sizes = level_sizes(n, opts.max_levels)
        self.levels: list[Level] = []  # index 0 = coarsest (level 1 of the paper)
        Z = ZJ.tocsr()
        fine_first = []
        for k, nk in enumerate(sizes):
            lev = Level(n=nk, m=nk - 1, Z=Z)
            if k + 1 < len(sizes):
                Pk = prolongation(d, sizes[k + 1] - 1)
                lev.P = Pk
                Z = (Pk.T @ Z @ Pk).tocsr()
            fine_first.append(lev)
        self.levels = fine_first[::-1]
        for j, lev in enumerate(self.levels):
            if j == 0:
                lev.coarse_lu = spla.splu(lev.Z.tocsc())
            else:
                self._setup_ras(lev)

    def _setup_ras(self, lev: Level):
        o = self.opts
        lev.patches = build_patches(self.d, lev.m, o.patch, o.overlap)
        mult = np.zeros(lev.m ** self.d)
        for p in lev.patches:
            mult[p.idx] += 1.0
        Zd = lev.Z
        for p in lev.patches:
            Ai = Zd[p.idx][:, p.idx].toarray()
            p.chol = sla.cho_factor(Ai, lower=True)
            if o.ras_weights == "multiplicity":
                lev.weights.append(1.0 / mult[p.idx])
            elif o.ras_weights == "restricted":
                lev.weights.append(p.core_mask.astype(np.float64))
            else:
                raise ValueError(o.ras_weights)

    @property
    def J(self) -> int:
        return len(self.levels)

    # -- operators ---------------------------------------------------------
    def ras_step(self, k: int, f: np.ndarray, z: np.ndarray) -> np.ndarray:
        """z + S_k (f - Z_k z), S_k = sum_i R_i^T D_i (Z_k)_i^{-1} R_i."""
        lev = self.levels[k - 1]
        r = f - lev.Z @ z
        znew = z.copy()
        for p, w in zip(lev.patches, lev.weights):
            y = sla.cho_solve(p.chol, r[p.idx])
            znew[p.idx] += w * y
        return znew

    def coarse_solve(self, f: np.ndarray) -> np.ndarray:
        return self.levels[0].coarse_lu.solve(f)

    def restrict(self, k: int, r: np.ndarray) -> np.ndarray:
        """Residual on level k -> level k-1: P^T r."""
        return self.levels[k - 1].P.T @ r

    def prolong(self, k: int, e: np.ndarray) -> np.ndarray:
        """Correction on level k-1 -> level k: P e."""
        return self.levels[k - 1].P @ e

    def wcycle(self, f: np.ndarray, z0: np.ndarray, k: int | None = None) -> np.ndarray:
        """One W-cycle (Algorithm 4) on level k (1 = coarsest)."""
        if k is None:
            k = self.J
        if k == 1:
            return self.coarse_solve(f)
        lev = self.levels[k - 1]
        z = z0.copy()
        for _ in range(self.opts.m1):
            z = self.ras_step(k, f, z)
        rc = self.restrict(k, f - lev.Z @ z)
        e_bar = self.wcycle(rc, np.zeros_like(rc), k - 1)
        e = self.wcycle(rc, e_bar, k - 1)
        z = z + self.prolong(k, e)
        for _ in range(self.opts.m2):
            z = self.ras_step(k, f, z)
        return z

    def multigrid(self, f: np.ndarray, tol: float, nmax: int, z0: np.ndarray | None = None):
        """Algorithm 3: repeat W-cycles while n < nmax and the relative
        residual exceeds tol. Returns (z, n)."""
        Z = self.levels[-1].Z
        z = np.zeros_like(f) if z0 is None else z0.copy()
        fn = np.linalg.norm(f)
        n = 0
        if fn == 0.0:
            return z, 0
        while n < nmax and np.linalg.norm(f - Z @ z) / fn > tol:
            z = self.wcycle(f, z)
            n += 1
        return z, n


def inner_matrix(V: sp.csr_matrix, A) -> sp.csr_matrix:
    """Z_J = V^T A V."""
    return (V.T @ (A @ V)).tocsr()


def sine_mode(d: int, n: int, modes) -> tuple[np.ndarray, float]:
    """Discrete sine mode prod_ax sin(pi j_ax (i_ax+1)/n) on interior nodes and
    its eigenvalue for the Q1 Laplacian stiffness (closed form):
    K1 s = kap s, M1 s = mu s with kap = (2/h)(1-cos t), mu = (h/3)(2+cos t),
    t = pi j / n; eigenvalue sum_i kap_i prod_{ax != i} mu_ax."""
    m, h = n - 1, 1.0 / n
    i = np.arange(1, m + 1)
    vecs, kap, mu = [], [], []
    for j in modes:
        t = math.pi * j / n
        vecs.append(np.sin(t * i))
        kap.append((2.0 / h) * (1.0 - math.cos(t)))
        mu.append((h / 3.0) * (2.0 + math.cos(t)))
    v = vecs[d - 1]
    for ax in range(d - 2, -1, -1):
        v = np.kron(v, vecs[ax])
    lam = 0.0
    for ii in range(d):
        term = kap[ii]
        for ax in range(d):
            if ax != ii:
                term *= mu[ax]
        lam += term
    return v, lam
