"""Plain CG and the flexible deflated CG (FDCG), oracle in FP64.

Test infrastructure only (see the package docstring).

FDCG follows Algorithm 2 with the outer FCG of Algorithm 1:

* pi(z, tol) = V * Multigrid(V^T z, tol)                      (Algorithm 2)
* M_D(z, tol) = A (z - pi(A z, tol))                           (Algorithm 2)
* f_D = f - A pi(f, tol): reading of the garbled "pi^T(f)"; it is
  (I - pi_A)^T f, the right-hand side of Eq. defl_sys. pi(f, tol) appears
  in Algorithm 2's f_D line and in its reconstruction line with the same
  arguments, so it is evaluated once and reused.
* x_hat = FCG(f_D, x0, M_D); x = x_hat - pi(A x_hat) + pi(f)   (Eq. x_defl)
* outer stop ||r_i||_2 <= tol ||f||_2 on the recursive deflated residual.
* inner tolerance, relative to ||V^T t||: fixed tau_c = c_F * tol (Eq.
  fixed_tol read with the experiments' "0.01 times the outer tolerance"),
  adaptive tau_c = c_A * tol ||f|| / ||r_i|| (Eq. tol, r_i the current outer
  residual). The solves for f_D and the reconstruction use c * tol.
* "exact" inner: Z_J solved by a direct method (Table 2's deflated CG).

Recurrences (Algorithm 1; truncation rule of the FCG remark):
* "fcg1": m_i = 1, d_i = r_i - beta d_{i-1}, beta = (r_i, q_{i-1})/(d_{i-1}, q_{i-1}),
  alpha = (d_i, r_i)/(d_i, q_i) with q = M_D(d).
* "fcg_inf": with m_max = None, d_i orthogonalised against every previous
  direction (Algorithm 1 as printed), q_k stored when computed (Notay's
  variant; the paper re-applies A*(d_k, tol)). With an integer m_max, the
  mixed truncation-restart rule of the remark after Table 4: m_0 = 0,
  m_i = max{1, mod(i, m_max + 1)}, and d_i is orthogonalised against the
  m_i most recent directions d_{i-m_i}, ..., d_{i-1} only. m_max = 0 gives
  FCG(1); m_max at least the iteration count gives the untruncated method.
* "fr": classical CG coefficients, alpha = (r,r)/(d,q), beta = (r',r')/(r,r).
* "gmres": GMRES on the deflated system (the alternative outer solver of the
  remarks in Sections 4.3 and 5.1): Arnoldi with modified Gram-Schmidt on
  the vectors M_D(v_j, tau_c) the inexact operator returns, each v_j's inner
  tolerance from Eq. tol with ||r_j|| the least-squares residual norm;
  Givens rotations give that norm after every step, which is the stopping
  test. m_max = None: full GMRES; an integer: restarted GMRES(m_max), each
  restart from the recursive residual f_D - M_D x_hat.

Reading (not in the paper): after reconstruction the true residual
||f - A x|| / ||f|| is computed in FP64; if it is above tol, the same FDCG is
run on the residual equation A e = f - A x (same absolute threshold
tol ||f||) and x += e, at most ``max_restarts`` times.

Optional stall restart (not in the paper, off unless ``stall_window`` > 0):
a pass whose recursive residual has not fallen below 0.99 x its best value
for max(stall_window, its/4) iterations ends, is reconstructed, and the
solve continues from its true residual like the restart above.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse.linalg as spla

from .mg import Hierarchy, MGOptions, inner_matrix


@dataclass
class SolveStats:
    outer_its: int = 0
    total_mg_cycles: int = 0
    iter_mg_cycles: int = 0
    restarts: int = 0
    true_relres: float = float("nan")
    converged: bool = False
    breakdown: bool = False
    history: list = field(default_factory=list)    # ||r_{i+1}|| after each outer iteration
    res0: list = field(default_factory=list)       # ||r_0|| of each pass
    inner_tols: list = field(default_factory=list)  # tau_c passed to Multigrid in M_D, per outer iteration

    @property
    def avg_inner(self) -> float:
        return self.iter_mg_cycles / max(1, self.outer_its)


def plain_cg(A, f: np.ndarray, tol: float = 1e-8, max_it: int = 100000, x0=None):
    """Textbook CG, x0 = 0 unless given; stop when ||r|| <= tol ||f||."""
    x = np.zeros_like(f) if x0 is None else x0.copy()
    r = f - A @ x if x0 is not None else f.copy()
    d = r.copy()
    rr = r @ r
    eps = tol * np.linalg.norm(f)
    st = SolveStats()
    if np.sqrt(rr) <= eps:
        st.converged = True
    while not st.converged and st.outer_its < max_it:
        q = A @ d
        dq = d @ q
        if not (dq > 0.0) or not np.isfinite(dq):
            st.breakdown = True
            break
        alpha = rr / dq
        x = x + alpha * d
        r = r - alpha * q
        rr_new = r @ r
        st.outer_its += 1
        st.history.append(np.sqrt(rr_new))
        if np.sqrt(rr_new) <= eps:
            st.converged = True
            break
        beta = rr_new / rr
        d = r + beta * d
        rr = rr_new
    st.true_relres = np.linalg.norm(f - A @ x) / np.linalg.norm(f)
    return x, st


@dataclass
class FDCGOptions:
    mg: MGOptions = field(default_factory=MGOptions)
    inner_rule: str = "fixed"      # "fixed" | "adaptive" | "exact"
    c: float = 0.01                # c_F or c_A
    inner_nmax: int = 100
    recurrence: str = "fcg1"       # "fcg1" | "fr" | "fcg_inf" | "gmres"
    m_max: int | None = None       # fcg_inf: truncation-restart parameter; gmres: restart length (None = none)
    max_restarts: int = 3
    stall_window: int = 0          # restart a pass whose residual stopped falling; 0 = off


class FDCG:
    """Setup (inner matrix, hierarchy) and solve of Algorithm 2."""

    def __init__(self, asm, opts: FDCGOptions = None):
        from .fem import V_matrix
        self.asm = asm
        self.opts = opts or FDCGOptions()
        self.A = asm.matrix().tocsr()
        self.V = V_matrix(asm.mesh)
        self.ZJ = inner_matrix(self.V, self.A)
        if self.opts.inner_rule == "exact":
            self.Z_lu = spla.splu(self.ZJ.tocsc())
            self.H = None
        else:
            self.H = Hierarchy(asm.mesh.d, asm.mesh.n, self.ZJ, self.opts.mg)

    # inner solve ------------------------------------------------------------
    def inner(self, g: np.ndarray, tc: float, st: SolveStats, in_iter: bool) -> np.ndarray:
        if self.opts.inner_rule == "exact":
            return self.Z_lu.solve(g)
        z, n = self.H.multigrid(g, tc, self.opts.inner_nmax)
        st.total_mg_cycles += n
        if in_iter:
            st.iter_mg_cycles += n
        return z

    def pi(self, z: np.ndarray, tc: float, st: SolveStats, in_iter: bool = False) -> np.ndarray:
        return self.V @ self.inner(self.V.T @ z, tc, st, in_iter)

    def M_D(self, d: np.ndarray, tc: float, st: SolveStats) -> np.ndarray:
        t = self.A @ d
        return self.A @ (d - self.pi(t, tc, st, in_iter=True))

    def _inner_tol(self, rnorm: float, eps: float, tol: float) -> float:
        c = self.opts.c
        if self.opts.inner_rule == "adaptive":
            return c * eps / rnorm
        return c * tol

    # one FDCG pass ----------------------------------------------------------
    def _pass(self, f, x0, eps, tol, max_it, st: SolveStats):
        A, o = self.A, self.opts
        tc0 = o.c * tol
        # pi(f, tol) enters Algorithm 2 twice (f_D and the reconstruction)
        # with the same arguments; it is evaluated once.
        pi_f = self.pi(f, tc0, st)
        f_D = f - A @ pi_f
        if x0 is None:
            xh = np.zeros_like(f)
            r = f_D.copy()
        else:
            xh = x0.copy()
            r = f_D - self.M_D(xh, tc0, st)
        dirs, qs, dqs = [], [], []
        d = r.copy()
        rr = r @ r
        its = 0
        conv = np.sqrt(rr) <= eps
        # stall test: the recursive residual has not fallen below 0.99 x its
        # best value for max(stall_window, its/4) iterations
        stalled = False
        best, its_best = np.sqrt(rr), 0
        st.res0.append(np.sqrt(rr))
        while not conv and st.outer_its < max_it:
            tc = self._inner_tol(np.sqrt(rr), eps, tol)
            st.inner_tols.append(tc)
            q = self.M_D(d, tc, st)
            dq = d @ q
            if not (dq > 0.0) or not np.isfinite(dq):
                st.breakdown = True
                break
            alpha = (rr if o.recurrence == "fr" else d @ r) / dq
            xh = xh + alpha * d
            r = r - alpha * q
            st.outer_its += 1
            its += 1
            rr_new = r @ r
            st.history.append(np.sqrt(rr_new))
            if np.sqrt(rr_new) <= eps:
                conv = True
                break
            if np.sqrt(rr_new) < 0.99 * best:
                best, its_best = np.sqrt(rr_new), its
            elif o.stall_window > 0 and its - its_best > max(o.stall_window, its // 4):
                stalled = True
                break
            if o.recurrence == "fr":
                d = r + (rr_new / rr) * d
            elif o.recurrence == "fcg1":
                d = r - ((r @ q) / dq) * d
            elif o.recurrence == "fcg_inf":
                # d_{i} for i = len(dirs) + 1 directions stored so far
                dirs.append(d)
                qs.append(q)
                dqs.append(dq)
                i = len(dirs)
                mi = i if o.m_max is None else max(1, i % (o.m_max + 1))
                dn = r.copy()
                for k in range(i - mi, i):
                    dn = dn - ((r @ qs[k]) / dqs[k]) * dirs[k]
                d = dn
            else:
                raise ValueError(o.recurrence)
            rr = rr_new
        x = xh - self.pi(A @ xh, tc0, st) + pi_f
        return x, conv, stalled

    # GMRES pass ------------------------------------------------------------
    def _pass_gmres(self, f, x0, eps, tol, max_it, st: SolveStats):
        A, o = self.A, self.opts
        tc0 = o.c * tol
        pi_f = self.pi(f, tc0, st)
        f_D = f - A @ pi_f
        xh = np.zeros_like(f) if x0 is None else x0.copy()
        r = f_D if x0 is None else f_D - self.M_D(xh, tc0, st)
        conv = False
        first = True
        while not conv and st.outer_its < max_it:
            beta = np.linalg.norm(r)
            if first:
                st.res0.append(beta)
                first = False
            if beta <= eps:
                conv = True
                break
            m = o.m_max if o.m_max is not None else max_it
            V = [r / beta]
            Hc = []        # columns of the rotated Hessenberg matrix (upper triangular R)
            cs, sn = [], []
            g = [beta]
            j = 0
            while j < m and st.outer_its < max_it:
                tc = self._inner_tol(abs(g[j]), eps, tol)
                st.inner_tols.append(tc)
                w = self.M_D(V[j], tc, st)
                h = np.zeros(j + 2)
                for i in range(j + 1):
                    h[i] = V[i] @ w
                    w = w - h[i] * V[i]
                h[j + 1] = np.linalg.norm(w)
                for i in range(j):  # previous rotations on the new column
                    a, b = h[i], h[i + 1]
                    h[i], h[i + 1] = cs[i] * a + sn[i] * b, -sn[i] * a + cs[i] * b
                den = np.hypot(h[j], h[j + 1])
                if den == 0.0:
                    st.breakdown = True
                    break
                cs.append(h[j] / den)
                sn.append(h[j + 1] / den)
                h[j], h[j + 1] = den, 0.0
                Hc.append(h[: j + 1])
                g.append(-sn[j] * g[j])
                g[j] = cs[j] * g[j]
                st.outer_its += 1
                st.history.append(abs(g[j + 1]))
                nrm = np.linalg.norm(w)
                if nrm > 0.0:
                    V.append(w / nrm)
                j += 1
                if abs(g[j]) <= eps or nrm == 0.0:
                    conv = True
                    break
            if j > 0:
                R = np.zeros((j, j))
                for c, col in enumerate(Hc[:j]):
                    R[: c + 1, c] = col
                y = np.linalg.solve(R, np.array(g[:j]))
                for i in range(j):
                    xh = xh + y[i] * V[i]
            if st.breakdown or conv:
                break
            r = f_D - self.M_D(xh, tc0, st)  # restart from the recursive residual
        x = xh - self.pi(A @ xh, tc0, st) + pi_f
        return x, conv, False

    def solve(self, f: np.ndarray, tol: float = 1e-8, max_it: int = 100000, x0=None):
        st = SolveStats()
        fn = np.linalg.norm(f)
        if fn == 0.0:
            st.converged, st.true_relres = True, 0.0
            return np.zeros_like(f), st
        eps = tol * fn
        run = self._pass_gmres if self.opts.recurrence == "gmres" else self._pass
        x, conv, stalled = run(f, x0, eps, tol, max_it, st)
        res = f - self.A @ x
        st.true_relres = np.linalg.norm(res) / fn
        claimed = 0  # restarts after passes that reported convergence
        while (st.true_relres > tol and (stalled or claimed < self.opts.max_restarts)
               and not st.breakdown and st.outer_its < max_it):
            if not stalled:
                claimed += 1
            st.restarts += 1
            e, conv, stalled = run(res, None, eps, tol, max_it, st)
            x = x + e
            res = f - self.A @ x
            st.true_relres = np.linalg.norm(res) / fn
        st.converged = bool(st.true_relres <= tol)
        return x, st


def dense_solve(asm, f: np.ndarray) -> np.ndarray:
    """Direct solve of A x = f (dense Cholesky) for tiny meshes."""
    import scipy.linalg as sla
    A = asm.matrix().toarray()
    return sla.cho_solve(sla.cho_factor(A, lower=True), f)
