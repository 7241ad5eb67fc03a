"""Implicit time stepping of the pseudo-stress Stokes problem and the
reconstruction of pressure and velocity, oracle in FP64.

Test infrastructure only (see the package docstring).

Section 2.3 (Eq. weak_IE): one step solves (M + alpha A) sigma^n = F*_n with
alpha = alpha(dt) of the chosen implicit scheme, F*_n depending on earlier
steps. This library's operator is A_alpha = M_dev / alpha + K_div (the
paper's M + alpha A divided by alpha), so a step solves A_alpha sigma^n = b^n
with, for the load vectors F^n of the forcing at t_n:

* implicit Euler (theta = 1), alpha = dt:
      b^n = (M_dev / alpha) sigma^{n-1} + F^n
* Crank-Nicolson (theta = 1/2), alpha = dt / 2:
      b^n = (M_dev / alpha - K_div) sigma^{n-1} + F^n + F^{n-1}
* BDF2, alpha = 2 dt / 3:
      b^n = (M_dev / alpha) (4/3 sigma^{n-1} - 1/3 sigma^{n-2}) + F^n
  (the first step takes sigma^{-1} = sigma^0).

Reconstruction (Section 5.2): pressure p = -(1/d) tr(sigma) at every node;
velocity u(t) = u_0 + int_0^t div(sigma) ds with (div sigma)_k =
sum_p d_p sigma_kp evaluated at element centres (exact there for Q1 fields),
integrated by the right-endpoint rule (implicit Euler, BDF2) or the
trapezoidal rule (Crank-Nicolson), the rules of the scheme itself.
"""
from __future__ import annotations

import numpy as np

from . import fem
from .solvers import FDCG, FDCGOptions

SCHEMES = ("ie", "cn", "bdf2")


def alpha_of(scheme: str, dt: float) -> float:
    return {"ie": dt, "cn": dt / 2.0, "bdf2": 2.0 * dt / 3.0}[scheme]


class TimeStepper:
    """A_alpha, M_dev and K_div assembled separately, and the FDCG solver of
    A_alpha (set up once: its inner matrix V^T A V does not depend on dt)."""

    def __init__(self, d: int, n: int, dt: float, scheme: str, nu: float = 1.0, opts: FDCGOptions | None = None):
        if scheme not in SCHEMES:
            raise ValueError(scheme)
        self.d, self.n, self.dt, self.scheme = d, n, dt, scheme
        self.alpha = alpha_of(scheme, dt)
        self.M = fem.assemble(d, n, 1.0, nu=nu, div=False).matrix().tocsr()
        self.K = fem.assemble(d, n, 1.0, nu=nu, mass=False).matrix().tocsr()
        self.asm = fem.assemble(d, n, self.alpha, nu=nu)
        self.solver = FDCG(self.asm, opts or FDCGOptions())

    def rhs(self, s1: np.ndarray, s2: np.ndarray | None, F1: np.ndarray, F0: np.ndarray | None) -> np.ndarray:
        a = self.alpha
        if self.scheme == "ie":
            return self.M @ s1 / a + F1
        if self.scheme == "cn":
            return self.M @ s1 / a - self.K @ s1 + F1 + F0
        w = (4.0 / 3.0) * s1 - (1.0 / 3.0) * (s1 if s2 is None else s2)
        return self.M @ w / a + F1

    def run(self, sigma0: np.ndarray, loads: list, tol: float = 1e-8):
        """loads[n] = F^n, n = 0..nsteps; returns sigma^1..sigma^nsteps and the
        solver statistics of each step (initial guess sigma^{n-1})."""
        out, stats = [], []
        prev, prev2 = sigma0, None
        for k in range(1, len(loads)):
            b = self.rhs(prev, prev2 if self.scheme == "bdf2" else None, loads[k], loads[k - 1])
            x, st = self.solver.solve(b, tol=tol, x0=prev)
            out.append(x)
            stats.append(st)
            prev2, prev = prev, x
        return out, stats


def pressure(mesh: fem.Mesh, sigma: np.ndarray) -> np.ndarray:
    """p = -(1/d) tr(sigma) at every interior node."""
    d = mesh.d
    s = sigma.reshape(mesh.n_nodes, d * d)
    return -sum(s[:, i * d + i] for i in range(d)) / d


def divergence_at_centres(mesh: fem.Mesh, sigma: np.ndarray) -> np.ndarray:
    """(div sigma)_k at every element centre, elements lexicographic (x
    fastest), d values per element: for a Q1 field the derivative along axis
    p at the centre is the mean over the element's 2^(d-1) edges along p of
    (value at the upper end - value at the lower end) / h. Boundary nodes
    carry zero (homogeneous Dirichlet)."""
    d, n, m, h = mesh.d, mesh.n, mesh.m, mesh.h
    full = np.zeros((n + 1,) * d + (d * d,))
    # interior nodes 1..m on every axis; array axes ordered slowest first
    inner = sigma.reshape(tuple([m] * d) + (d * d,))
    full[tuple([slice(1, m + 1)] * d) + (slice(None),)] = inner
    out = np.zeros((n,) * d + (d,))
    for k in range(d):
        for p in range(d):
            comp = full[..., k * d + p]
            ax = d - 1 - p  # array axis of coordinate p (x is the last array axis)
            diff = np.diff(comp, axis=ax) / h
            # average over the other axes' two element corners
            for q in range(d):
                if q == ax:
                    continue
                diff = 0.5 * (np.take(diff, range(0, n), axis=q) + np.take(diff, range(1, n + 1), axis=q))
            out[..., k] += diff
    return out.reshape(n ** d, d)


def velocity(mesh: fem.Mesh, sigmas: list, dt: float, scheme: str, u0: np.ndarray | None = None,
             sigma0: np.ndarray | None = None) -> np.ndarray:
    """u^N at element centres from u^0 (zero by default) and the steps
    sigma^1..sigma^N (sigma^0 needed by the trapezoidal rule)."""
    u = np.zeros((mesh.n ** mesh.d, mesh.d)) if u0 is None else u0.copy()
    prev = None if sigma0 is None else divergence_at_centres(mesh, sigma0)
    for s in sigmas:
        cur = divergence_at_centres(mesh, s)
        if scheme == "cn":
            u = u + 0.5 * dt * (cur + prev)
        else:
            u = u + dt * cur
        prev = cur
    return u
