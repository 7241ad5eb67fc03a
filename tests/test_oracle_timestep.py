"""Pins of the oracle's time stepping (Section 2.3) and reconstruction
(Section 5.2), no GPU: closed-form decay of generalised eigenmodes for each
scheme, the pressure of the pure-trace and pure-deviatoric fields, and the
centre divergence against a direct evaluation of the Q1 basis derivatives."""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import fem, solvers, timestep
from paper_2606_13429_gb300 import inputs


def _modes(d, n):
    """Generalised eigenpairs K v = lam M v of the pseudo-stress forms (from
    K v = theta (M + K) v, lam = theta / (1 - theta) for theta < 1)."""
    M = fem.assemble(d, n, 1.0, div=False).matrix().toarray()
    K = fem.assemble(d, n, 1.0, mass=False).matrix().toarray()
    th, V = sla.eigh(K, M + K)
    keep = th < 1.0 - 1e-9
    return th[keep] / (1.0 - th[keep]), V[:, keep]


@pytest.mark.parametrize("scheme", ["ie", "cn", "bdf2"])
def test_eigenmode_decay(scheme):
    """sigma^0 = v with K v = lam M v and no forcing: every step multiplies v
    by the scheme's amplification factor (implicit Euler 1/(1 + lam dt),
    Crank-Nicolson (1 - lam dt/2)/(1 + lam dt/2), BDF2 from its recurrence
    (1 + alpha lam) c_n = 4/3 c_{n-1} - 1/3 c_{n-2}, c_{-1} = c_0 = 1)."""
    d, n, dt = 2, 6, 1e-2
    lam, V = _modes(d, n)
    for j in [0, len(lam) // 2, len(lam) - 1]:
        v = V[:, j] / np.linalg.norm(V[:, j])
        ts = timestep.TimeStepper(d, n, dt, scheme, opts=solvers.FDCGOptions(inner_rule="exact"))
        zero = np.zeros_like(v)
        sig, _ = ts.run(v, [zero, zero, zero], tol=1e-13)
        a = ts.alpha
        if scheme == "ie":
            c = [1.0 / (1 + lam[j] * dt)]
            c.append(c[0] ** 2)
        elif scheme == "cn":
            r = (1 - lam[j] * dt / 2) / (1 + lam[j] * dt / 2)
            c = [r, r * r]
        else:
            c1 = 1.0 / (1 + a * lam[j])
            c2 = (4.0 / 3.0 * c1 - 1.0 / 3.0) / (1 + a * lam[j])
            c = [c1, c2]
        for k in range(2):
            assert np.linalg.norm(sig[k] - c[k] * v) <= 1e-9, (scheme, j, k)


def test_alpha_of_schemes():
    assert timestep.alpha_of("ie", 0.3) == 0.3
    assert timestep.alpha_of("cn", 0.3) == 0.15
    assert abs(timestep.alpha_of("bdf2", 0.3) - 0.2) < 1e-15


def test_pressure_of_trace_and_deviatoric_fields():
    """p = -(1/d) tr(sigma): for sigma = V q (q/sqrt(d) on every diagonal
    component) p = -q/sqrt(d); a traceless field has p = 0."""
    for d in (2, 3):
        mesh = fem.Mesh(d, 5)
        q = inputs.rhs(1, mesh.n_nodes)
        assert np.allclose(timestep.pressure(mesh, fem.embed(mesh, q)), -q / np.sqrt(d), rtol=0, atol=1e-15)
        s = inputs.rhs(2, mesh.n_unknowns).reshape(mesh.n_nodes, d * d)
        tr = sum(s[:, i * d + i] for i in range(d)) / d
        for i in range(d):
            s[:, i * d + i] -= tr
        assert np.abs(timestep.pressure(mesh, s.reshape(-1))).max() <= 1e-15


@pytest.mark.parametrize("d,n", [(2, 5), (3, 4)])
def test_centre_divergence_against_basis_derivatives(d, n):
    """(div sigma)_k at each element centre from the gradients of the 2^d
    local Q1 basis functions at the centre (each the product of a 1D hat
    derivative +-1/h and 1D hat values 1/2), summed over the element's nodes."""
    mesh = fem.Mesh(d, n)
    sigma = inputs.rhs(4, mesh.n_unknowns)
    got = timestep.divergence_at_centres(mesh, sigma)
    m, h = mesh.m, mesh.h
    s = sigma.reshape(mesh.n_nodes, d * d)
    want = np.zeros((n ** d, d))
    for e, ec in enumerate(itertools.product(range(n), repeat=d)):
        ec = ec[::-1]  # x fastest
        for bits in itertools.product((0, 1), repeat=d):
            node = [ec[ax] + bits[ax] for ax in range(d)]  # 0..n, boundary at 0 and n
            if any(c == 0 or c == n for c in node):
                continue
            a = sum((node[ax] - 1) * m ** ax for ax in range(d))
            for p in range(d):
                g = (1.0 / h if bits[p] else -1.0 / h) * 0.5 ** (d - 1)
                for k in range(d):
                    want[e, k] += g * s[a, k * d + p]
    assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max())


def test_velocity_rules():
    """Right-endpoint sums for implicit Euler / BDF2, trapezoid for CN."""
    mesh = fem.Mesh(2, 4)
    sig = [inputs.rhs(10 + k, mesh.n_unknowns) for k in range(3)]
    dv = [timestep.divergence_at_centres(mesh, s) for s in sig]
    u = timestep.velocity(mesh, sig[1:], 0.1, "ie")
    assert np.allclose(u, 0.1 * (dv[1] + dv[2]))
    u = timestep.velocity(mesh, sig[1:], 0.1, "cn", sigma0=sig[0])
    assert np.allclose(u, 0.05 * (dv[0] + 2 * dv[1] + dv[2]))
