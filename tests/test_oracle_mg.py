"""Pins of the oracle's multigrid (no GPU): Galerkin hierarchy, RAS smoother,
coarse solve and W-cycle, against closed forms, brute force and textbook
special cases."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem, mg
from paper_2606_13429_gb300 import inputs


def _hier(d, n, **kw):
    ZJ = fem.laplacian_kron(d, n) / d
    return mg.Hierarchy(d, n, ZJ, mg.MGOptions(**kw))


@pytest.mark.parametrize("d,n", [(2, 16), (2, 64), (3, 8)])
def test_galerkin_equals_rediscretisation(d, n):
    """P5: P^T L_h P = L_2h for nested Q1 with nodal interpolation."""
    Lh = fem.laplacian_kron(d, n)
    L2h = fem.laplacian_kron(d, n // 2)
    P = mg.prolongation(d, n // 2 - 1)
    G = P.T @ Lh @ P
    assert abs(G - L2h).max() <= 1e-13 * abs(L2h).max()


def test_prolongation_interpolates_linear_functions():
    """P reproduces functions that are linear per axis and vanish on the
    boundary's supporting lines (interpolation of coarse nodal values)."""
    m_c = 7
    P1 = mg.prolongation_1d(m_c).toarray()
    xc = (np.arange(m_c) + 1) * 2.0
    xf = np.arange(2 * m_c + 1) + 1.0
    # hat-shaped piecewise linear: u(x) = x (coarse nodal values) restricted
    # away from the boundary; check interior fine nodes between coarse nodes
    uf = P1 @ xc
    assert np.allclose(uf[1:-1], xf[1:-1])
    assert uf[0] == 1.0 and uf[-1] == 0.5 * xc[-1]


def test_level_sizes_rule():
    assert mg.level_sizes(32) == [32, 16, 8, 4]
    assert mg.level_sizes(1024) == [1024, 512, 256, 128]
    assert mg.level_sizes(1024, 99) == [1024, 512, 256, 128, 64, 32, 16, 8, 4]
    assert mg.level_sizes(20, 99) == [20, 10, 5]
    assert mg.level_sizes(12, 99) == [12, 6]
    assert mg.level_sizes(6) == [6]


@pytest.mark.parametrize("d,m,P,o", [(2, 9, 4, 1), (2, 15, 8, 2), (3, 7, 4, 1), (2, 7, 1, 0), (2, 11, 4, 3)])
def test_ras_operator_brute_force(d, m, P, o):
    """RAS step == z + S (f - Z z) with S = sum_i R_i^T D_i (R_i Z R_i^T)^-1 R_i
    assembled densely from boxes enumerated by brute force over all nodes."""
    n = m + 1
    for weights in ["multiplicity", "restricted"]:
        H = _hier(d, n, patch=P, overlap=o, max_levels=2, ras_weights=weights)
        assert H.J == 2  # the finest level is smoothed, not solved exactly
        k = H.J  # finest
        lev = H.levels[-1]
        Z = lev.Z.toarray()
        N = m ** d
        coords = np.array([[(j // m ** ax) % m for ax in range(d)] for j in range(N)])
        boxes = []
        ntile = -(-m // P)
        for t in itertools.product(range(ntile), repeat=d):
            core = [(t[ax] * P, min((t[ax] + 1) * P, m)) for ax in range(d)]
            ext = [(max(0, c[0] - o), min(m, c[1] + o)) for c in core]
            inside = np.all([(coords[:, ax] >= ext[ax][0]) & (coords[:, ax] < ext[ax][1]) for ax in range(d)], axis=0)
            incore = np.all([(coords[:, ax] >= core[ax][0]) & (coords[:, ax] < core[ax][1]) for ax in range(d)], axis=0)
            boxes.append((np.nonzero(inside)[0], incore))
        mult = np.zeros(N)
        for idx, _ in boxes:
            mult[idx] += 1
        S = np.zeros((N, N))
        for idx, incore in boxes:
            R = np.zeros((len(idx), N))
            R[np.arange(len(idx)), idx] = 1.0
            Dw = (1.0 / mult[idx]) if weights == "multiplicity" else incore[idx].astype(float)
            S += R.T @ np.diag(Dw) @ np.linalg.inv(R @ Z @ R.T) @ R
        rng = np.random.default_rng(0)
        f, z = rng.standard_normal(N), rng.standard_normal(N)
        want = z + S @ (f - Z @ z)
        got = H.ras_step(k, f, z)
        assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
        # partition of unity: weights sum to one on every node
        pu = np.zeros(N)
        for p, w in zip(lev.patches, lev.weights):
            pu[p.idx] += w
        assert np.allclose(pu, 1.0)


def test_ras_single_node_patches_is_jacobi():
    """P8: P=1, o=0 gives z + D^-1 (f - Z z), D = diag(Z)."""
    H = _hier(2, 12, patch=1, overlap=0, max_levels=2)
    Z = H.levels[-1].Z
    rng = np.random.default_rng(1)
    f, z = rng.standard_normal(Z.shape[0]), rng.standard_normal(Z.shape[0])
    want = z + (f - Z @ z) / Z.diagonal()
    assert np.allclose(H.ras_step(H.J, f, z), want, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("d,n", [(2, 16), (3, 8)])
def test_ras_one_global_patch_is_exact(d, n):
    """P8: one patch covering the level makes one smoothing step an exact
    solve, hence one W-cycle converges."""
    m = n - 1
    H = _hier(d, n, patch=m, overlap=1, m1=1, m2=0)
    f = np.random.default_rng(2).standard_normal(m ** d)
    z = H.wcycle(f, np.zeros_like(f))
    Z = H.levels[-1].Z
    assert np.linalg.norm(f - Z @ z) <= 1e-12 * np.linalg.norm(f)
    z2, ncyc = H.multigrid(f, 1e-10, 10)
    assert ncyc == 1


@pytest.mark.parametrize("d,n,modes", [(2, 8, (1, 1)), (2, 8, (3, 5)), (3, 4, (1, 2, 3)), (2, 16, (7, 2))])
def test_coarse_solve_sine_modes(d, n, modes):
    """Exact coarsest solve against the closed-form eigenpairs of the Q1
    Laplacian (sine modes): Z^-1 s = d s / lambda."""
    H = _hier(d, n, max_levels=1)
    s, lam = mg.sine_mode(d, n, modes)
    assert np.allclose(fem.laplacian_kron(d, n) @ s, lam * s, rtol=0, atol=1e-12 * lam)
    z = H.coarse_solve(s)
    assert np.allclose(z, d * s / lam, rtol=1e-12, atol=1e-14)


def test_wcycle_visits_and_linearity():
    """W-cycle is an affine stationary iteration: W(f, z) = z + W(f - Z z, 0)."""
    H = _hier(2, 32)
    Z = H.levels[-1].Z
    rng = np.random.default_rng(3)
    f, z = rng.standard_normal(Z.shape[0]), rng.standard_normal(Z.shape[0])
    a = H.wcycle(f, z)
    b = z + H.wcycle(f - Z @ z, np.zeros_like(z))
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12 * np.abs(a).max())


def test_wcycle_convergence_h_independent():
    """P9: W-cycle contraction factor bounded away from 1 and roughly
    independent of h (textbook multigrid behaviour)."""
    rates = []
    for n in [16, 32, 64, 128]:
        H = _hier(2, n)
        Z = H.levels[-1].Z
        f = np.random.default_rng(4).standard_normal(Z.shape[0])
        z = np.zeros_like(f)
        r0 = np.linalg.norm(f)
        for _ in range(4):
            z = H.wcycle(f, z)
        rates.append((np.linalg.norm(f - Z @ z) / r0) ** 0.25)
    assert max(rates) < 0.2, rates
    assert max(rates) / min(rates) < 3.0, rates


def test_multigrid_driver_counts():
    """Algorithm 3: residual test before each cycle; zero RHS gives zero
    cycles; the cap n_max is honoured."""
    H = _hier(2, 16)
    f = np.ones(15 * 15)
    z, n = H.multigrid(np.zeros_like(f), 1e-10, 100)
    assert n == 0 and not z.any()
    z, n = H.multigrid(f, 1e-30, 3)
    assert n == 3
    z, n = H.multigrid(f, 1e-10, 100)
    Z = H.levels[-1].Z
    assert np.linalg.norm(f - Z @ z) <= 1e-10 * np.linalg.norm(f)
    assert 1 <= n <= 12
    # one cycle fewer leaves the residual above the tolerance
    zb, nb = H.multigrid(f, 1e-10, n - 1)
    assert nb == n - 1
    assert np.linalg.norm(f - Z @ zb) > 1e-10 * np.linalg.norm(f)


def test_coarsest_wcycle_ignores_its_initial_guess():
    """On the coarsest level Algorithm 4's W is the exact solve, so its second
    recursive call W_1(r_c, e1) returns the same vector as the first, W_1(r_c, 0):
    a two-level W-cycle equals one that solves the coarse problem once."""
    d, n = 2, 16
    asm = fem.assemble(d, n, 1e-3)
    V = fem.V_matrix(asm.mesh)
    H = mg.Hierarchy(d, n, mg.inner_matrix(V, asm.matrix()),
                     mg.MGOptions(patch=4, overlap=1, max_levels=2))
    assert H.J == 2
    rc = inputs.rhs(1, H.levels[0].Z.shape[0])
    e1 = H.wcycle(rc, np.zeros_like(rc), 1)
    e2 = H.wcycle(rc, e1, 1)
    assert np.array_equal(e1, e2)
    assert np.array_equal(e1, H.wcycle(rc, inputs.rhs(2, rc.size), 1))
    # and the full two-level cycle with one coarse solve gives the same result
    f = inputs.rhs(3, H.levels[1].Z.shape[0])
    z_ref = H.wcycle(f, np.zeros_like(f))
    lev = H.levels[1]
    z = np.zeros_like(f)
    for _ in range(H.opts.m1):
        z = H.ras_step(2, f, z)
    rc2 = H.restrict(2, f - lev.Z @ z)
    z = z + H.prolong(2, H.coarse_solve(rc2))
    for _ in range(H.opts.m2):
        z = H.ras_step(2, f, z)
    assert np.array_equal(z, z_ref)
