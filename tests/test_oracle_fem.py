"""Pins of the oracle's discretisation (no GPU).

Each check ties the oracle to something other than itself: the matrices the
paper prints (Section 3.1), textbook Q1 stencils, a second derivation of the
element integrals, brute force, and algebraic identities of the method.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem, mg

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("h", [1.0, 0.25, 1.0 / 1024])
def test_element_integrals_closed_form_equal_quadrature(d, h):
    """P1: tensor-product closed forms == 2-point Gauss quadrature."""
    Me = fem.element_mass(d, h)
    Ge = fem.element_grad(d, h)
    Mq, Gq = fem.element_matrices_quadrature(d, h)
    assert np.allclose(Me, Mq, rtol=1e-14, atol=1e-15 * np.abs(Mq).max())
    assert np.allclose(Ge, Gq, rtol=1e-14, atol=1e-14 * np.abs(Gq).max())
    # partition of unity: mass sums to the element volume; gradients of a
    # constant vanish
    assert math.isclose(Me.sum(), h ** d, rel_tol=1e-14)
    assert np.allclose(Ge.sum(axis=3), 0.0, atol=1e-14 * np.abs(Ge).max())


@pytest.mark.parametrize("d", [2, 3])
def test_dev_matrix_matches_paper(d):
    """D_d equals the matrix printed in Section 3.1; D_d^2 = D_d, D_d v = 0."""
    g = _gold("paper_matrices.json")
    key = "D2" if d == 2 else "D3"
    printed = g[key]["scale"] * np.array(g[key]["entries"], dtype=float)
    D = fem.dev_matrix(d)
    assert np.allclose(D, printed, rtol=0, atol=1e-15)
    assert np.allclose(D @ D, D, atol=1e-15)
    v = np.array(g["v2" if d == 2 else "v3"], dtype=float)
    assert np.array_equal(np.array([1.0 if j in fem.diag_components(d) else 0.0 for j in range(d * d)]), v)
    assert np.allclose(D @ v, 0.0, atol=1e-15)


@pytest.mark.parametrize("d,n", [(2, 2), (2, 5), (3, 2), (3, 4)])
def test_pattern_brute_force(d, n):
    """Pattern == all node pairs sharing an element, columns ascending."""
    mesh = fem.Mesh(d, n)
    row_ptr, col_idx = fem.bsr_pattern(mesh)
    en = fem.element_nodes(mesh)
    pairs = set()
    for e in range(mesh.n_elem):
        for a in en[e]:
            for b in en[e]:
                if a >= 0 and b >= 0:
                    pairs.add((int(a), int(b)))
    got = set()
    for a in range(mesh.n_nodes):
        cols = col_idx[row_ptr[a]:row_ptr[a + 1]]
        assert np.all(np.diff(cols) > 0)
        for b in cols:
            got.add((a, int(b)))
    assert got == pairs
    assert row_ptr.dtype == np.int32 and col_idx.dtype == np.int32


def test_pattern_counts_closed_form():
    """nnzb = (3m-2)^d for m interior nodes per axis (3 neighbours per axis
    except 2 at each end)."""
    for d, n in [(2, 32), (2, 1024), (3, 16)]:
        mesh = fem.Mesh(d, n)
        row_ptr, col_idx = fem.bsr_pattern(mesh)
        m = n - 1
        assert col_idx.shape[0] == (3 * m - 2) ** d
        assert row_ptr[-1] == (3 * m - 2) ** d


@pytest.mark.parametrize("d,n", [(2, 6), (3, 3)])
def test_symmetry_bitwise(d, n):
    """P2: A == A^T bit for bit (Section 4.1: A* symmetric)."""
    asm = fem.assemble(d, n, 1e-3, nu_elem=None)
    A = asm.matrix().toarray()
    assert np.array_equal(A, A.T)
    rng = np.random.default_rng(1)
    nu_e = np.exp(rng.standard_normal(n ** d))
    A2 = fem.assemble(d, n, 0.37, nu_elem=nu_e).matrix().toarray()
    assert np.array_equal(A2, A2.T)


@pytest.mark.parametrize("d,n", [(2, 7), (3, 4)])
def test_mass_kernel_is_V_bitwise(d, n):
    """P3: M_dev V = 0 exactly (span V = ker M, Eq. Vmatrix), also with
    per-element viscosity; and V^T V = I."""
    rng = np.random.default_rng(2)
    nu_e = np.exp(rng.standard_normal(n ** d))
    Mdev = fem.assemble(d, n, 1e-5, nu_elem=nu_e, div=False).matrix()
    V = fem.V_matrix(fem.Mesh(d, n))
    MV = (Mdev @ V).toarray()
    assert np.count_nonzero(MV) == 0
    assert np.allclose((V.T @ V).toarray(), np.eye(V.shape[1]), atol=1e-15)
    # and the complement is positive: M_dev is PSD with exactly n_s-dim kernel
    ev = np.linalg.eigvalsh(Mdev.toarray())
    ns = (n - 1) ** d
    assert np.sum(ev < 1e-10 * ev.max()) == ns


@pytest.mark.parametrize("d,n", [(2, 8), (2, 32), (3, 6)])
def test_inner_matrix_is_laplacian(d, n):
    """P4 (Corollary 1): V^T A V = L/d with L an independently built Q1
    Laplacian (1D Kronecker route); independent of dt and nu."""
    L = fem.laplacian_kron(d, n)
    rng = np.random.default_rng(3)
    for dt, nu_e in [(1e-1, None), (1e-6, None), (3e-3, np.exp(rng.standard_normal(n ** d)))]:
        asm = fem.assemble(d, n, dt, nu_elem=nu_e)
        V = fem.V_matrix(asm.mesh)
        Z = mg.inner_matrix(V, asm.matrix())
        diff = abs(Z - L / d).max()
        # 1e-13 relative to L, or the rounding of A's entries when the mass
        # part (~mt/dt) dwarfs the Laplacian part: each entry of V^T A V sums
        # d^2 entries of A carrying a relative error <= 2^-53 each.
        bound = max(1e-13 * abs(L).max(), d * d * 2.0 ** -52 * abs(asm.matrix()).max())
        assert diff <= bound, (dt, diff, bound)
        if dt >= 1e-3:
            assert diff <= 1e-13 * abs(L).max()


@pytest.mark.parametrize("d", [2, 3])
def test_laplacian_textbook_stencil(d):
    """Interior row of V^T A V * d equals the textbook Q1 stencil."""
    g = _gold("q1_laplacian_stencils.json")["2d" if d == 2 else "3d"]
    n = 8
    h = 1.0 / n
    asm = fem.assemble(d, n, 1e-2)
    Z = mg.inner_matrix(fem.V_matrix(asm.mesh), asm.matrix()).toarray() * d
    m = n - 1
    c = [m // 2] * d
    lin = lambda cc: sum(cc[ax] * m ** ax for ax in range(d))
    scale = h ** g["h_power"]
    for off in itertools.product([-1, 0, 1], repeat=d):
        nz = sum(1 for o in off if o != 0)
        key = {0: "center", 1: "face" if d == 3 else "edge", 2: "edge" if d == 3 else "corner", 3: "corner"}[nz]
        want = g[key] * scale
        got = Z[lin(c), lin([c[ax] + off[ax] for ax in range(d)])]
        assert math.isclose(got, want, rel_tol=1e-13, abs_tol=1e-15), (off, got, want)


@pytest.mark.parametrize("d,n", [(2, 5), (3, 3)])
def test_spmv_assembled_equals_elementwise(d, n):
    """Assembled BSR product == element-by-element product == per-row product."""
    rng = np.random.default_rng(4)
    nu_e = np.exp(rng.standard_normal(n ** d))
    for nu_elem in [None, nu_e]:
        asm = fem.assemble(d, n, 2e-3, nu_elem=nu_elem)
        x = rng.uniform(-1, 1, asm.mesh.n_unknowns)
        y1 = asm.matrix() @ x
        y2 = fem.apply_elementwise(asm.mesh, 2e-3, x, nu_elem=nu_elem)
        nodes = np.arange(asm.mesh.n_nodes)
        y3 = fem.rows_of_Ax(asm.mesh, 2e-3, x, nodes, nu_elem=nu_elem).reshape(-1)
        s = np.abs(y1).max()
        assert np.allclose(y1, y2, rtol=0, atol=1e-13 * s)
        assert np.allclose(y1, y3, rtol=0, atol=1e-13 * s)


def test_block_structural_nonzeros():
    """A_ab has the structural pattern of D_d (+) kron(I, G): 10 of 16 entries
    in 2D, 33 of 81 in 3D (Section 3.1 block structure)."""
    for d, want in [(2, 10), (3, 33)]:
        D = fem.dev_matrix(d) != 0
        K = np.kron(np.eye(d), np.ones((d, d))) != 0
        assert np.count_nonzero(D | K) == want
        asm = fem.assemble(d, 4, 1e-3)
        nz = np.any(asm.values != 0, axis=0)
        assert np.count_nonzero(nz) == want
        assert np.array_equal(nz, D | K)


def test_spd():
    """A is SPD (ker M cap ker A_div = {0}, Section 2.4)."""
    for d, n in [(2, 4), (3, 3)]:
        A = fem.assemble(d, n, 1e-6).matrix().toarray()
        assert np.linalg.eigvalsh(A).min() > 0


def test_input_generators_follow_their_recipes():
    """The seeded inputs: uniform[-1,1) right-hand sides, lognormal(0,1)
    viscosities, batched sizes log-uniform in [64,512] rounded to multiples
    of 16 and dt log-uniform in [1e-6,1e-1]; deterministic per seed."""
    from paper_2606_13429_gb300 import inputs
    f = inputs.rhs(3, 200_000)
    assert f.min() >= -1.0 and f.max() < 1.0
    assert abs(f.mean()) < 0.01 and abs(f.var() - 1.0 / 3.0) < 0.01
    assert np.array_equal(f, inputs.rhs(3, 200_000)) and not np.array_equal(f, inputs.rhs(4, 200_000))
    assert not np.array_equal(inputs.rhs(3, 1000, p=1), inputs.rhs(3, 1000, p=2))
    nu = inputs.nu_elements(4, 200_000)
    g = np.log(nu)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1.0) < 0.01
    plist = inputs.batched_problems(11, 4096)
    ns = np.array([n for n, _ in plist])
    dts = np.array([dt for _, dt in plist])
    assert ns.min() >= 64 and ns.max() <= 512 and np.all(ns % 16 == 0)
    assert dts.min() >= 1e-6 and dts.max() <= 1e-1
    # log-uniform: log10(dt) spread evenly over [-6, -1]
    h, _ = np.histogram(np.log10(dts), bins=5, range=(-6, -1))
    assert h.min() > 0.15 * len(dts)
    assert abs(np.mean(np.log(ns)) - (math.log(64) + math.log(512)) / 2) < 0.05
