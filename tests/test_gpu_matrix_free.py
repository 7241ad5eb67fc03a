"""GPU parity of the matrix-free 3D operator (element-by-element product,
regrouped per output node) against the oracle's element-by-element product,
the assembled BSR product, and sampled rows at the full 256^3 size; and the
deflated CG solver driven by it.

Bars: FP64 products to 1e-12 relative (1e-13 against BSR); FP32 products to
1e-5 relative (single-precision arithmetic over ~100 terms per row); solves
at true relative residual 1e-8 to 1e-7 relative error, FP64 outer iteration
counts within +-2 of the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem, mg, solvers
from paper_2606_13429_gb300 import dcg, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2606_13429_gb300 import build
    build.build()
    dcg.load()
    torch.cuda.set_device(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _nu(n, lognormal):
    return inputs.nu_elements(4, n ** 3) if lognormal else None


@pytest.mark.parametrize("n", [4, 8, 11, 37])
@pytest.mark.parametrize("dt", [1e-1, 1e-5])
@pytest.mark.parametrize("lognormal", [False, True])
def test_mf_product_matches_oracle(n, dt, lognormal):
    """n = 37 spans two 32-node tiles in x, several in y and z chunks, with
    ragged edges; n = 4 is the smallest mesh the operator accepts."""
    nu = _nu(n, lognormal)
    prob = dcg.dcg_assemble(3, n, dt, nu_elem=nu, matrix_free=True)
    mesh = fem.Mesh(3, n)
    x = inputs.rhs(2, mesh.n_unknowns)
    ref = fem.apply_elementwise(mesh, dt, x, nu_elem=nu)
    y = torch.empty(prob.N, dtype=torch.float64, device="cuda")
    dcg.dcg_spmv(prob, dev(x), y)
    assert relerr(host(y), ref) <= 1e-12
    dcg.dcg_spmv_prec(prob, dev(x), y, dcg.DCG_MIXED)
    assert relerr(host(y), ref) <= 1e-5


@pytest.mark.parametrize("n,lognormal", [(9, True), (16, False)])
def test_mf_equals_assembled(n, lognormal):
    nu = _nu(n, lognormal)
    pa = dcg.dcg_assemble(3, n, 1e-4, nu_elem=nu)
    pm = dcg.dcg_assemble(3, n, 1e-4, nu_elem=nu, matrix_free=True)
    assert pm.nnzb == 0 and pm.N == pa.N
    x = dev(inputs.rhs(6, pa.N))
    ya, ym = torch.empty_like(x), torch.empty_like(x)
    dcg.dcg_spmv(pa, x, ya)
    dcg.dcg_spmv(pm, x, ym)
    assert relerr(host(ym), host(ya)) <= 1e-13


def test_mf_full_size_sampled_rows():
    """256^3 elements (255^3 interior nodes, 149,232,375 unknowns), lognormal
    nu: sampled block rows of the product against the oracle computed one
    node at a time (corners, faces, tile seams and random nodes)."""
    n = 256
    m = n - 1
    nu = inputs.nu_elements(4, n ** 3)
    prob = dcg.dcg_assemble(3, n, 1e-5, nu_elem=nu, matrix_free=True)
    mesh = fem.Mesh(3, n)
    x = inputs.rhs(8, mesh.n_unknowns)
    xd = dev(x)
    y = torch.empty_like(xd)
    rng = np.random.default_rng(0)
    picks = [(0, 0, 0), (m - 1, m - 1, m - 1), (31, 7, 0), (32, 8, 1), (m - 1, 0, 128), (0, m - 1, 63), (64, 64, 64)]
    nodes = [a + m * (b + m * c) for a, b, c in picks] + list(rng.integers(0, m ** 3, 25))
    nodes = np.array(nodes, dtype=np.int64)
    ref = fem.rows_of_Ax(mesh, 1e-5, x, nodes, nu_elem=nu)
    scale = np.abs(ref).max()
    idx = (nodes[:, None] * 9 + np.arange(9)[None, :]).reshape(-1)
    dcg.dcg_spmv(prob, xd, y)
    got = y[torch.from_numpy(idx).cuda()].cpu().numpy().reshape(-1, 9)
    assert np.abs(got - ref).max() <= 1e-12 * scale
    dcg.dcg_spmv_prec(prob, xd, y, dcg.DCG_MIXED)
    got = y[torch.from_numpy(idx).cuda()].cpu().numpy().reshape(-1, 9)
    assert np.abs(got - ref).max() <= 1e-5 * scale


@pytest.mark.parametrize("n,dt", [(8, 1e-4), (12, 1e-2)])
def test_mf_dcg_fp64_matches_oracle(n, dt):
    nu = inputs.nu_elements(4, n ** 3)
    o = mg.MGOptions(patch=4, overlap=1, m1=2, m2=2, max_levels=4)
    asm = fem.assemble(3, n, dt, nu_elem=nu)
    f = inputs.rhs(0, asm.mesh.n_unknowns)
    x_o, st_o = solvers.FDCG(asm, solvers.FDCGOptions(mg=o)).solve(f)
    prob = dcg.dcg_assemble(3, n, dt, nu_elem=nu, matrix_free=True)
    dcg.dcg_setup(prob, dcg.options(patch=4, overlap=1, m1=2, m2=2, max_levels=4))
    x = torch.zeros(prob.N, dtype=torch.float64, device="cuda")
    st = dcg.dcg_solve(prob, dev(f), x, tol=1e-8)
    assert st["status"] == dcg.DCG_OK and st["true_relres"] <= 1e-8
    assert abs(st["outer_its"] - st_o.outer_its) <= 2, (st, st_o.outer_its)
    assert relerr(host(x), x_o) <= 1e-7


def test_mf_dcg_mixed_converges():
    """FP32 products inside the outer iterations, FP64 true residual: the
    solve still reaches 1e-8 and agrees with the FP64 matrix-free solve."""
    n, dt = 16, 1e-4
    nu = inputs.nu_elements(4, n ** 3)
    f = dev(inputs.rhs(0, 9 * (n - 1) ** 3))
    xs = {}
    for prec in (dcg.DCG_FP64, dcg.DCG_MIXED):
        prob = dcg.dcg_assemble(3, n, dt, nu_elem=nu, matrix_free=True)
        dcg.dcg_setup(prob, dcg.options(patch=4, overlap=1, precision=prec))
        x = torch.zeros_like(f)
        st = dcg.dcg_solve(prob, f, x, tol=1e-8)
        assert st["status"] == dcg.DCG_OK and st["true_relres"] <= 1e-8, st
        # the residual once more, from the FP64 product
        r = torch.empty_like(f)
        dcg.dcg_spmv(prob, x, r)
        assert torch.linalg.norm(f - r).item() <= 1.0001e-8 * torch.linalg.norm(f).item()
        xs[prec] = host(x)
    # two solutions at relative residual 1e-8 differ by at most cond(A) 2e-8
    assert relerr(xs[dcg.DCG_MIXED], xs[dcg.DCG_FP64]) <= 1e-4


def test_mf_rejects_unsupported():
    with pytest.raises(dcg.DCGError):
        dcg.dcg_assemble(2, 16, 1e-3, matrix_free=True)
    with pytest.raises(dcg.DCGError):
        dcg.dcg_assemble(3, 3, 1e-3, matrix_free=True)
    pa = dcg.dcg_assemble(3, 6, 1e-3)
    x = torch.zeros(pa.N, dtype=torch.float64, device="cuda")
    with pytest.raises(dcg.DCGError):
        dcg.dcg_spmv_prec(pa, x, torch.empty_like(x), dcg.DCG_MIXED)
