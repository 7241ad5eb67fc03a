"""GPU parity: every kernel of the hot path, called through the C ABI, against
the FP64 oracle on the same seeded inputs.

Bars: indices bit-exact; FP64 assembly values to 1e-14 relative; FP64 SpMV,
embed/extract and stencil products to 1e-12; FP64 smoother, coarse solve and
W-cycles to 1e-10; solves at true relative residual 1e-8 to 1e-7 relative
error with outer iteration counts within +-2. Mixed precision (FP32
W-cycle) is held to its own bars (FP32 rounding, ~1e-5) and the same
true-residual target. Kernel-level comparisons are element by element:
max |gpu - oracle| over max |oracle| (a wrong boundary row or tile seam
cannot hide behind a norm).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem, mg, solvers
from paper_2606_13429_gb300 import dcg, inputs

pytestmark = pytest.mark.gpu

SMALL = [(2, 32), (2, 21), (3, 8), (3, 11)]


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


def maxrel(a, b):
    """Element-wise error: max |a - b| / max |b|."""
    a, b = np.asarray(a), np.asarray(b)
    assert a.shape == b.shape
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def mg_opts(patch=4, overlap=1, m1=2, m2=2, max_levels=4, weights="multiplicity"):
    return mg.MGOptions(patch=patch, overlap=overlap, m1=m1, m2=m2, max_levels=max_levels, ras_weights=weights)


def gpu_opts(o: mg.MGOptions, **kw):
    kw.setdefault("stall_window", 0)  # the oracle's default: Algorithm 2 without the stall rule
    return dcg.options(patch=o.patch, overlap=o.overlap, m1=o.m1, m2=o.m2, max_levels=o.max_levels,
                       ras_weights=dcg.DCG_RAS_RESTRICTED if o.ras_weights == "restricted" else dcg.DCG_RAS_MULTIPLICITY,
                       **kw)


# --------------------------------------------------------------------------- assembly


@pytest.mark.parametrize("d,n", SMALL + [(2, 1024), (3, 48)])
def test_pattern_bit_exact(d, n):
    prob = dcg.dcg_assemble(d, n, 1e-3)
    rp, ci = dcg.dcg_export_pattern(prob)
    rp_o, ci_o = fem.bsr_pattern(fem.Mesh(d, n))
    assert np.array_equal(rp, rp_o) and np.array_equal(ci, ci_o)


@pytest.mark.parametrize("d,n", [(2, 32), (2, 7), (3, 8), (3, 5)])
@pytest.mark.parametrize("dt", [1e-1, 1e-6])
@pytest.mark.parametrize("per_elem", [False, True])
def test_values(d, n, dt, per_elem):
    nu_e = inputs.nu_elements(5, n ** d) if per_elem else None
    prob = dcg.dcg_assemble(d, n, dt, nu=1.0, nu_elem=nu_e)
    v = dcg.dcg_export_values(prob)
    asm = fem.assemble(d, n, dt, nu_elem=nu_e)
    scale = np.abs(asm.values).max()
    assert np.abs(v - asm.values).max() <= 1e-14 * scale
    # the assembly uses round-to-nearest operations in the oracle's order
    assert np.mean(v == asm.values) > 0.999


# --------------------------------------------------------------------------- SpMV and deflation


@pytest.mark.parametrize("d,n", SMALL)
@pytest.mark.parametrize("dt", [1e-1, 1e-4])
def test_spmv(d, n, dt):
    asm = fem.assemble(d, n, dt)
    prob = dcg.dcg_assemble(d, n, dt)
    x = inputs.rhs(7, asm.mesh.n_unknowns)
    y = torch.empty(prob.N, dtype=torch.float64, device="cuda")
    dcg.dcg_spmv(prob, dev(x), y)
    assert maxrel(host(y), asm.matrix() @ x) <= 1e-12


@pytest.mark.parametrize("d,n", [(2, 1024), (3, 128)])
def test_spmv_full_size_sampled_rows(d, n):
    """The bench's operators: sampled block rows against the oracle's
    one-node-at-a-time product (first, last, boundary and random nodes)."""
    dt = 1e-4
    prob = dcg.dcg_assemble(d, n, dt)
    mesh = fem.Mesh(d, n)
    x = inputs.rhs(11, mesh.n_unknowns)
    y = torch.empty(prob.N, dtype=torch.float64, device="cuda")
    dcg.dcg_spmv(prob, dev(x), y)
    yh = host(y).reshape(mesh.n_nodes, mesh.b)
    rng = np.random.default_rng(0)
    nodes = np.unique(np.concatenate([[0, 1, mesh.m - 1, mesh.m, mesh.n_nodes // 2, mesh.n_nodes - 1],
                                      rng.integers(0, mesh.n_nodes, 40)]))
    want = fem.rows_of_Ax(mesh, dt, x, nodes)
    assert maxrel(yh[nodes], want) <= 1e-12
    prob.close()


@pytest.mark.parametrize("d,n", [(2, 21), (3, 8)])
def test_embed_extract(d, n):
    prob = dcg.dcg_assemble(d, n, 1e-3)
    mesh = fem.Mesh(d, n)
    y = inputs.rhs(3, mesh.n_unknowns)
    q = torch.empty(prob.n_nodes, dtype=torch.float64, device="cuda")
    dcg.dcg_extract(prob, dev(y), q)
    assert maxrel(host(q), fem.extract(mesh, y)) <= 1e-15
    qq = inputs.rhs(4, mesh.n_nodes)
    yy = torch.empty(prob.N, dtype=torch.float64, device="cuda")
    dcg.dcg_embed(prob, dev(qq), yy)
    assert np.array_equal(host(yy), fem.embed(mesh, qq))


# --------------------------------------------------------------------------- multigrid pieces


def _pair(d, n, dt, o: mg.MGOptions, precision=dcg.DCG_FP64):
    asm = fem.assemble(d, n, dt)
    V = fem.V_matrix(asm.mesh)
    H = mg.Hierarchy(d, n, mg.inner_matrix(V, asm.matrix()), o)
    prob = dcg.dcg_assemble(d, n, dt)
    dcg.dcg_setup(prob, gpu_opts(o, precision=precision))
    return asm, H, prob


@pytest.mark.parametrize("d,n", [(2, 32), (2, 20), (3, 8), (3, 12)])
@pytest.mark.parametrize("dt", [1e-1, 1e-6])
def test_inner_operator(d, n, dt):
    asm, H, prob = _pair(d, n, dt, mg_opts())
    assert prob.levels == H.J
    z = inputs.rhs(9, asm.mesh.n_nodes)
    y = torch.empty_like(dev(z))
    dcg.dcg_inner_apply(prob, dev(z), y)
    assert maxrel(host(y), H.levels[-1].Z @ z) <= 1e-12


@pytest.mark.parametrize("d,n,P,o", [(2, 32, 4, 1), (2, 20, 4, 1), (2, 32, 8, 2), (3, 8, 4, 1), (3, 12, 4, 1),
                                     (2, 24, 3, 1), (2, 16, 1, 0)])
@pytest.mark.parametrize("weights", ["multiplicity", "restricted"])
def test_ras_step(d, n, P, o, weights):
    asm, H, prob = _pair(d, n, 1e-3, mg_opts(patch=P, overlap=o, weights=weights))
    for k in range(2, H.J + 1):
        nn = H.levels[k - 1].Z.shape[0]
        f = inputs.rhs(20 + k, nn)
        z = inputs.rhs(40 + k, nn)
        zt = dev(z)
        dcg.dcg_ras_step(prob, k, dev(f), zt)
        assert maxrel(host(zt), H.ras_step(k, f, z)) <= 1e-11, k


@pytest.mark.parametrize("d,n", [(2, 32), (2, 64), (3, 8), (3, 16), (2, 2), (2, 3)])
def test_coarse_solve(d, n):
    asm, H, prob = _pair(d, n, 1e-3, mg_opts())
    nn = H.levels[0].Z.shape[0]
    f = inputs.rhs(5, nn)
    z = torch.empty_like(dev(f))
    dcg.dcg_coarse_solve(prob, dev(f), z)
    assert maxrel(host(z), H.coarse_solve(f)) <= 1e-11


@pytest.mark.parametrize("d,n,P,o", [(2, 32, 4, 1), (2, 40, 4, 1), (3, 8, 4, 1), (3, 16, 4, 1), (2, 64, 8, 2)])
def test_wcycles(d, n, P, o):
    asm, H, prob = _pair(d, n, 1e-3, mg_opts(patch=P, overlap=o))
    g = inputs.rhs(13, asm.mesh.n_nodes)
    for ncyc in [1, 3]:
        zt = torch.zeros(prob.n_nodes, dtype=torch.float64, device="cuda")
        dcg.dcg_mg_cycles(prob, dev(g), zt, ncyc)
        z = np.zeros_like(g)
        for _ in range(ncyc):
            z = H.wcycle(g, z)
        assert maxrel(host(zt), z) <= 1e-10, ncyc


@pytest.mark.parametrize("d,n", [(2, 32), (3, 8)])
def test_wcycles_mixed(d, n):
    asm, H, prob = _pair(d, n, 1e-3, mg_opts(), precision=dcg.DCG_MIXED)
    g = inputs.rhs(13, asm.mesh.n_nodes)
    zt = torch.zeros(prob.n_nodes, dtype=torch.float64, device="cuda")
    dcg.dcg_mg_cycles(prob, dev(g), zt, 1)
    z = H.wcycle(g, np.zeros_like(g))
    assert maxrel(host(zt), z) <= 1e-5
    # FP64 residuals make the FP32 cycle converge to FP64 accuracy
    zt.zero_()
    ncyc = dcg.dcg_mg_solve(prob, dev(g), zt, 1e-11)
    zo, no = H.multigrid(g, 1e-11, 100)
    assert maxrel(host(zt), zo) <= 1e-9
    assert abs(ncyc - no) <= 2


@pytest.mark.parametrize("d,n", [(2, 32), (3, 8)])
def test_mg_solve_counts(d, n):
    asm, H, prob = _pair(d, n, 1e-3, mg_opts())
    g = inputs.rhs(17, asm.mesh.n_nodes)
    for tol in [1e-4, 1e-10]:
        zt = torch.zeros(prob.n_nodes, dtype=torch.float64, device="cuda")
        ncyc = dcg.dcg_mg_solve(prob, dev(g), zt, tol)
        zo, no = H.multigrid(g, tol, 100)
        assert ncyc == no
        assert maxrel(host(zt), zo) <= 1e-9


# --------------------------------------------------------------------------- solves


RULES = {"fixed": dcg.DCG_INNER_FIXED, "adaptive": dcg.DCG_INNER_ADAPTIVE, "exact": dcg.DCG_INNER_EXACT}
RECS = {"fcg1": dcg.DCG_FCG1, "fr": dcg.DCG_FR, "fcg_inf": dcg.DCG_FCG_INF}


def _solve_pair(d, n, dt, o: mg.MGOptions, rule="fixed", rec="fcg1", c=0.01, precision=dcg.DCG_FP64, seed=0,
                deflate=True, m_max=None, ras_inverse=dcg.DCG_INV_FP32, max_it=100000):
    asm = fem.assemble(d, n, dt)
    f = inputs.rhs(seed, asm.mesh.n_unknowns)
    prob = dcg.dcg_assemble(d, n, dt)
    dcg.dcg_setup(prob, gpu_opts(o, inner_rule=RULES[rule], recurrence=RECS[rec], c=c, precision=precision,
                                 deflate=int(deflate), fcg_max_dirs=m_max or 0, ras_inverse=ras_inverse))
    x = torch.zeros(prob.N, dtype=torch.float64, device="cuda")
    st = dcg.dcg_solve(prob, dev(f), x, tol=1e-8, max_it=max_it)
    if deflate:
        x_o, st_o = solvers.FDCG(asm, solvers.FDCGOptions(mg=o, inner_rule=rule, recurrence=rec, c=c,
                                                          m_max=m_max)).solve(f, max_it=max_it)
    else:
        x_o, st_o = solvers.plain_cg(asm.matrix(), f, max_it=max_it)
    return host(x), st, x_o, st_o, asm, f


@pytest.mark.parametrize("d,n,dt", [(2, 32, 1e-3), (2, 32, 1e-6), (2, 21, 1e-2), (3, 8, 1e-4), (3, 11, 1e-1)])
def test_plain_cg(d, n, dt):
    x, st, x_o, st_o, asm, f = _solve_pair(d, n, dt, mg_opts(), deflate=False)
    assert st["status"] == dcg.DCG_OK and st["true_relres"] <= 1e-8
    assert abs(st["outer_its"] - st_o.outer_its) <= 2
    assert relerr(x, x_o) <= 1e-7


@pytest.mark.parametrize("d,n,dt", [(2, 32, 1e-3), (2, 32, 1e-1), (2, 32, 1e-6), (2, 20, 1e-4), (3, 8, 1e-4),
                                    (3, 12, 1e-2)])
@pytest.mark.parametrize("rule", ["fixed", "adaptive", "exact"])
def test_dcg_fp64(d, n, dt, rule):
    x, st, x_o, st_o, asm, f = _solve_pair(d, n, dt, mg_opts(), rule=rule)
    assert st["status"] == dcg.DCG_OK and st["true_relres"] <= 1e-8, st
    assert st["restarts"] == 0 and st_o.restarts == 0
    assert abs(st["outer_its"] - st_o.outer_its) <= 2, (st, st_o.outer_its)
    if rule != "exact":
        assert abs(st["total_mg_cycles"] - st_o.total_mg_cycles) <= max(4, 0.05 * st_o.total_mg_cycles)
    assert relerr(x, x_o) <= 1e-7
    A = asm.matrix()
    assert np.linalg.norm(f - A @ x) <= 1e-8 * np.linalg.norm(f)


@pytest.mark.parametrize("rec", ["fr", "fcg_inf"])
def test_dcg_recurrences(rec):
    x, st, x_o, st_o, asm, f = _solve_pair(2, 32, 1e-4, mg_opts(), rec=rec)
    assert st["status"] == dcg.DCG_OK and st["true_relres"] <= 1e-8
    assert st["restarts"] == 0 and st_o.restarts == 0
    assert abs(st["outer_its"] - st_o.outer_its) <= 2
    assert relerr(x, x_o) <= 1e-7
    assert st["fcg_truncated"] == 0


@pytest.mark.parametrize("window", [0, 50])
def test_dcg_stall_restart(window):
    """Loose inner tolerance at dt = 0.1: without the stall restart both the
    GPU solver and the oracle stagnate; with it both reach 1e-8 after
    restarting from the true residual."""
    o = mg_opts(patch=4, overlap=1, max_levels=2)
    asm = fem.assemble(2, 24, 0.1)
    f = inputs.rhs(5, asm.mesh.n_unknowns)
    prob = dcg.dcg_assemble(2, 24, 0.1)
    dcg.dcg_setup(prob, gpu_opts(o, c=50.0, stall_window=window))
    x = torch.zeros(prob.N, dtype=torch.float64, device="cuda")
    st = dcg.dcg_solve(prob, dev(f), x, tol=1e-8, max_it=1500)
    x_o, st_o = solvers.FDCG(asm, solvers.FDCGOptions(mg=o, c=50.0, stall_window=window)).solve(f, max_it=1500)
    if window == 0:
        assert st["status"] == dcg.DCG_ERR_NOT_CONVERGED and st["true_relres"] > 1e-6
        assert not st_o.converged
    else:
        assert st["status"] == dcg.DCG_OK and st["true_relres"] <= 1e-8 and st["restarts"] >= 1
        assert st_o.converged
        assert st["restarts"] == st_o.restarts
        assert abs(st["outer_its"] - st_o.outer_its) <= 2
        assert relerr(host(x), x_o) <= 1e-7


@pytest.mark.parametrize("d,n,dt", [(2, 32, 1e-3), (2, 64, 1e-5), (3, 8, 1e-4)])
def test_dcg_mixed(d, n, dt):
    x, st, x_o, st_o, asm, f = _solve_pair(d, n, dt, mg_opts(), precision=dcg.DCG_MIXED)
    assert st["status"] == dcg.DCG_OK and st["true_relres"] <= 1e-8
    assert st["restarts"] == 0
    assert abs(st["outer_its"] - st_o.outer_its) <= 3
    assert relerr(x, x_o) <= 1e-7


def test_dcg_cfg2_patches():
    """The large-config smoother (8x8 cores, overlap 2) at a size the oracle
    finishes in seconds."""
    x, st, x_o, st_o, asm, f = _solve_pair(2, 64, 1e-5, mg_opts(patch=8, overlap=2))
    assert st["status"] == dcg.DCG_OK and abs(st["outer_its"] - st_o.outer_its) <= 2
    assert relerr(x, x_o) <= 1e-7


# --------------------------------------------------------------------------- edge cases


def test_edge_cases():
    d, n, dt = 2, 16, 1e-3
    prob = dcg.dcg_assemble(d, n, dt)
    dcg.dcg_setup(prob, dcg.options())
    N = prob.N
    # zero right-hand side
    x = torch.ones(N, dtype=torch.float64, device="cuda")
    st = dcg.dcg_solve(prob, torch.zeros(N, dtype=torch.float64, device="cuda"), x)
    assert st["status"] == dcg.DCG_OK and st["outer_its"] == 0 and not x.any().item()
    # iteration cap
    f = dev(inputs.rhs(0, N))
    x = torch.zeros_like(f)
    st = dcg.dcg_solve(prob, f, x, tol=1e-12, max_it=3)
    assert st["status"] == dcg.DCG_ERR_NOT_CONVERGED and st["outer_its"] == 3
    # warm start from the solution
    x = torch.zeros_like(f)
    dcg.dcg_solve(prob, f, x, tol=1e-10)
    st = dcg.dcg_solve(prob, f, x, tol=1e-10)
    assert st["outer_its"] <= 1 and st["true_relres"] <= 1e-10
    # host-array entry point gives the same answer
    xh = np.zeros(N)
    st_h = dcg.dcg_solve_host(prob, inputs.rhs(0, N), xh, tol=1e-10)
    assert st_h["status"] == dcg.DCG_OK and relerr(xh, host(x)) <= 1e-9
    # invalid options
    with pytest.raises(dcg.DCGError):
        dcg.dcg_setup(prob, dcg.options(overlap=9, patch=4))
    with pytest.raises(dcg.DCGError):
        dcg.dcg_setup(prob, dcg.options(patch=16, overlap=1))
    with pytest.raises(dcg.DCGError):
        dcg.dcg_setup(prob, dcg.options(device_loop=2))


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_tiny_meshes_dense(n):
    """Degenerate sizes (one interior node per axis and up): dense solve."""
    for d in (2, 3):
        asm = fem.assemble(d, n, 1e-2)
        f = inputs.rhs(1, asm.mesh.n_unknowns)
        x_ref = solvers.dense_solve(asm, f)
        prob = dcg.dcg_assemble(d, n, 1e-2)
        dcg.dcg_setup(prob, dcg.options())
        x = torch.zeros(prob.N, dtype=torch.float64, device="cuda")
        st = dcg.dcg_solve(prob, dev(f), x, tol=1e-12)
        assert st["status"] == dcg.DCG_OK
        assert relerr(host(x), x_ref) <= 1e-9


def test_batched_matches_single():
    probs, fs, xs, ref = [], [], [], []
    for p, (n, dt) in enumerate([(16, 1e-3), (24, 1e-5)]):
        prob = dcg.dcg_assemble(2, n, dt)
        dcg.dcg_setup(prob, dcg.options())
        probs.append(prob)
        for r in range(2):
            f = dev(inputs.rhs(0, prob.N, p=p, r=r))
            fs.append(f)
            xs.append(torch.zeros_like(f))
            x1 = torch.zeros_like(f)
            dcg.dcg_solve(prob, f, x1)
            ref.append(host(x1))
    code, stats = dcg.dcg_solve_batched(probs, 2, fs, xs)
    assert code == dcg.DCG_OK
    for k in range(4):
        assert stats[k]["true_relres"] <= 1e-8
        assert relerr(host(xs[k]), ref[k]) <= 1e-9


def _uneven_batch(nprob=20, nrhs=3):
    """Problems of both dimensions, several sizes, time steps and precisions
    (more problems than the library's 16 batch workers)."""
    probs, fs = [], []
    for p in range(nprob):
        d = 3 if p % 5 == 4 else 2
        n = [16, 24, 32, 40][p % 4] if d == 2 else [8, 12][p % 2]
        dt = [1e-6, 1e-4, 1e-2][p % 3]
        prob = dcg.dcg_assemble(d, n, dt)
        dcg.dcg_setup(prob, dcg.options(precision=dcg.DCG_MIXED if p % 2 else dcg.DCG_FP64))
        probs.append(prob)
        for r in range(nrhs):
            fs.append(dev(inputs.rhs(7, prob.N, p=p, r=r)))
    return probs, fs


def test_batched_uneven_equals_sequential_bitwise():
    """Concurrent batched solves give the same bits as one-at-a-time solves:
    every reduction is deterministic and independent of the stream."""
    nrhs = 3
    probs, fs = _uneven_batch(20, nrhs)
    seq, seq_stats = [], []
    for k, f in enumerate(fs):
        x = torch.zeros_like(f)
        seq_stats.append(dcg.dcg_solve(probs[k // nrhs], f, x))
        seq.append(host(x))
    xs = [torch.zeros_like(f) for f in fs]
    code, stats = dcg.dcg_solve_batched(probs, nrhs, fs, xs)
    assert code == dcg.DCG_OK
    for k in range(len(fs)):
        assert stats[k]["status"] == dcg.DCG_OK
        assert stats[k]["true_relres"] <= 1e-8
        assert stats[k]["outer_its"] == seq_stats[k]["outer_its"]
        assert stats[k]["total_mg_cycles"] == seq_stats[k]["total_mg_cycles"]
        assert np.array_equal(host(xs[k]), seq[k])


def test_batched_orders_against_caller_stream():
    """Work queued on the caller's stream before the call is seen by the
    batch, and work queued after it sees the solutions."""
    probs, fs = _uneven_batch(4, 2)
    ref = []
    for k, f in enumerate(fs):
        x = torch.zeros_like(f)
        dcg.dcg_solve(probs[k // 2], f, x)
        ref.append(host(x))
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        big = torch.empty(1 << 26, dtype=torch.float64, device="cuda")
        big.normal_()  # a long kernel ahead of the inputs on s
        f2 = [f * 1.0 + 0.0 * big[: f.numel()] for f in fs]
        xs = [torch.zeros_like(f) for f in fs]
        code, _ = dcg.dcg_solve_batched(probs, 2, f2, xs, stream=s.cuda_stream)
        out = [x.clone() for x in xs]
    s.synchronize()
    assert code == dcg.DCG_OK
    for k in range(len(fs)):
        assert np.array_equal(out[k].cpu().numpy(), ref[k])


def test_batched_not_converged_reports_per_pair():
    probs, fs = _uneven_batch(3, 2)
    xs = [torch.zeros_like(f) for f in fs]
    code, stats = dcg.dcg_solve_batched(probs, 2, fs, xs, max_it=1)
    assert code == dcg.DCG_ERR_NOT_CONVERGED
    assert all(st["status"] == dcg.DCG_ERR_NOT_CONVERGED for st in stats)
    assert all(st["true_relres"] > 1e-8 for st in stats)


def test_batched_rejects_duplicates_and_unset_problems():
    prob = dcg.dcg_assemble(2, 16, 1e-3)
    f = dev(inputs.rhs(0, prob.N))
    x1, x2 = torch.zeros_like(f), torch.zeros_like(f)
    with pytest.raises(dcg.DCGError):
        dcg.dcg_solve_batched([prob], 1, [f], [x1])  # not set up
    dcg.dcg_setup(prob, dcg.options())
    with pytest.raises(dcg.DCGError):
        dcg.dcg_solve_batched([prob, prob], 1, [f, f], [x1, x2])


@pytest.mark.parametrize("d,n,prec", [(2, 64, dcg.DCG_MIXED), (2, 48, dcg.DCG_FP64), (3, 16, dcg.DCG_FP64)])
def test_autotune_picks_a_valid_candidate(d, n, prec):
    prob = dcg.dcg_assemble(d, n, 1e-4)
    f = dev(inputs.rhs(3, prob.N))
    best, ms = dcg.dcg_autotune(prob, f, dcg.options(precision=prec), inner_tol=1e-6, reps=2)
    assert ms > 0
    assert best.precision == prec
    assert (best.patch, best.overlap) in [(4, 1), (8, 1), (8, 2), (12, 2)]
    assert (best.patch + 2 * best.overlap) ** d <= 256
    assert 2 <= best.max_levels <= 4
    if prec == dcg.DCG_FP64:
        assert best.ras_inverse == dcg.DCG_INV_FP32
    # the problem is left set up with the winner, and it solves
    assert prob.levels == len(mg.level_sizes(n, best.max_levels))
    x = torch.zeros_like(f)
    st = dcg.dcg_solve(prob, f, x)
    assert st["status"] == dcg.DCG_OK and st["true_relres"] <= 1e-8
    x_ref = torch.zeros_like(f)
    prob2 = dcg.dcg_assemble(d, n, 1e-4)
    dcg.dcg_setup(prob2, best)
    dcg.dcg_solve(prob2, f, x_ref)
    assert np.array_equal(host(x), host(x_ref))


# --------------------------------------------------------------------------- tensor-core RAS (BF16 inverses)


@pytest.mark.parametrize("d,n,P,o", [(2, 32, 4, 1), (2, 64, 8, 2), (3, 12, 4, 1)])
def test_ras_step_tensor_cores(d, n, P, o):
    """RAS step with BF16 inverses and BF16 residuals on tcgen05 (FP32
    accumulation): the update z_new - z matches the oracle's to BF16 rounding
    (8 significant bits per operand)."""
    asm, H, prob = _pair(d, n, 1e-3, mg_opts(patch=P, overlap=o), precision=dcg.DCG_MIXED)
    dcg.dcg_setup(prob, gpu_opts(mg_opts(patch=P, overlap=o), precision=dcg.DCG_MIXED, ras_inverse=dcg.DCG_INV_BF16))
    for k in range(2, H.J + 1):
        nn = H.levels[k - 1].Z.shape[0]
        f = inputs.rhs(20 + k, nn)
        z = inputs.rhs(40 + k, nn)
        zt = dev(z)
        dcg.dcg_ras_step(prob, k, dev(f), zt)
        want = H.ras_step(k, f, z) - z
        got = host(zt) - z
        assert relerr(got, want) <= 2e-2, (k, relerr(got, want))


@pytest.mark.parametrize("d,n,dt", [(2, 64, 1e-5), (3, 12, 1e-4)])
def test_dcg_tensor_cores(d, n, dt):
    x, st, x_o, st_o, asm, f = _solve_pair(d, n, dt, mg_opts(), precision=dcg.DCG_MIXED)
    prob = dcg.dcg_assemble(d, n, dt)
    dcg.dcg_setup(prob, gpu_opts(mg_opts(), precision=dcg.DCG_MIXED, ras_inverse=dcg.DCG_INV_BF16))
    xt = torch.zeros(prob.N, dtype=torch.float64, device="cuda")
    st2 = dcg.dcg_solve(prob, dev(f), xt, tol=1e-8)
    assert st2["status"] == dcg.DCG_OK and st2["true_relres"] <= 1e-8
    assert abs(st2["outer_its"] - st_o.outer_its) <= 3
    assert relerr(host(xt), x_o) <= 1e-7
    # BF16 smoothing costs at most a few extra W-cycles per inner solve
    assert st2["total_mg_cycles"] <= 2 * st_o.total_mg_cycles
