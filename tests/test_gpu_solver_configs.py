"""GPU parity of the configurations the bench times, of the truncated FCG,
and of the failure paths, through the C ABI against the FP64 oracle.

* The bench's hierarchy: two levels (the coarsest solved exactly by sine
  transforms of length 2(m+1) up to 1024), RAS 8x8 cores with overlap 2, in
  FP64 and in the mixed mode with BF16 inverses on the tensor cores.
* FCG with the truncation-restart rule m_i = max{1, mod(i, m_max+1)} (remark
  after Table 4) and the FCG(1) breakdown that motivates it (Tables 3-4).
* Batched pairs against the oracle, not only against sequential solves.
* Failure reporting made on the host: a NaN right-hand side, and the bounded
  device wait made to run out on an mbarrier nothing completes.
"""
import functools

import numpy as np
import pytest
import scipy.sparse.linalg as spla

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


def maxrel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


BENCH_MG = mg.MGOptions(patch=8, overlap=2, m1=2, m2=2, max_levels=2)


def gpu_opts(o: mg.MGOptions, **kw):
    kw.setdefault("stall_window", 0)
    return dcg.options(patch=o.patch, overlap=o.overlap, m1=o.m1, m2=o.m2, max_levels=o.max_levels, **kw)


# --------------------------------------------------------------------------- the bench's configuration


@pytest.mark.parametrize("d,n,levels", [(2, 256, 2), (2, 512, 2), (2, 1024, 2), (2, 96, 2), (3, 64, 2)])
def test_coarse_solve_long_transforms(d, n, levels):
    """The exact coarsest solve at the bench's sizes: m + 1 = 128, 256, 512
    (sine transforms by FFT of length 2(m+1) up to 1024) and 48 (dense
    passes), against a sparse LU of the Galerkin coarse matrix P^T Z_J P,
    Z_J = L / d (Corollary 1), element by element."""
    prob = dcg.dcg_assemble(d, n, 1e-4)
    dcg.dcg_setup(prob, dcg.options(max_levels=levels, patch=8 if d == 2 else 4, overlap=2 if d == 2 else 1))
    sizes = mg.level_sizes(n, levels)
    mc = sizes[-1] - 1
    ZJ = fem.laplacian_kron(d, n) / d
    P = mg.prolongation(d, mc)
    Zc = (P.T @ ZJ @ P).tocsc()
    nn = mc ** d
    assert prob.level_nodes(1) == nn
    for seed in (5, 6):
        f = inputs.rhs(seed, nn)
        z = torch.empty(nn, dtype=torch.float64, device="cuda")
        dcg.dcg_coarse_solve(prob, dev(f), z)
        want = spla.splu(Zc).solve(f)
        assert maxrel(host(z), want) <= 1e-11
    prob.close()


@functools.lru_cache(maxsize=None)
def _oracle_bench(n, dt):
    """The oracle's FDCG with the bench hierarchy (shared by the FP64 and the
    mixed-precision tests of the same case)."""
    asm = fem.assemble(2, n, dt)
    f = inputs.rhs(0, asm.mesh.n_unknowns)
    x_o, st_o = solvers.FDCG(asm, solvers.FDCGOptions(mg=BENCH_MG)).solve(f, max_it=20000)
    return asm, f, x_o, st_o


def _bench_pair(n, dt, precision, ras_inverse):
    asm, f, x_o, st_o = _oracle_bench(n, dt)
    prob = dcg.dcg_assemble(2, n, dt)
    dcg.dcg_setup(prob, gpu_opts(BENCH_MG, precision=precision, ras_inverse=ras_inverse))
    assert prob.levels == 2
    x = torch.zeros(prob.N, dtype=torch.float64, device="cuda")
    st = dcg.dcg_solve(prob, dev(f), x, tol=1e-8, max_it=20000)
    prob.close()
    return host(x), st, x_o, st_o, asm, f


@pytest.mark.parametrize("n,dt", [(128, 1e-6), (128, 1e-4), (256, 1e-6)])
def test_dcg_bench_config_mixed_bf16(n, dt):
    """The timed configuration of the mixed arm: 2 levels, 8x8 cores with
    overlap 2, FP32 W-cycle with BF16 inverses x BF16 residuals on tcgen05,
    FFT coarse solve; FP64 outer iteration. Against the FP64 oracle with the
    same hierarchy: counts within 3, solution within 1e-7, true residual 1e-8."""
    x, st, x_o, st_o, asm, f = _bench_pair(n, dt, dcg.DCG_MIXED, dcg.DCG_INV_BF16)
    assert st["status"] == dcg.DCG_OK and st["true_relres"] <= 1e-8, st
    assert st_o.converged and st_o.restarts == 0 and st["restarts"] == 0
    assert abs(st["outer_its"] - st_o.outer_its) <= 3, (st["outer_its"], st_o.outer_its)
    assert relerr(x, x_o) <= 1e-7
    assert np.linalg.norm(f - asm.matrix() @ x) <= 1e-8 * np.linalg.norm(f)


@pytest.mark.parametrize("n,dt", [(128, 1e-6), (128, 1e-4), (256, 1e-6)])
def test_dcg_bench_config_fp64(n, dt):
    """The timed configuration of the all-FP64 arm (the same hierarchy in
    FP64): counts within 2 and W-cycle totals within 5%."""
    x, st, x_o, st_o, asm, f = _bench_pair(n, dt, dcg.DCG_FP64, dcg.DCG_INV_FP32)
    assert st["status"] == dcg.DCG_OK and st["true_relres"] <= 1e-8, st
    assert st_o.restarts == 0 and st["restarts"] == 0
    assert abs(st["outer_its"] - st_o.outer_its) <= 2, (st["outer_its"], st_o.outer_its)
    assert abs(st["total_mg_cycles"] - st_o.total_mg_cycles) <= max(4, 0.05 * st_o.total_mg_cycles)
    assert relerr(x, x_o) <= 1e-7


@pytest.mark.parametrize("precision,inv", [(dcg.DCG_FP64, dcg.DCG_INV_FP32), (dcg.DCG_MIXED, dcg.DCG_INV_BF16)])
def test_wcycle_bench_config(precision, inv):
    """One W-cycle of the bench hierarchy at 256^2 (coarsest 127^2 by FFT),
    element by element against the oracle's Algorithm 4."""
    n = 256
    ZJ = fem.laplacian_kron(2, n) / 2
    H = mg.Hierarchy(2, n, ZJ, BENCH_MG)
    prob = dcg.dcg_assemble(2, n, 1e-4)
    dcg.dcg_setup(prob, gpu_opts(BENCH_MG, precision=precision, ras_inverse=inv))
    g = inputs.rhs(13, prob.n_nodes)
    zt = torch.zeros(prob.n_nodes, dtype=torch.float64, device="cuda")
    dcg.dcg_mg_cycles(prob, dev(g), zt, 1)
    z = H.wcycle(g, np.zeros_like(g))
    err = maxrel(host(zt), z)
    # FP64: rounding only; mixed: BF16 operands (8 significant bits) in the
    # smoother products, FP32 elsewhere
    assert err <= (1e-10 if precision == dcg.DCG_FP64 else 3e-2), err
    prob.close()


# --------------------------------------------------------------------------- truncated FCG


@pytest.mark.parametrize("m_max", [2, 4])
def test_fcg_truncation_restart_rule(m_max):
    """FCG(m_max) with the rule of the remark after Table 4, on a solve long
    enough for the truncation to act (the device reports how many directions
    it built from a truncated window), against the oracle's same rule."""
    o = mg.MGOptions(patch=4, overlap=1, max_levels=4)
    asm = fem.assemble(2, 32, 1e-4)
    f = inputs.rhs(0, asm.mesh.n_unknowns)
    prob = dcg.dcg_assemble(2, 32, 1e-4)
    dcg.dcg_setup(prob, gpu_opts(o, recurrence=dcg.DCG_FCG_INF, fcg_max_dirs=m_max, inner_rule=dcg.DCG_INNER_ADAPTIVE,
                                 c=0.05))
    x = torch.zeros(prob.N, dtype=torch.float64, device="cuda")
    st = dcg.dcg_solve(prob, dev(f), x, tol=1e-8)
    x_o, st_o = solvers.FDCG(asm, solvers.FDCGOptions(mg=o, recurrence="fcg_inf", m_max=m_max, inner_rule="adaptive",
                                                      c=0.05)).solve(f)
    assert st["status"] == dcg.DCG_OK and st_o.converged
    assert abs(st["outer_its"] - st_o.outer_its) <= 2
    # directions d_i with i > m_max and i mod (m_max + 1) < i: all but the first m_max
    assert st["fcg_truncated"] == max(0, st["outer_its"] - 1 - m_max)
    assert relerr(host(x), x_o) <= 1e-7


def test_fcg1_breakdown_and_fcg_inf_robustness():
    """Tables 3-4 on Q1: under a loose adaptive inner tolerance (c_A = 0.2,
    dt = 0.1) FCG(1) meets (d, M_D d) <= 0 and reports DCG_ERR_BREAKDOWN, like
    the oracle; FCG(inf) keeps reducing the residual without breakdown."""
    o = mg.MGOptions(patch=4, overlap=1, max_levels=2)
    asm = fem.assemble(2, 12, 0.1)
    f = inputs.rhs(5, asm.mesh.n_unknowns)
    prob = dcg.dcg_assemble(2, 12, 0.1)
    res = {}
    for rec in ("fcg1", "fcg_inf"):
        # fcg_max_dirs = 400 >= max_it: the untruncated FCG(inf) of Algorithm 1
        dcg.dcg_setup(prob, gpu_opts(o, recurrence=dcg.DCG_FCG1 if rec == "fcg1" else dcg.DCG_FCG_INF,
                                     inner_rule=dcg.DCG_INNER_ADAPTIVE, c=0.2, max_restarts=0, fcg_max_dirs=400))
        x = torch.zeros(prob.N, dtype=torch.float64, device="cuda")
        res[rec] = dcg.dcg_solve(prob, dev(f), x, tol=1e-8, max_it=400)
    _, s1 = solvers.FDCG(asm, solvers.FDCGOptions(mg=o, recurrence="fcg1", inner_rule="adaptive", c=0.2,
                                                  max_restarts=0)).solve(f, max_it=400)
    assert s1.breakdown
    assert res["fcg1"]["status"] == dcg.DCG_ERR_BREAKDOWN
    assert abs(res["fcg1"]["outer_its"] - s1.outer_its) <= 10
    assert res["fcg_inf"]["status"] == dcg.DCG_ERR_NOT_CONVERGED and res["fcg_inf"]["outer_its"] == 400
    assert res["fcg_inf"]["true_relres"] < 0.1 * res["fcg1"]["true_relres"]


# --------------------------------------------------------------------------- batched against the oracle


def test_batched_pairs_against_oracle():
    """Two problems of one batched call, a 2D and a 3D one with two
    right-hand sides each, against the oracle's FDCG."""
    specs = [(2, 24, 1e-5), (3, 8, 1e-4)]
    probs, fs, asms = [], [], []
    for p, (d, n, dt) in enumerate(specs):
        prob = dcg.dcg_assemble(d, n, dt)
        dcg.dcg_setup(prob, gpu_opts(mg.MGOptions()))
        probs.append(prob)
        asms.append(fem.assemble(d, n, dt))
        for r in range(2):
            fs.append(dev(inputs.rhs(3, prob.N, p=p, r=r)))
    xs = [torch.zeros_like(f) for f in fs]
    code, stats = dcg.dcg_solve_batched(probs, 2, fs, xs)
    assert code == dcg.DCG_OK
    for k in range(4):
        asm = asms[k // 2]
        x_o, st_o = solvers.FDCG(asm, solvers.FDCGOptions()).solve(host(fs[k]))
        assert stats[k]["true_relres"] <= 1e-8 and st_o.converged
        assert abs(stats[k]["outer_its"] - st_o.outer_its) <= 2
        assert relerr(host(xs[k]), x_o) <= 1e-7


# --------------------------------------------------------------------------- failure paths


def test_nan_rhs_reports_breakdown():
    prob = dcg.dcg_assemble(2, 16, 1e-3)
    dcg.dcg_setup(prob, dcg.options())
    f = dev(inputs.rhs(0, prob.N))
    f[17] = float("nan")
    x = torch.zeros_like(f)
    st = dcg.dcg_solve(prob, f, x)
    assert st["status"] == dcg.DCG_ERR_BREAKDOWN
    assert "non-finite" in dcg.last_error()
    # the problem stays usable
    f[17] = 0.5
    st = dcg.dcg_solve(prob, f, x)
    assert st["status"] == dcg.DCG_OK and st["true_relres"] <= 1e-8


def test_bounded_wait_gives_up_and_context_survives():
    """The mbarrier wait of the bulk-copy kernels, on a barrier nothing
    completes, gives up after its poll limit; the kernel returns normally and
    the context stays usable."""
    assert dcg.dcg_selftest_bounded_wait(1000)
    assert dcg.dcg_selftest_bounded_wait(1 << 16)
    prob = dcg.dcg_assemble(2, 16, 1e-3)
    dcg.dcg_setup(prob, dcg.options())
    f = dev(inputs.rhs(0, prob.N))
    x = torch.zeros_like(f)
    st = dcg.dcg_solve(prob, f, x)
    assert st["status"] == dcg.DCG_OK


def test_fma_rate_diagnostic():
    """The measured FMA rates are positive, and FP32 is far above FP64 on this
    GPU (the reason the W-cycle runs in FP32 in the mixed mode)."""
    r64 = dcg.dcg_measure_fma_rate(dcg.DCG_FP64)
    r32 = dcg.dcg_measure_fma_rate(dcg.DCG_MIXED)
    assert r64 > 0.1 and r32 > 10 * r64


# --------------------------------------------------------------------------- GMRES outer solver


@pytest.mark.parametrize("d,n,dt,rule,m", [(2, 32, 1e-4, "fixed", None), (2, 32, 1e-2, "adaptive", None),
                                           (3, 8, 1e-4, "adaptive", None), (2, 24, 1e-3, "fixed", 5)])
def test_gmres_against_oracle(d, n, dt, rule, m):
    """GMRES on the deflated system (remarks in Sections 4.3 and 5.1): the
    device's classical Gram-Schmidt applied twice against the oracle's
    modified Gram-Schmidt, full and restarted."""
    o = mg.MGOptions()
    asm = fem.assemble(d, n, dt)
    f = inputs.rhs(4, asm.mesh.n_unknowns)
    prob = dcg.dcg_assemble(d, n, dt)
    rules = {"fixed": dcg.DCG_INNER_FIXED, "adaptive": dcg.DCG_INNER_ADAPTIVE}
    dcg.dcg_setup(prob, gpu_opts(o, recurrence=dcg.DCG_GMRES, inner_rule=rules[rule], c=0.05, fcg_max_dirs=m or 0))
    x = torch.zeros(prob.N, dtype=torch.float64, device="cuda")
    st = dcg.dcg_solve(prob, dev(f), x, tol=1e-8)
    x_o, st_o = solvers.FDCG(asm, solvers.FDCGOptions(mg=o, recurrence="gmres", inner_rule=rule, c=0.05,
                                                      m_max=m)).solve(f)
    assert st["status"] == dcg.DCG_OK and st["true_relres"] <= 1e-8 and st_o.converged
    assert abs(st["outer_its"] - st_o.outer_its) <= 2, (st["outer_its"], st_o.outer_its)
    assert relerr(host(x), x_o) <= 1e-7


def test_gmres_converges_where_fcg1_breaks_down():
    o = mg.MGOptions(patch=4, overlap=1, max_levels=2)
    asm = fem.assemble(2, 12, 0.1)
    f = inputs.rhs(5, asm.mesh.n_unknowns)
    prob = dcg.dcg_assemble(2, 12, 0.1)
    dcg.dcg_setup(prob, gpu_opts(o, recurrence=dcg.DCG_GMRES, inner_rule=dcg.DCG_INNER_ADAPTIVE, c=0.2,
                                 fcg_max_dirs=400))
    x = torch.zeros(prob.N, dtype=torch.float64, device="cuda")
    st = dcg.dcg_solve(prob, dev(f), x, tol=1e-8, max_it=400)
    assert st["status"] == dcg.DCG_OK and st["true_relres"] <= 1e-8 and st["outer_its"] < 400
