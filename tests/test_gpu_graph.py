"""The solve captured into one CUDA graph (device_loop = 1: conditional
WHILE nodes for the restarts, the outer FCG iteration and every multigrid
call, driven by device-side tests) against the host-driven loop
(device_loop = 0) and against the oracle.

For a zero initial guess both loops launch the same kernels in the same
order, so their iterates agree bit for bit; a batch captured into one graph
agrees with solving its pairs one by one.
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


CASES = [
    # d, n, dt, options
    (2, 32, 1e-4, dict()),
    (2, 32, 1e-1, dict(inner_rule=dcg.DCG_INNER_ADAPTIVE, c=0.05)),
    (2, 48, 1e-6, dict(recurrence=dcg.DCG_FR)),
    (2, 32, 1e-4, dict(recurrence=dcg.DCG_FCG_INF, fcg_max_dirs=3, inner_rule=dcg.DCG_INNER_ADAPTIVE, c=0.05)),
    (2, 64, 1e-5, dict(precision=dcg.DCG_MIXED, ras_inverse=dcg.DCG_INV_BF16, patch=8, overlap=2, max_levels=2)),
    (2, 24, 0.1, dict(c=50.0, stall_window=50, max_levels=2)),
    (3, 8, 1e-4, dict()),
    (3, 12, 1e-2, dict(precision=dcg.DCG_MIXED)),
]


@pytest.mark.parametrize("d,n,dt,kw", CASES)
def test_graph_equals_host_loop_bitwise(d, n, dt, kw):
    prob = dcg.dcg_assemble(d, n, dt)
    f = dev(inputs.rhs(2, prob.N))
    out = {}
    for loop in (0, 1):
        dcg.dcg_setup(prob, dcg.options(device_loop=loop, **kw))
        x = torch.zeros_like(f)
        st = dcg.dcg_solve(prob, f, x, tol=1e-8, max_it=3000)
        out[loop] = (st, host(x))
    s0, x0 = out[0]
    s1, x1 = out[1]
    for key in ("status", "outer_its", "total_mg_cycles", "iter_mg_cycles", "restarts", "fcg_truncated"):
        assert s0[key] == s1[key], (key, s0[key], s1[key])
    assert s0["true_relres"] == s1["true_relres"]
    assert np.array_equal(x0, x1)
    assert s1["status"] == dcg.DCG_OK and s1["true_relres"] <= 1e-8
    prob.close()


def test_graph_solve_against_oracle_and_repeated_launches():
    """The captured graph is reused for repeated solves of the same arrays and
    re-captured when they change; every result matches the oracle."""
    d, n, dt = 2, 32, 1e-3
    asm = fem.assemble(d, n, dt)
    prob = dcg.dcg_assemble(d, n, dt)
    dcg.dcg_setup(prob, dcg.options(stall_window=0))
    for seed in (0, 1):
        f_np = inputs.rhs(seed, asm.mesh.n_unknowns)
        x_o, st_o = solvers.FDCG(asm, solvers.FDCGOptions()).solve(f_np)
        f = dev(f_np)
        for _ in range(2):
            x = torch.zeros_like(f)
            st = dcg.dcg_solve(prob, f, x)
            assert st["status"] == dcg.DCG_OK and abs(st["outer_its"] - st_o.outer_its) <= 2
            assert np.linalg.norm(host(x) - x_o) <= 1e-7 * np.linalg.norm(x_o)


def test_graph_edge_cases():
    prob = dcg.dcg_assemble(2, 16, 1e-3)
    dcg.dcg_setup(prob, dcg.options())
    N = prob.N
    x = torch.ones(N, dtype=torch.float64, device="cuda")
    st = dcg.dcg_solve(prob, torch.zeros(N, dtype=torch.float64, device="cuda"), x)
    assert st["status"] == dcg.DCG_OK and st["outer_its"] == 0 and not x.any().item()
    f = dev(inputs.rhs(0, N))
    x = torch.zeros_like(f)
    st = dcg.dcg_solve(prob, f, x, tol=1e-12, max_it=3)
    assert st["status"] == dcg.DCG_ERR_NOT_CONVERGED and st["outer_its"] == 3
    # warm start from the solution: the residual equation needs no iteration
    x = torch.zeros_like(f)
    dcg.dcg_solve(prob, f, x, tol=1e-10)
    st = dcg.dcg_solve(prob, f, x, tol=1e-10)
    assert st["outer_its"] == 0 and st["true_relres"] <= 1e-10
    # a nonzero initial guess converges to the same solution
    x_ref = host(x)
    x = dev(inputs.rhs(9, N))
    st = dcg.dcg_solve(prob, f, x, tol=1e-10)
    assert st["status"] == dcg.DCG_OK and np.linalg.norm(host(x) - x_ref) <= 1e-8 * np.linalg.norm(x_ref)


def test_graph_launch_counts_reported():
    """dcg_kernel_launches counts the kernels a captured solve ran (loop
    bodies times their iterations): the same count as the host-driven loop."""
    prob = dcg.dcg_assemble(2, 32, 1e-4)
    f = dev(inputs.rhs(3, prob.N))
    counts = {}
    for loop in (0, 1):
        dcg.dcg_setup(prob, dcg.options(device_loop=loop))
        x = torch.zeros_like(f)
        dcg.dcg_solve(prob, f, x)  # capture / warm-up
        x.zero_()
        k0 = dcg.dcg_kernel_launches()
        dcg.dcg_solve(prob, f, x)
        counts[loop] = dcg.dcg_kernel_launches() - k0
    # the graph adds its zero and copy kernels where the host loop uses
    # memset and memcpy calls, and its one-thread control kernels
    assert counts[1] >= counts[0] > 0
    assert counts[1] <= 2 * counts[0]


@pytest.mark.parametrize("loop", [0, 1])
def test_batched_graph_equals_sequential_and_oracle(loop):
    """A batch of 2D and 3D problems (several sizes, dt, precisions), 3
    right-hand sides each, driven by host workers (device_loop = 0) or
    captured into one graph (device_loop = 1): bitwise equal to solving the
    pairs one by one, and the FP64 pairs equal to the oracle's."""
    specs = [(2, 16, 1e-6, dcg.DCG_FP64), (2, 24, 1e-4, dcg.DCG_MIXED), (3, 8, 1e-4, dcg.DCG_FP64),
             (2, 40, 1e-2, dcg.DCG_FP64), (3, 12, 1e-5, dcg.DCG_MIXED)]
    nrhs = 3
    probs, fs = [], []
    for p, (d, n, dt, prec) in enumerate(specs):
        prob = dcg.dcg_assemble(d, n, dt)
        dcg.dcg_setup(prob, dcg.options(precision=prec, stall_window=0, device_loop=loop))
        probs.append(prob)
        for r in range(nrhs):
            fs.append(dev(inputs.rhs(7, prob.N, p=p, r=r)))
    seq, seq_st = [], []
    for k, f in enumerate(fs):
        x = torch.zeros_like(f)
        seq_st.append(dcg.dcg_solve(probs[k // nrhs], f, x))
        seq.append(host(x))
    xs = [torch.zeros_like(f) for f in fs]
    code, stats = dcg.dcg_solve_batched(probs, nrhs, fs, xs)
    assert code == dcg.DCG_OK
    for k in range(len(fs)):
        assert stats[k]["outer_its"] == seq_st[k]["outer_its"]
        assert stats[k]["total_mg_cycles"] == seq_st[k]["total_mg_cycles"]
        assert np.array_equal(host(xs[k]), seq[k])
    for p, (d, n, dt, prec) in enumerate(specs):
        if prec != dcg.DCG_FP64:
            continue
        asm = fem.assemble(d, n, dt)
        k = p * nrhs
        x_o, st_o = solvers.FDCG(asm, solvers.FDCGOptions()).solve(host(fs[k]))
        assert abs(stats[k]["outer_its"] - st_o.outer_its) <= 2
        assert np.linalg.norm(host(xs[k]) - x_o) <= 1e-7 * np.linalg.norm(x_o)
