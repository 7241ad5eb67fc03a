"""Time stepping (Section 2.3) and reconstruction (Section 5.2) on the GPU
through the C ABI, against the oracle's TimeStepper: the right-hand side of
each scheme, the divergence form alone, pressure, element-centre divergence,
and whole runs of implicit Euler, Crank-Nicolson and BDF2 with a forcing,
including the velocity integral."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem, solvers, timestep
from paper_2606_13429_gb300 import dcg, inputs

pytestmark = pytest.mark.gpu

SCHEMES = {"ie": dcg.DCG_IMPLICIT_EULER, "cn": dcg.DCG_CRANK_NICOLSON, "bdf2": dcg.DCG_BDF2}


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


def maxrel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("d,n", [(2, 20), (3, 7)])
def test_apply_div_and_pressure_and_divergence(d, n):
    prob = dcg.dcg_assemble(d, n, 1e-2)
    mesh = fem.Mesh(d, n)
    K = fem.assemble(d, n, 1.0, mass=False).matrix()
    x = inputs.rhs(3, prob.N)
    y = torch.empty(prob.N, dtype=torch.float64, device="cuda")
    dcg.dcg_apply_div(prob, dev(x), y)
    assert maxrel(host(y), K @ x) <= 1e-12
    pres = torch.empty(prob.n_nodes, dtype=torch.float64, device="cuda")
    dcg.dcg_pressure(prob, dev(x), pres)
    assert np.array_equal(host(pres), timestep.pressure(mesh, x))
    dv = torch.empty(n ** d * d, dtype=torch.float64, device="cuda")
    dcg.dcg_divergence(prob, dev(x), dv)
    assert maxrel(host(dv).reshape(-1, d), timestep.divergence_at_centres(mesh, x)) <= 1e-13


@pytest.mark.parametrize("scheme", ["ie", "cn", "bdf2"])
@pytest.mark.parametrize("dt", [1e-1, 1e-4])
def test_time_rhs(scheme, dt):
    d, n = 2, 24
    ts = timestep.TimeStepper(d, n, dt, scheme)
    prob = dcg.dcg_assemble(d, n, dcg.dcg_scheme_alpha(SCHEMES[scheme], dt))
    s1, s2, F1, F0 = (inputs.rhs(k, prob.N) for k in (1, 2, 3, 4))
    out = torch.empty(prob.N, dtype=torch.float64, device="cuda")
    dcg.dcg_time_rhs(prob, SCHEMES[scheme], dev(s1), dev(F1), out, s2=dev(s2), F0=dev(F0))
    want = ts.rhs(s1, s2 if scheme == "bdf2" else None, F1, F0)
    # (M/alpha) w is formed as A w - K w: the cancellation leaves rounding of
    # the size of K w next to the size of the result
    assert maxrel(host(out), want) <= 1e-11


@pytest.mark.parametrize("scheme", ["ie", "cn", "bdf2"])
@pytest.mark.parametrize("d,n,dt", [(2, 24, 1e-3), (3, 8, 1e-2)])
def test_time_integrate_against_oracle(scheme, d, n, dt):
    """Four steps from a seeded stress with a time-dependent forcing F^n =
    cos(t_n) F_a + t_n F_b; stresses and the element-centre velocity against
    the oracle's run (both solve every step to 1e-10 from the previous step)."""
    nsteps = 4
    alpha = dcg.dcg_scheme_alpha(SCHEMES[scheme], dt)
    prob = dcg.dcg_assemble(d, n, alpha)
    dcg.dcg_setup(prob, dcg.options(stall_window=0))
    mesh = fem.Mesh(d, n)
    sigma0 = inputs.rhs(20, prob.N)
    Fa, Fb = inputs.rhs(21, prob.N), inputs.rhs(22, prob.N)
    loads = [np.cos(k * dt) * Fa + (k * dt) * Fb for k in range(nsteps + 1)]
    outs = [torch.empty(prob.N, dtype=torch.float64, device="cuda") for _ in range(nsteps)]
    u = torch.zeros(n ** d * d, dtype=torch.float64, device="cuda")
    code, stats = dcg.dcg_time_integrate(prob, SCHEMES[scheme], dt, dev(sigma0), [dev(F) for F in loads], outs,
                                         u_elem=u, tol=1e-10)
    assert code == dcg.DCG_OK and all(st["true_relres"] <= 1e-10 for st in stats)
    ts = timestep.TimeStepper(d, n, dt, scheme)
    sig_o, st_o = ts.run(sigma0, loads, tol=1e-12)
    # two solutions at relative residual 1e-10 differ by at most cond(A) x
    # 1e-10; a wrong load index or coefficient would differ at O(1)
    for k in range(nsteps):
        got = host(outs[k])
        assert np.linalg.norm(got - sig_o[k]) <= 1e-6 * np.linalg.norm(sig_o[k]), k
    u_o = timestep.velocity(mesh, sig_o, dt, scheme, sigma0=sigma0)
    assert maxrel(host(u).reshape(-1, d), u_o) <= 1e-6


def test_time_integrate_rejects_mismatched_alpha():
    prob = dcg.dcg_assemble(2, 16, 1e-3)
    dcg.dcg_setup(prob, dcg.options())
    x = torch.zeros(prob.N, dtype=torch.float64, device="cuda")
    with pytest.raises(dcg.DCGError) as err:
        dcg.dcg_time_integrate(prob, dcg.DCG_CRANK_NICOLSON, 1e-3, x, [x, x], [torch.zeros_like(x)])
    assert err.value.code == dcg.DCG_ERR_INVALID_ARG and "alpha" in str(err.value)
