"""Pins of the oracle's solvers (no GPU): dense direct solves, the deflated
residual's orthogonality, textbook CG equivalences and the dt trends of the
paper's Tables 1-3 (on Q1, so as trends only)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import fem, mg, solvers
from paper_2606_13429_gb300 import inputs


def _f(asm, seed=0):
    return inputs.rhs(seed, asm.mesh.n_unknowns)


@pytest.mark.parametrize("d,n", [(2, 2), (2, 3), (2, 4), (2, 6), (3, 2), (3, 4)])
def test_dense_cg_dcg_agree(d, n):
    """P6: dense Cholesky == CG == DCG(exact inner) == DCG(MG inner) to 1e-10."""
    for dt in [1e-1, 1e-4]:
        asm = fem.assemble(d, n, dt)
        f = _f(asm)
        x_ref = solvers.dense_solve(asm, f)
        sc = np.linalg.norm(x_ref)
        x_cg, st = solvers.plain_cg(asm.matrix(), f, tol=1e-13)
        assert np.linalg.norm(x_cg - x_ref) <= 1e-10 * sc
        for rule in ["exact", "fixed", "adaptive"]:
            o = solvers.FDCGOptions(inner_rule=rule, c=0.01)
            x, st = solvers.FDCG(asm, o).solve(f, tol=1e-13)
            assert st.converged
            assert np.linalg.norm(x - x_ref) <= 1e-10 * sc, (rule, dt)


def test_deflated_residual_orthogonal_to_S():
    """P7: V^T r_i = 0 for r_i in the range of (I - pi_A)^T (from Eq.
    defl_sys); exact inner to rounding, MG inner to ~ inner tolerance."""
    asm = fem.assemble(2, 16, 1e-4)
    f = _f(asm)
    for rule, bound in [("exact", 1e-11), ("fixed", 1e-6)]:
        S = solvers.FDCG(asm, solvers.FDCGOptions(inner_rule=rule))
        A, V = S.A, S.V
        st = solvers.SolveStats()
        # replay the first iterations, checking V^T r after each update
        f_D = f - A @ S.pi(f, 1e-10, st)
        r = f_D.copy()
        d = r.copy()
        assert np.linalg.norm(V.T @ r) <= bound * np.linalg.norm(r)
        for _ in range(6):
            q = S.M_D(d, 1e-10, st)
            dq = d @ q
            alpha = (d @ r) / dq
            r = r - alpha * q
            assert np.linalg.norm(V.T @ r) <= bound * np.linalg.norm(f), rule
            d = r - ((r @ q) / dq) * d


def test_fcg_inf_exact_equals_cg_iterates():
    """P13: with exact inner solves the deflated operator is fixed and
    symmetric, so FCG(inf), FCG(1) and classical CG produce the same iterates."""
    asm = fem.assemble(2, 12, 1e-3)
    f = _f(asm)
    hist = {}
    for rec in ["fr", "fcg1", "fcg_inf"]:
        o = solvers.FDCGOptions(inner_rule="exact", recurrence=rec)
        x, st = solvers.FDCG(asm, o).solve(f, tol=1e-10)
        hist[rec] = (np.array(st.history[:12]), st.outer_its, x)
    h0 = hist["fr"][0]
    for rec in ["fcg1", "fcg_inf"]:
        assert np.allclose(hist[rec][0], h0, rtol=1e-8)
        assert abs(hist[rec][1] - hist["fr"][1]) <= 1
        assert np.linalg.norm(hist[rec][2] - hist["fr"][2]) <= 1e-10 * np.linalg.norm(hist["fr"][2])


def test_condition_number_trend():
    """P10 (Table 1 trend): kappa(A) grows like 1/dt for dt << h^2 and like
    dt/h^2 for dt >> h^2 (U-shape); kappa_eff of the deflated operator stays
    bounded as dt -> 0."""
    n = 8
    kap, keff = {}, {}
    for dt in [1e0, 1e-2, 1e-4, 1e-6, 1e-8]:
        asm = fem.assemble(2, n, dt)
        A = asm.matrix().toarray()
        ev = np.linalg.eigvalsh(A)
        kap[dt] = ev[-1] / ev[0]
        V = fem.V_matrix(asm.mesh).toarray()
        Z = V.T @ A @ V
        PiA = V @ np.linalg.solve(Z, V.T @ A)
        AD = A @ (np.eye(A.shape[0]) - PiA)
        AD = 0.5 * (AD + AD.T)
        evd = np.linalg.eigvalsh(AD)
        nz = evd[evd > 1e-9 * evd[-1]]
        keff[dt] = nz[-1] / nz[0]
    # small dt: kappa ~ 1/dt (x100 per two decades)
    assert 50 < kap[1e-8] / kap[1e-6] < 200 and 50 < kap[1e-6] / kap[1e-4] < 200
    # large dt: kappa grows again with dt (div-free modes of K_div, A ~ M/dt)
    assert kap[1e0] > 3 * kap[1e-2]
    # minimum near dt ~ h^2 = 1/64
    assert min(kap, key=kap.get) == 1e-2
    # kappa_eff bounded as dt -> 0
    assert keff[1e-8] < 1.5 * keff[1e-6] and keff[1e-8] < 1e-5 * kap[1e-8]


def test_iteration_trends():
    """P11 (Table 2 trend): for dt << h^2 plain-CG counts grow as dt shrinks,
    deflated-CG counts do not; P12 (Tables 2-3): DCG with the MG inner at
    c_F = 0.01 needs the same outer count as with an exact inner solve (+-2)."""
    asm_cache = {}
    cg_its, dcg_its = {}, {}
    for dt in [1e-4, 1e-6, 1e-8]:
        asm = fem.assemble(2, 32, dt)
        asm_cache[dt] = asm
        f = _f(asm)
        _, st = solvers.plain_cg(asm.matrix(), f)
        cg_its[dt] = st.outer_its
        _, st_e = solvers.FDCG(asm, solvers.FDCGOptions(inner_rule="exact")).solve(f)
        _, st_m = solvers.FDCG(asm, solvers.FDCGOptions(inner_rule="fixed", c=0.01)).solve(f)
        dcg_its[dt] = st_e.outer_its
        assert abs(st_m.outer_its - st_e.outer_its) <= 2, dt
        assert st_m.true_relres <= 1e-8 and st_e.true_relres <= 1e-8
    # h^2 ~ 1e-3 here: plain CG grows steadily below it, DCG stays flat
    assert cg_its[1e-8] > cg_its[1e-6] > cg_its[1e-4]
    assert cg_its[1e-8] > 5 * cg_its[1e-4]
    assert dcg_its[1e-8] <= dcg_its[1e-6] + 2
    assert dcg_its[1e-8] < cg_its[1e-8] / 10


@pytest.mark.parametrize("rule", ["fixed", "adaptive"])
def test_true_residual_and_restart(rule):
    """P14: true relative residual <= tol; with a very loose inner tolerance
    the restart on the residual equation still delivers it."""
    asm = fem.assemble(2, 16, 1e-5)
    f = _f(asm, seed=3)
    x_ref = solvers.dense_solve(asm, f)
    for c in [0.01, 1.0]:
        o = solvers.FDCGOptions(inner_rule=rule, c=c, max_restarts=5)
        x, st = solvers.FDCG(asm, o).solve(f, tol=1e-8)
        assert st.converged and st.true_relres <= 1e-8, (c, st.true_relres)
        A = asm.matrix()
        assert np.linalg.norm(f - A @ x) <= 1e-8 * np.linalg.norm(f)
        assert np.linalg.norm(x - x_ref) <= 1e-4 * np.linalg.norm(x_ref)


def test_initial_guess_and_zero_rhs():
    asm = fem.assemble(2, 8, 1e-3)
    f = _f(asm)
    S = solvers.FDCG(asm)
    x, st = S.solve(f, tol=1e-10)
    x2, st2 = S.solve(f, tol=1e-10, x0=x)
    assert st2.outer_its <= 1
    z, st3 = S.solve(np.zeros_like(f))
    assert not z.any() and st3.converged and st3.outer_its == 0


def test_max_it_cap_reports_not_converged():
    asm = fem.assemble(2, 16, 1e-2)
    f = _f(asm)
    x, st = solvers.FDCG(asm).solve(f, tol=1e-12, max_it=3)
    assert st.outer_its == 3 and not st.converged
    x, st = solvers.plain_cg(asm.matrix(), f, tol=1e-12, max_it=3)
    assert st.outer_its == 3 and not st.converged


def test_stall_restart_recovers_from_stagnation():
    """A very loose inner tolerance (c_F = 50) perturbs the deflated operator
    enough that the FCG(1) recursion stops reducing its residual at large dt;
    without the stall restart the solve stagnates far above 1e-8, with it the
    restarted passes reach the tolerance."""
    asm = fem.assemble(2, 24, 0.1)
    f = inputs.rhs(5, asm.mesh.n_unknowns)
    o = mg.MGOptions(patch=4, overlap=1, max_levels=2)
    _, st0 = solvers.FDCG(asm, solvers.FDCGOptions(mg=o, c=50.0, stall_window=0)).solve(f, max_it=1500)
    assert not st0.converged and st0.true_relres > 1e-6 and st0.outer_its == 1500
    x, st = solvers.FDCG(asm, solvers.FDCGOptions(mg=o, c=50.0, stall_window=50)).solve(f, max_it=1500)
    assert st.converged and st.true_relres <= 1e-8 and st.restarts >= 1 and st.outer_its < 500
    assert np.linalg.norm(f - asm.matrix() @ x) <= 1e-8 * np.linalg.norm(f)


def test_adaptive_inner_tolerance_follows_eq_tol():
    """Eq. tol: at outer iteration i the multigrid inside M_D gets
    tau_c = c_A * tol * ||f|| / ||r_i||, r_i the current recursive deflated
    residual (r_0 = f_D for the first iteration). The norms come from the
    residual history the outer loop records; a slip such as c * tol,
    c * eps * ||r_i|| or the previous residual fails here."""
    asm = fem.assemble(2, 16, 1e-5)
    f = _f(asm, seed=2)
    tol, c = 1e-8, 0.02
    x, st = solvers.FDCG(asm, solvers.FDCGOptions(inner_rule="adaptive", c=c)).solve(f, tol=tol)
    assert st.converged and st.restarts == 0
    r = [st.res0[0]] + list(st.history)
    assert len(st.inner_tols) == st.outer_its
    fn = np.linalg.norm(f)
    for i, tc in enumerate(st.inner_tols):
        assert np.isclose(tc, c * tol * fn / r[i], rtol=1e-12, atol=0.0), i
    # the tolerance loosens as the outer residual falls, and is at most c_A
    # when the outer iteration stops (||r|| ~ tol ||f||)
    assert st.inner_tols[-1] > 100 * st.inner_tols[0]
    assert st.inner_tols[-1] <= 10 * c


def test_fixed_inner_tolerance_is_c_times_tol():
    """Eq. fixed_tol with the experiments' reading: tau_c = c_F * tol at every
    outer iteration."""
    asm = fem.assemble(2, 16, 1e-5)
    f = _f(asm, seed=2)
    x, st = solvers.FDCG(asm, solvers.FDCGOptions(inner_rule="fixed", c=0.01)).solve(f, tol=1e-8)
    assert st.inner_tols and all(t == 0.01 * 1e-8 for t in st.inner_tols)


def test_adaptive_tolerance_cuts_total_cycles():
    """Table 3 trend: the adaptive rule needs far fewer W-cycles in total
    (Tot) than the fixed rule with the same constant, at the same outer count."""
    for dt in [1e-4, 1e-6]:
        asm = fem.assemble(2, 32, dt)
        f = _f(asm)
        _, st_f = solvers.FDCG(asm, solvers.FDCGOptions(inner_rule="fixed", c=0.01)).solve(f)
        _, st_a = solvers.FDCG(asm, solvers.FDCGOptions(inner_rule="adaptive", c=0.01)).solve(f)
        assert st_f.converged and st_a.converged
        assert abs(st_f.outer_its - st_a.outer_its) <= 2
        assert st_a.total_mg_cycles < 0.8 * st_f.total_mg_cycles, (dt, st_a.total_mg_cycles, st_f.total_mg_cycles)
        assert st_a.avg_inner < st_f.avg_inner - 1.0


def test_truncated_fcg_special_cases():
    """Remark after Table 4: m_i = max{1, mod(i, m_max + 1)}. m_max = 0 is
    FCG(1) and an m_max beyond the iteration count is the untruncated
    FCG(inf), both bit for bit; with exact inner solves every truncation gives
    the iterates of classical CG (the directions are conjugate already)."""
    asm = fem.assemble(2, 16, 1e-4)
    f = _f(asm, seed=1)
    o = mg.MGOptions(patch=4, overlap=1, max_levels=2)

    def run(rec, m_max=None, rule="adaptive"):
        return solvers.FDCG(asm, solvers.FDCGOptions(mg=o, inner_rule=rule, c=0.05, recurrence=rec,
                                                     m_max=m_max)).solve(f)

    x1, s1 = run("fcg1")
    x0, s0 = run("fcg_inf", 0)
    assert s0.history == s1.history and np.array_equal(x0, x1)
    xi, si = run("fcg_inf")
    xb, sb = run("fcg_inf", 10 * si.outer_its)
    assert sb.history == si.history and np.array_equal(xb, xi)
    # a truncation that actually restarts differs from both ends
    x3, s3 = run("fcg_inf", 3)
    assert s3.converged and s3.history != s1.history and s3.history != si.history
    he = {}
    for m_max in [None, 2, 5]:
        _, st = solvers.FDCG(asm, solvers.FDCGOptions(inner_rule="exact", recurrence="fcg_inf",
                                                      m_max=m_max)).solve(f, tol=1e-10)
        he[m_max] = np.array(st.history[:15])
    _, st_fr = solvers.FDCG(asm, solvers.FDCGOptions(inner_rule="exact", recurrence="fr")).solve(f, tol=1e-10)
    for m_max, h in he.items():
        assert np.allclose(h, np.array(st_fr.history[:15]), rtol=1e-7), m_max


def test_fcg1_breaks_down_where_fcg_inf_does_not():
    """Tables 3-4 trend on Q1: with a loose adaptive inner tolerance the
    inexact deflated operator stops being positive on the FCG(1) direction
    ((d, M_D d) <= 0: the paper's failed runs), while FCG(inf), which keeps
    every direction, goes on reducing the residual."""
    asm = fem.assemble(2, 12, 0.1)
    f = inputs.rhs(5, asm.mesh.n_unknowns)
    o = mg.MGOptions(patch=4, overlap=1, max_levels=2)
    opts = dict(mg=o, inner_rule="adaptive", c=0.2, max_restarts=0)
    _, s1 = solvers.FDCG(asm, solvers.FDCGOptions(recurrence="fcg1", **opts)).solve(f, max_it=400)
    _, si = solvers.FDCG(asm, solvers.FDCGOptions(recurrence="fcg_inf", **opts)).solve(f, max_it=400)
    assert s1.breakdown and not s1.converged and s1.outer_its < 400
    assert not si.breakdown and si.outer_its == 400
    assert si.true_relres < 0.1 * s1.true_relres


def test_gmres_minimal_residual_with_exact_inner():
    """With exact inner solves the deflated operator is fixed and SPD: GMRES
    minimises the residual 2-norm over the Krylov space, so its residual at
    every step is at most CG's (FCG(inf) = CG here), and it converges."""
    asm = fem.assemble(2, 16, 1e-4)
    f = _f(asm, seed=1)
    _, sg = solvers.FDCG(asm, solvers.FDCGOptions(recurrence="gmres", inner_rule="exact")).solve(f, tol=1e-10)
    _, sc = solvers.FDCG(asm, solvers.FDCGOptions(recurrence="fcg_inf", inner_rule="exact")).solve(f, tol=1e-10)
    assert sg.converged and sg.true_relres <= 1e-10
    k = min(len(sg.history), len(sc.history))
    assert np.all(np.array(sg.history[:k]) <= np.array(sc.history[:k]) * (1 + 1e-10))
    assert sg.outer_its <= sc.outer_its


def test_gmres_restart_special_cases():
    """GMRES(m) with m beyond the iteration count is full GMRES bit for bit; a
    short restart still converges (the restarts begin from f_D - M_D x_hat)."""
    asm = fem.assemble(2, 16, 1e-5)
    f = _f(asm, seed=2)
    xf, sf = solvers.FDCG(asm, solvers.FDCGOptions(recurrence="gmres")).solve(f)
    xb, sb = solvers.FDCG(asm, solvers.FDCGOptions(recurrence="gmres", m_max=10 * sf.outer_its)).solve(f)
    assert sb.history == sf.history and np.array_equal(xb, xf)
    x4, s4 = solvers.FDCG(asm, solvers.FDCGOptions(recurrence="gmres", m_max=4)).solve(f)
    assert s4.converged and s4.outer_its > sf.outer_its
    assert np.linalg.norm(x4 - xf) <= 1e-6 * np.linalg.norm(xf)


def test_gmres_converges_where_fcg1_breaks_down():
    """Remark after Table 4: GMRES with the adaptive inner tolerance
    converges where FCG(1) breaks down (the case of
    test_fcg1_breaks_down_where_fcg_inf_does_not)."""
    asm = fem.assemble(2, 12, 0.1)
    f = inputs.rhs(5, asm.mesh.n_unknowns)
    o = mg.MGOptions(patch=4, overlap=1, max_levels=2)
    x, st = solvers.FDCG(asm, solvers.FDCGOptions(mg=o, recurrence="gmres", inner_rule="adaptive", c=0.2,
                                                  max_restarts=3)).solve(f, max_it=400)
    assert st.converged and not st.breakdown and st.outer_its < 400
    assert np.linalg.norm(f - asm.matrix() @ x) <= 1e-8 * np.linalg.norm(f)
