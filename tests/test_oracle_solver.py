"""Pins of the oracle's Krylov solver layer against dense linear algebra, brute force
and the majorisation property.

The projected machinery (QR of eq. (QR), DP/GCV of Sec. 4.1.3, the stacked
least-squares form of eq. (minKryov2)) is checked against explicitly formed
matrices; GKB against its defining relation; GKS and one MMGKS step against
dense normal-equation solves once the subspace is the whole space; the outer
loop against the Galerkin condition and the monotone decrease that the
quadratic tangent majorant (eq. (QuadraticMajorantQ)) guarantees.
"""
import numpy as np
import pytest

from oracle import ops, solver
from paper_2501_12497_gb300 import synth


def orth(n, k, seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, k)))
    return q


def test_gkb_relations():
    """H V_l = U_{l+1} B_l with orthonormal V_l and U_{l+1} (Sec. 4.1.1)."""
    rng = np.random.default_rng(0)
    A = rng.standard_normal((40, 25))
    b = rng.standard_normal(40)
    V, U, B = solver.gkb(lambda x: A @ x, lambda y: A.T @ y, b, 10)
    assert V.shape == (25, 10) and U.shape == (40, 11) and B.shape == (11, 10)
    np.testing.assert_allclose(A @ V, U @ B, atol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(10), atol=1e-13)
    np.testing.assert_allclose(U.T @ U, np.eye(11), atol=1e-13)
    np.testing.assert_allclose(U[:, 0], b / np.linalg.norm(b), atol=1e-15)
    assert np.all(np.diag(B) > 0) and np.all(np.diag(B, -1) > 0)


def test_gkb_breakdown_on_low_rank():
    """A rank-3 operator ends the bidiagonalisation after 3 steps."""
    rng = np.random.default_rng(1)
    A = rng.standard_normal((20, 3)) @ rng.standard_normal((3, 15))
    V, U, B = solver.gkb(lambda x: A @ x, lambda y: A.T @ y, rng.standard_normal(20), 10)
    assert V.shape[1] == 3


def _dense_problem(seed, m=30, n=16, p=20, k=7):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    L = rng.standard_normal((p, n))
    b = rng.standard_normal(m)
    V = orth(n, k, seed + 1)
    return A, L, b, V


def test_projected_problem_matches_dense_definitions():
    """z_lam, ||A V z - b||^2 and the GCV function equal their definitions written with
    explicit matrices: the projected normal equations of eq. (minKryov2) and
    G(lam) = ||R_A z - Q_A^T b||^2 / trace(I - R_A (R_A^T R_A + lam R_L^T R_L)^-1 R_A^T)^2."""
    A, L, b, V = _dense_problem(2)
    AV, LV = A @ V, L @ V
    pp = solver.ProjectedProblem(AV, LV, b)
    QA, RA = np.linalg.qr(AV)
    _, RL = np.linalg.qr(LV)
    c = QA.T @ b
    k = V.shape[1]
    for lam in (1e-3, 0.1, 1.0, 7.0, 100.0):
        G = AV.T @ AV + lam * LV.T @ LV
        z = np.linalg.solve(G, AV.T @ b)
        np.testing.assert_allclose(pp.solve(lam), z, rtol=1e-10, atol=1e-12)
        r2 = np.sum((AV @ z - b) ** 2)
        assert abs(pp.resid2(lam) - r2) <= 1e-10 * r2
        S = RA @ np.linalg.solve(RA.T @ RA + lam * RL.T @ RL, RA.T)
        gcv = np.sum((RA @ z - c) ** 2) / (k - np.trace(S)) ** 2
        assert abs(pp.gcv(lam) - gcv) <= 1e-8 * gcv


def test_dp_meets_discrepancy_equation():
    """The chosen lam satisfies ||A V z_lam - b|| = eta delta (Sec. 4.1.3) to 1e-10."""
    A, L, b, V = _dense_problem(3)
    AV, LV = A @ V, L @ V
    lam_true = 0.37
    z = np.linalg.solve(AV.T @ AV + lam_true * LV.T @ LV, AV.T @ b)
    target2 = np.sum((AV @ z - b) ** 2)
    pp = solver.ProjectedProblem(AV, LV, b)
    lam, flag = solver.choose_lambda_dp(pp, target2)
    assert flag == 0
    z2 = np.linalg.solve(AV.T @ AV + lam * LV.T @ LV, AV.T @ b)
    got = np.linalg.norm(AV @ z2 - b)
    assert abs(got - np.sqrt(target2)) <= 1e-10 * np.sqrt(target2)
    assert abs(lam / lam_true - 1) < 1e-8


def test_dp_no_root_flags():
    A, L, b, V = _dense_problem(4)
    pp = solver.ProjectedProblem(A @ V, L @ V, b)
    lam, flag = solver.choose_lambda_dp(pp, 0.0)
    assert flag == 1 and np.isclose(np.log10(lam), pp.log_lo)
    lam, flag = solver.choose_lambda_dp(pp, 10 * np.sum(b * b))
    assert flag == 2 and np.isclose(np.log10(lam), pp.log_hi)


def test_gcv_choice_matches_brute_force():
    """On a Solve-OF projected problem (a moving-disk pair), the GCV choice attains the minimum
    of the explicitly formed GCV function over a fine brute-force grid of the whole bracket."""
    w = synth.moving_disks(32, 2, 8, 32, radii=(5.0, 8.0), seed=3)
    ux, uy, ut = ops.of_fields(w.u_true, 1)
    ny, nx = ut.shape[1:]
    ns = nx * ny
    b = -ut[0].ravel()
    fx, fy = ux[0].ravel(), uy[0].ravel()
    A = lambda v: fx * v[:ns] + fy * v[ns:]
    AT = lambda r: np.concatenate([fx * r, fy * r])
    Lop = lambda v: ops.vgrad(v.reshape(1, 2, ny, nx)).ravel()
    V, _, _ = solver.gkb(A, AT, b, 10)
    AV = np.column_stack([A(V[:, j]) for j in range(V.shape[1])])
    LV = np.column_stack([Lop(V[:, j]) for j in range(V.shape[1])])
    pp = solver.ProjectedProblem(AV, LV, b)
    lam, _ = solver.choose_lambda_gcv(pp)
    QA, RA = np.linalg.qr(AV)
    _, RL = np.linalg.qr(LV)
    c = QA.T @ b
    k = V.shape[1]

    def G(l):
        M = RA.T @ RA + l * RL.T @ RL
        z = np.linalg.solve(M, RA.T @ c)
        S = RA @ np.linalg.solve(M, RA.T)
        return np.sum((RA @ z - c) ** 2) / (k - np.trace(S)) ** 2

    # the direct formula loses accuracy near the bracket ends (0/0 and cancellation); the
    # minimum is interior, so brute force over the middle 20 decades of the 24-decade bracket
    grid = 10.0 ** np.linspace(pp.log_lo + 2, pp.log_hi - 2, 8001)
    vals = np.array([G(l) for l in grid])
    best = grid[np.argmin(vals)]
    assert pp.log_lo + 2 < np.log10(lam) < pp.log_hi - 2
    assert G(lam) <= vals.min() * (1 + 1e-9)
    assert abs(np.log10(lam) - np.log10(best)) < 0.01


def test_gks_full_subspace_equals_dense_solution():
    """When the generalized Krylov subspace has grown to the whole space, the GKS iterate is
    the dense Tikhonov solution (A^T A + lam L^T L)^-1 A^T b at the lam it chose."""
    rng = np.random.default_rng(1)
    n = 12
    A = rng.standard_normal((18, n)) @ np.diag(np.logspace(0, -2, n))
    L = np.diff(np.eye(n), axis=0)
    b = A @ (0.3 * np.cumsum(rng.standard_normal(n))) + 0.05 * rng.standard_normal(18)
    x, info = solver.gks(lambda v: A @ v, lambda y: A.T @ y, lambda v: L @ v, lambda g: L.T @ g,
                         b, 3, 20)
    assert info["k"] == n
    lam = info["gamma"][-1]
    assert 1e-4 < lam < 1.0  # an interior GCV minimum
    xd = np.linalg.solve(A.T @ A + lam * L.T @ L, A.T @ b)
    np.testing.assert_allclose(x, xd, rtol=1e-9, atol=1e-11)


def test_solve_of_satisfies_galerkin_condition_of_its_tikhonov_problem():
    """The Solve-OF iterate (Alg. 2, p = q = 2) lies in its basis V and satisfies
    V^T ((Ups^T Ups + gamma (L+L)^T (L+L)) s - Ups^T (-u_t)) = 0 with dense Ups (the pointwise
    rows [u_x u_y] of Sec. 2.2) and dense L (+) L, at the gamma GCV chose (interior)."""
    w = synth.moving_disks(16, 2, 8, 16, radii=(3.0, 5.0), seed=4)
    ux, uy, ut = ops.of_fields(w.u_true, 1)
    ny, nx = ut.shape[1:]
    ns = nx * ny
    s, info = solver.solve_of_pair(ux[0], uy[0], ut[0], solver.Params(of_ell=6, of_iters=8))
    V = info["V"]
    g = info["gamma"][-1]
    Ups = np.hstack([np.diag(ux[0].ravel()), np.diag(uy[0].ravel())])
    LL = _dense_of(lambda e: ops.vgrad(e[None]), 2 * ns, (2, ny, nx))
    M = Ups.T @ Ups + g * LL.T @ LL
    rhs = Ups.T @ (-ut[0].ravel())
    sv = s.ravel()
    np.testing.assert_allclose(V @ (V.T @ sv), sv, atol=1e-12 * np.linalg.norm(sv))
    gal = V.T @ (M @ sv - rhs)
    assert np.linalg.norm(gal) <= 1e-10 * np.linalg.norm(V.T @ rhs)
    lo = np.log10(info["gamma"][-1])
    assert V.shape[1] == 6 + 7 and -12 < lo - np.log10(g) + 1 < 12


def test_solve_of_zero_time_derivative_gives_zero_velocity():
    u = synth.random_images(2, 8, 8, seed=3)
    u[1] = u[0]
    ux, uy, ut = ops.of_fields(u, 1)
    s, info = solver.solve_of_pair(ux[0], uy[0], ut[0], solver.Params())
    assert np.all(s == 0) and info["k"] == 0


# ------------------------------------------------ MM-GKS, p = q = 1 (App. A)
def _l1_problem(seed=5, m=30, n=18):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)) @ np.diag(np.logspace(0, -1.5, n))
    L = np.diff(np.eye(n), axis=0)
    x0 = np.cumsum(rng.standard_normal(n) * (rng.uniform(size=n) < 0.3))
    b = A @ x0 + 0.05 * rng.standard_normal(m) + 0.8 * (rng.uniform(size=m) < 0.1)
    return A, L, b


def _smoothed_l1(A, L, b, lam, eps, x):
    return np.sum(np.sqrt((A @ x - b) ** 2 + eps * eps)) + lam * np.sum(np.sqrt((L @ x) ** 2 + eps * eps))


def test_mm_gks_with_a_huge_eps_is_gks():
    """With eps far above every residual the IRLS weights are one constant for both terms,
    so the majorant is the p = q = 2 problem scaled and MM-GKS reproduces GKS (same GCV lam)."""
    rng = np.random.default_rng(1)
    n = 12
    A = rng.standard_normal((18, n)) @ np.diag(np.logspace(0, -2, n))
    L = np.diff(np.eye(n), axis=0)
    b = A @ (0.3 * np.cumsum(rng.standard_normal(n))) + 0.05 * rng.standard_normal(18)
    ops_ = (lambda v: A @ v, lambda y: A.T @ y, lambda v: L @ v, lambda g: L.T @ g)
    x2, i2 = solver.gks(*ops_, b, 3, 9)
    x1, i1 = solver.mm_gks(*ops_, b, 3, 9, eps=1e9)
    assert 1e-4 < i2["gamma"][-1] < 1.0  # interior GCV minimum at the end
    # (the first GCV functions are flat near their minima: lam to 1e-4)
    np.testing.assert_allclose(i1["gamma"], i2["gamma"], rtol=1e-4)
    assert i1["k"] == i2["k"]
    np.testing.assert_allclose(x1, x2, rtol=1e-6, atol=1e-8 * np.linalg.norm(x2))


def test_mm_gks_fixed_lambda_decreases_the_smoothed_l1_objective():
    """MM: each iterate minimises a quadratic majorant of the smoothed l1 objective over a
    subspace that holds the previous iterate, so the objective never increases."""
    A, L, b = _l1_problem()
    lam, eps = 0.7, 0.05
    vals = []
    for it in range(1, 25):
        x, _ = solver.mm_gks(lambda v: A @ v, lambda y: A.T @ y, lambda v: L @ v, lambda g: L.T @ g, b, 3, it,
                             eps=eps, lam_fixed=lam)
        vals.append(_smoothed_l1(A, L, b, lam, eps, x))
    assert all(vals[i + 1] <= vals[i] * (1 + 1e-12) for i in range(len(vals) - 1)), vals
    assert vals[-1] < 0.9 * vals[0]


def test_mm_gks_reaches_the_smoothed_l1_minimiser():
    """Once the subspace is the whole space the iteration is IRLS, whose limit is the
    minimiser of the smoothed l1 objective; scipy's BFGS on the same objective agrees."""
    from scipy.optimize import minimize
    A, L, b = _l1_problem()
    lam, eps = 0.7, 0.05
    x, info = solver.mm_gks(lambda v: A @ v, lambda y: A.T @ y, lambda v: L @ v, lambda g: L.T @ g, b, 3, 400,
                            eps=eps, lam_fixed=lam)
    assert info["k"] == A.shape[1]

    def grad(v):
        rf, rl = A @ v - b, L @ v
        return A.T @ (rf / np.sqrt(rf * rf + eps * eps)) + lam * L.T @ (rl / np.sqrt(rl * rl + eps * eps))

    ref = minimize(lambda v: _smoothed_l1(A, L, b, lam, eps, v), np.zeros(A.shape[1]), jac=grad, method="BFGS",
                   options={"gtol": 1e-12, "maxiter": 10000})
    assert np.linalg.norm(grad(x)) < 1e-7
    np.testing.assert_allclose(x, ref.x, atol=1e-6 * np.linalg.norm(ref.x))


def test_solve_of_pq1_runs_mm_gks_on_the_flow_problem():
    """Solve-OF with p = q = 1: the MM-GKS iterate of the pair problem; with a huge eps it
    equals the p = q = 2 Solve-OF."""
    w = synth.moving_disks(16, 2, 8, 16, radii=(3.0, 5.0), seed=4)
    ux, uy, ut = ops.of_fields(w.u_true, 1)
    s2, _ = solver.solve_of_pair(ux[0], uy[0], ut[0], solver.Params(of_ell=6, of_iters=8))
    s1, i1 = solver.solve_of_pair(ux[0], uy[0], ut[0], solver.Params(of_ell=6, of_iters=8, of_pq=1, eps=1e9))
    np.testing.assert_allclose(s1, s2, rtol=1e-5, atol=1e-7 * np.abs(s2).max())
    s1, i1 = solver.solve_of_pair(ux[0], uy[0], ut[0], solver.Params(of_ell=6, of_iters=8, of_pq=1))
    assert i1["k"] == 13 and np.linalg.norm(s1 - s2) > 1e-3 * np.linalg.norm(s2)


def _tiny_problem(seed=0, nx=4, ny=4, nt=2, na=6, nb=8):
    rng = np.random.default_rng(seed)
    na_arr, ang = synth.shifted_angles(nt, na)
    g = ops.Geometry(nx, ny, nt, nb, na_arr, ang)
    u_true = synth.random_images(nt, ny, nx, seed=seed, smooth=1)
    b = ops.project(g, u_true) + 0.01 * rng.standard_normal(g.m)
    return g, b


def _dense_of(fn, n_in, shape):
    cols = []
    for q in range(n_in):
        e = np.zeros(n_in)
        e[q] = 1.0
        cols.append(np.ravel(fn(e.reshape(shape))))
    return np.array(cols).T


def test_mmgks_step_full_subspace_equals_dense_normal_equations():
    """With V spanning R^n, one MMGKS step returns the solution of the normal equations
    (H^T H + lam Theta^T P^2 Theta) u = H^T b (eq. (normaleqQuadMajorant)), for the first
    step (weights from u^(0) = 0) and the second (weights from u^(1))."""
    g, b = _tiny_problem()
    n = g.n
    shape = (g.nt, g.ny, g.nx)
    s = synth.random_velocities(g.nt - 1, g.ny, g.nx, 1.5, seed=4)
    prm = solver.Params(ell=n, tau=0, image_rule=solver.RULE_FIXED, lam_fixed=0.05, eps=0.1)
    Hd = _dense_of(lambda x: ops.project(g, x), n, shape)
    assert np.linalg.matrix_rank(Hd) == n
    sr = ops.reverse_flow(s)
    th = solver.Theta(shape, s, sr)
    Th = _dense_of(th, n, shape)
    u = np.zeros(n)
    for n_outer in (1, 2):
        res = solver.mmgks_of(g, b, prm, n_outer, s_init=s)
        w = 1.0 / np.sqrt((Th @ u) ** 2 + prm.eps ** 2)
        u = np.linalg.solve(Hd.T @ Hd + prm.lam_fixed * Th.T @ (w[:, None] * Th), Hd.T @ b)
        np.testing.assert_allclose(res.u.ravel(), u, rtol=1e-8, atol=1e-10)


def test_mmgks_residual_is_orthogonal_to_basis():
    """The normal-equation residual r^(k+1) (eq. after (minKryov2)) of the projected solution
    is orthogonal to V_{l+k} (Galerkin condition); a wrong sign, weight or operator in r
    breaks it."""
    w = synth.moving_disks(24, 3, 6, 24, radii=(4.0, 6.0), seed=1)
    g = ops.Geometry(w.nx, w.ny, w.nt, w.nb, w.na, w.angles)
    prm = solver.Params(ell=6, of_iters=4, of_ell=4, noise_norm=w.noise_norm)
    seen = []

    def hook(k, V, r):
        seen.append(np.linalg.norm(V.T @ r) / np.linalg.norm(r))

    solver.mmgks_of(g, w.b, prm, 4, hook=hook)
    assert len(seen) == 3 and max(seen) < 1e-9


def test_mm_objective_is_monotone_with_fixed_lambda_and_flow():
    """With lam and s fixed, J(u) = ||Hu - b||^2 + 2 lam sum sqrt((Theta u)^2 + eps^2) is
    non-increasing along the MMGKS iterates (the majorant Q of eq. (QuadraticMajorantQ)
    touches J at u^(k) and the subspaces are nested)."""
    w = synth.moving_disks(24, 4, 6, 24, radii=(4.0, 6.0), seed=2)
    g = ops.Geometry(w.nx, w.ny, w.nt, w.nb, w.na, w.angles)
    s = synth.random_velocities(w.nt - 1, w.ny, w.nx, 1.0, seed=5)
    prm = solver.Params(ell=5, tau=0, image_rule=solver.RULE_FIXED, lam_fixed=0.3, eps=0.05)
    res = solver.mmgks_of(g, w.b, prm, 12, s_init=s, objective=True)
    J = np.array([r["J"] for r in res.report])
    assert np.all(np.diff(J) <= 1e-10 * J[:-1]), J
    assert J[-1] < J[0]


def test_theta_adjoint_identity():
    rng = np.random.default_rng(9)
    shape = (3, 6, 7)
    s = synth.random_velocities(2, 6, 7, 2.0, seed=1)
    th = solver.Theta(shape, s, ops.reverse_flow(s))
    x = rng.standard_normal(np.prod(shape))
    y = rng.standard_normal(th(x).size)
    assert abs(np.dot(th(x), y) - np.dot(x, th.T(y))) < 1e-11


# ------------------------------------------------------------ D1-OF (AnisoTV-OF, Table 2)
def test_time_differences_closed_forms():
    """L_t of Table 2 (forward differences between frames, no boundary row): zero on a
    sequence constant in time, the slope b on u_t = a + b t, and the transpose spreads
    r_t to frames t+1 (+) and t (-)."""
    rng = np.random.default_rng(3)
    a = rng.standard_normal((5, 7))
    const = np.broadcast_to(a, (4, 5, 7))
    assert np.all(solver.time_diff(const) == 0)
    ramp = a[None] + 0.75 * np.arange(4)[:, None, None]
    assert np.allclose(solver.time_diff(ramp), 0.75, rtol=0, atol=1e-14)
    r = np.zeros((3, 5, 7))
    r[1, 2, 3] = 1.0
    t = solver.time_diffT(r)
    assert t[2, 2, 3] == 1.0 and t[1, 2, 3] == -1.0 and np.count_nonzero(t) == 2


def test_theta_with_time_differences_adjoint_identity():
    rng = np.random.default_rng(10)
    shape = (4, 6, 7)
    s = synth.random_velocities(3, 6, 7, 2.0, seed=2)
    th = solver.Theta(shape, s, ops.reverse_flow(s), temporal=True)
    x = rng.standard_normal(np.prod(shape))
    y = rng.standard_normal(th(x).size)
    assert th(x).size == (2 * 4 + 3 + 2 * 3) * 6 * 7
    assert abs(np.dot(th(x), y) - np.dot(x, th.T(y))) < 1e-11


def test_d1_of_mm_step_full_subspace_equals_dense_normal_equations():
    """D1-OF: with V spanning R^n, one MMGKS step solves (H^T H + lam Theta^T P^2 Theta) u =
    H^T b with Theta = [Psi; L_t; Mhat], L_t assembled here from its definition."""
    g, b = _tiny_problem()
    n = g.n
    shape = (g.nt, g.ny, g.nx)
    s = synth.random_velocities(g.nt - 1, g.ny, g.nx, 1.5, seed=6)
    prm = solver.Params(ell=n, tau=0, image_rule=solver.RULE_FIXED, lam_fixed=0.05, eps=0.1, temporal_tv=1)
    Hd = _dense_of(lambda x: ops.project(g, x), n, shape)
    sr = ops.reverse_flow(s)
    Tm = _dense_of(solver.Theta(shape, s, sr), n, shape)  # [Psi; Mhat]
    npsi = 2 * n
    Lt = np.zeros(((g.nt - 1) * g.ny * g.nx, n))  # row (t, p): u[t+1, p] - u[t, p]
    ns = g.ny * g.nx
    for t in range(g.nt - 1):
        for q in range(ns):
            Lt[t * ns + q, (t + 1) * ns + q] = 1.0
            Lt[t * ns + q, t * ns + q] = -1.0
    Th = np.vstack([Tm[:npsi], Lt, Tm[npsi:]])
    u = np.zeros(n)
    for n_outer in (1, 2):
        res = solver.mmgks_of(g, b, prm, n_outer, s_init=s)
        w = 1.0 / np.sqrt((Th @ u) ** 2 + prm.eps ** 2)
        u = np.linalg.solve(Hd.T @ Hd + prm.lam_fixed * Th.T @ (w[:, None] * Th), Hd.T @ b)
        np.testing.assert_allclose(res.u.ravel(), u, rtol=1e-8, atol=1e-10)


def test_round_warp_mm_step_full_subspace_equals_dense_normal_equations():
    """Rounding-and-clipping M(s) inside MMGKS-OF: with V spanning R^n one step solves the dense
    normal equations whose Mhat rows pick, per pixel, the frame value at the clamped rounded
    displacement (assembled here pixel by pixel; halves away from zero)."""
    import math
    g, b = _tiny_problem(seed=3)
    n = g.n
    shape = (g.nt, g.ny, g.nx)
    s = synth.random_velocities(g.nt - 1, g.ny, g.nx, 1.5, seed=7)
    s[0, 0, 0, :] = 0.5  # exact halves in the first rows
    s[0, 1, 1, :] = -0.5
    prm = solver.Params(ell=n, tau=0, image_rule=solver.RULE_FIXED, lam_fixed=0.05, eps=0.1, warp_round=1)
    Hd = _dense_of(lambda x: ops.project(g, x), n, shape)
    sr = ops.reverse_flow(s)
    Psi = _dense_of(lambda x: ops.grad(x), n, shape)
    ns = g.ny * g.nx

    def pick(v):
        r = math.floor(abs(v) + 0.5)
        return int(r if v >= 0 else -r)

    rows = []
    for t in range(g.nt - 1):
        for fa, fb, vel in ((t, t + 1, s[t]), (t + 1, t, sr[t])):
            for y in range(g.ny):
                for x in range(g.nx):
                    X = min(max(x + pick(vel[0, y, x]), 0), g.nx - 1)
                    Y = min(max(y + pick(vel[1, y, x]), 0), g.ny - 1)
                    row = np.zeros(n)
                    row[fa * ns + y * g.nx + x] += 1.0
                    row[fb * ns + Y * g.nx + X] -= 1.0
                    rows.append(row)
    Th = np.vstack([Psi, np.array(rows)])
    u = np.zeros(n)
    for n_outer in (1, 2):
        res = solver.mmgks_of(g, b, prm, n_outer, s_init=s)
        w = 1.0 / np.sqrt((Th @ u) ** 2 + prm.eps ** 2)
        u = np.linalg.solve(Hd.T @ Hd + prm.lam_fixed * Th.T @ (w[:, None] * Th), Hd.T @ b)
        np.testing.assert_allclose(res.u.ravel(), u, rtol=1e-8, atol=1e-10)



def test_solve_of_pq1_is_sensitive_at_the_rounding_level():
    """The conditioning behind the p = q = 1 parity bound: the oracle's own Solve-OF with
    p = q = 1 (MM-GKS, App. A, default 10 + 20 iterations) on the 64x64x8 two-disk frames
    moves by more than 1e-6 when the frames are perturbed by 1e-15 relative (the IRLS
    weights reach 1/eps and each GCV minimum is resolved to about the square root of the
    FP64 rounding), while p = q = 2 moves by less than 1e-6. Two FP64 implementations that
    round differently therefore agree on p = q = 1 velocities only to about 1e-5."""
    from paper_2501_12497_gb300 import synth
    w = synth.plain_fp64(0)
    u = w.u_true
    up = u * (1 + 1e-15 * np.random.default_rng(5).standard_normal(u.shape))

    def rel(a, b):
        return np.linalg.norm(a - b) / np.linalg.norm(b)

    d1 = rel(solver.solve_of(up, solver.Params(of_pq=1)), solver.solve_of(u, solver.Params(of_pq=1)))
    d2 = rel(solver.solve_of(up, solver.Params()), solver.solve_of(u, solver.Params()))
    assert d1 > 1e-6 and d2 < 1e-6, (d1, d2)
