"""FP64 CPU oracle of the MMGKS-OF scheme (Alg. 1, Alg. 2, Alg. 3), in numpy.

TEST INFRASTRUCTURE ONLY: used by tests/, the package smoke check and the
bench's CPU-baseline leg; the product path never imports it.

It follows the paper's steps in order, using library primitives (QR, SVD,
least squares) as single steps:

* Golub-Kahan bidiagonalisation start, H V_l = U_{l+1} B_l (Sec. 4.1.1), with
  full reorthogonalisation of both bases.
* Thin QR of A V and of P Theta V (eq. (QR)), the projected least-squares
  problem (eq. (minKryov2)) solved as the stacked problem
  [R_A; sqrt(lam) R_L] z ~ [Q_A^T b; 0].
* lam by the discrepancy principle (Sec. 4.1.3, ||A x - b|| = eta delta) or by
  GCV (Sec. 4.1.3), both evaluated on the projected problem through the
  generalized singular values of (R_A, R_L).
* Residual of the normal equations (eq. after (minKryov2)), reorthogonalised
  against V twice, normalised and appended (eq. (enlargeMM-GKS)).
* Solve-OF (Alg. 2) with p = q = 2: the same machinery with constant weights,
  A = Upsilon(u(t)), b = -u_t, L = blockdiag(L, L), lam = gamma by GCV; with
  p = q = 1 (the stand-alone optical-flow choice the paper mentions in Sec.
  4.1.2) the MM-GKS of App. A with IRLS weights on both terms.
* MMGKS-OF (Alg. 1): Solve-OF on every pair, reverse flow by the remark of
  Sec. 3, Theta = [Psi; Mhat], IRLS weights w = (nu^2 + eps^2)^(-1/2)
  (P = w^(1/2)), one MMGKS step.

Readings of ambiguous passages: GCV denominator is
the squared trace of the projected (I - influence) matrix; DP/GCV search
bracket [1e-12, 1e12] * ||R_A||_F^2 / ||R_L||_F^2 in log10; DP by 100
bisection steps; GCV by a 200-point log grid refined by 60 golden-section
steps, ties to the smaller lam; breakdown rule: a new basis vector whose norm
is <= tol * ||A^T b|| (GKB: alpha_j <= tol*alpha_1, beta_j <= tol*beta_1)
ends the growth of the subspace.
"""
from dataclasses import dataclass, field

import numpy as np

from . import ops

RULE_DP = "dp"
RULE_GCV = "gcv"
RULE_FIXED = "fixed"

GRID_POINTS = 200
GOLDEN_STEPS = 60
BISECT_STEPS = 100
BRACKET_DECADES = 12.0
THETA_TINY = 1e-14


@dataclass
class Params:
    """Parameters of Alg. 1 and Alg. 2 (defaults: Sec. 5 where stated)."""
    ell: int = 10            # initial GKB subspace dimension (Sec. 5)
    tau: int = 1             # OF update period (Sec. 4.1.5); 0 = never update s
    of_scale: int = 1        # Solve-OF on frames downsampled by this factor (Sec. 4.1.5, Sec. 5)
    temporal_tv: int = 0     # 1: Theta also holds the temporal differences L_t (D1-OF, Table 2)
    warp_round: int = 0      # 1: M(s) by rounding and clipping (Sec. 3, item 1); 0: bilinear (item 2)
    of_iters: int = 20       # MMGKS iterations per Solve-OF call (Sec. 5)
    of_ell: int = 10         # GKB start of Solve-OF
    of_dr: int = 1           # box half-width of App. C
    eps: float = 1e-3        # smoothing of the l1 norm (Alg. 1 input)
    eta: float = 1.01        # DP safety factor (Sec. 4.1.3)
    noise_norm: float = -1.0  # delta = ||e||; < 0 means unknown -> GCV
    image_rule: str = RULE_DP
    lam_fixed: float = 0.0    # used when image_rule == "fixed"
    breakdown_tol: float = 1e-10
    of_pq: int = 2            # Solve-OF norms: 2 (p = q = 2, Sec. 5) or 1 (p = q = 1 by MM-GKS, App. A)


# ------------------------------------------------------------------ helpers

def reorth(w, Q):
    """Classical Gram-Schmidt against the columns of Q, applied twice."""
    if Q.shape[1] == 0:
        return w
    w = w - Q @ (Q.T @ w)
    w = w - Q @ (Q.T @ w)
    return w


def gkb(A, AT, b, ell, tol=1e-10):
    """Golub-Kahan bidiagonalisation from u_1 = b/||b|| (Sec. 4.1.1).

    Returns V (n x l'), U (m x (l'+1) or l'), B, with A V = U B up to rounding
    and l' <= ell (smaller only on breakdown).
    """
    beta1 = np.linalg.norm(b)
    n = AT(b).size
    if beta1 == 0.0:
        return np.zeros((n, 0)), np.zeros((b.size, 0)), np.zeros((0, 0))
    U = [b / beta1]
    V = []
    alphas, betas = [], [beta1]
    alpha1 = None
    for j in range(ell):
        w = AT(U[j])
        if j > 0:
            w = w - betas[j] * V[j - 1]
        w = reorth(w, np.array(V).T if V else np.zeros((n, 0)))
        alpha = np.linalg.norm(w)
        if alpha1 is None:
            alpha1 = alpha
        if alpha == 0.0 or alpha <= tol * alpha1:
            break
        V.append(w / alpha)
        alphas.append(alpha)
        p = A(V[j]) - alpha * U[j]
        p = reorth(p, np.array(U).T)
        beta = np.linalg.norm(p)
        if beta <= tol * beta1:
            break
        U.append(p / beta)
        betas.append(beta)
    k = len(V)
    Vm = np.array(V).T if k else np.zeros((n, 0))
    Um = np.array(U).T
    B = np.zeros((Um.shape[1], k))
    for j in range(k):
        B[j, j] = alphas[j]
        if j + 1 < Um.shape[1]:
            B[j + 1, j] = betas[j + 1]
    return Vm, Um, B


def _square(R, k):
    """The k x k upper-left block of an R factor, zero-padded when it has fewer rows."""
    out = np.zeros((k, k))
    r = min(k, R.shape[0])
    out[:r] = R[:r, :k]
    return out


class ProjectedProblem:
    """min_z ||A V z - b||^2 + lam ||L V z||^2 restricted to range(V).

    Built from the thin QR factorizations of eq. (QR); the lam-dependent
    quantities come from the generalized singular values of (R_A, R_L),
    obtained through the CS decomposition of the stacked [R_A; sqrt(rho) R_L].
    """

    def __init__(self, AV, LV, b):
        k = self.k = AV.shape[1]
        # R of [A V | b] = [[R_A, Q_A^T b], [0, ||b - Q_A Q_A^T b||]]: the thin QR of
        # eq. (QR) together with the projected right-hand side.
        Rab = _square(np.linalg.qr(np.column_stack([AV, b]), mode="r"), k + 1)
        RL = _square(np.linalg.qr(LV, mode="r"), k)
        RA = Rab[:k, :k]
        self.RA, self.RL = RA, RL
        self.c = Rab[:k, k].copy()
        out_of_range2 = float(Rab[k, k] ** 2)
        ta, tl = np.sum(RA * RA), np.sum(RL * RL)
        self.rho = ta / tl if (ta > 0 and tl > 0) else 1.0
        Q, _ = np.linalg.qr(np.vstack([RA, np.sqrt(self.rho) * RL]))
        Ua, cs, _ = np.linalg.svd(Q[:k])
        self.theta = np.clip(cs * cs, 0.0, 1.0)
        chat = Ua.T @ self.c
        drop = self.theta <= THETA_TINY
        # components of Q_A^T b along directions A V does not reach count as out of range
        self.rho0sq = out_of_range2 + float(np.sum(chat[drop] ** 2))
        chat[drop] = 0.0
        self.chat2 = chat * chat
        self.log_lo = np.log10(self.rho) - BRACKET_DECADES
        self.log_hi = np.log10(self.rho) + BRACKET_DECADES

    def one_minus_f(self, lam):
        """1 - f_i(lam) for scalar or 1-D lam (broadcast over a trailing axis of theta),
        with the filter factors f_i = theta_i / (theta_i + (lam/rho)(1 - theta_i))."""
        mu = np.asarray(lam, dtype=np.float64)[..., None] / self.rho
        th = self.theta
        den = th + mu * (1.0 - th)
        with np.errstate(invalid="ignore", divide="ignore"):
            out = np.where(den > 0, mu * (1.0 - th) / den, 1.0)
        return out

    def proj_resid2(self, lam):
        """||R_A z_lam - Q_A^T b||^2."""
        g = self.one_minus_f(lam)
        return np.sum(self.chat2 * g * g, axis=-1)

    def resid2(self, lam):
        """||A V z_lam - b||^2."""
        return self.proj_resid2(lam) + self.rho0sq

    def gcv(self, lam):
        """GCV function of Sec. 4.1.3 on the projected problem:
        ||R_A z - Q_A^T b||^2 / trace(I_k - R_A (R_A^T R_A + lam R_L^T R_L)^-1 R_A^T)^2."""
        g = self.one_minus_f(lam)
        den = np.sum(g, axis=-1)
        return np.sum(self.chat2 * g * g, axis=-1) / (den * den)

    def solve(self, lam):
        """z from the stacked least-squares form of eq. (minKryov2)."""
        M = np.vstack([self.RA, np.sqrt(lam) * self.RL])
        rhs = np.concatenate([self.c, np.zeros(self.k)])
        z, *_ = np.linalg.lstsq(M, rhs, rcond=None)
        return z


def choose_lambda_dp(pp: ProjectedProblem, target2):
    """Discrepancy principle ||A x_lam - b||^2 = (eta delta)^2 by bisection in log10 lam.

    Returns (lam, flag): flag 0 = root found, 1 = no root, residual above
    target even at the bracket's low end, 2 = residual below target at the
    high end."""
    a, b = pp.log_lo, pp.log_hi
    if pp.resid2(10.0 ** a) >= target2:
        return 10.0 ** a, 1
    if pp.resid2(10.0 ** b) <= target2:
        return 10.0 ** b, 2
    for _ in range(BISECT_STEPS):
        mid = 0.5 * (a + b)
        if pp.resid2(10.0 ** mid) > target2:
            b = mid
        else:
            a = mid
    return 10.0 ** (0.5 * (a + b)), 0


def choose_lambda_gcv(pp: ProjectedProblem):
    """Minimise the GCV function: log grid, then golden section around the grid minimum."""
    ts = np.linspace(pp.log_lo, pp.log_hi, GRID_POINTS)
    vals = pp.gcv(10.0 ** ts)
    i = int(np.argmin(vals))  # first minimal -> ties go to the smaller lam
    a = ts[max(i - 1, 0)]
    b = ts[min(i + 1, GRID_POINTS - 1)]
    gr = (np.sqrt(5.0) - 1.0) / 2.0
    for _ in range(GOLDEN_STEPS):
        c = b - gr * (b - a)
        d = a + gr * (b - a)
        if pp.gcv(10.0 ** c) <= pp.gcv(10.0 ** d):
            b = d
        else:
            a = c
    t = 0.5 * (a + b)
    if pp.gcv(10.0 ** t) > vals[i]:
        t = ts[i]
    return 10.0 ** t, 0


def expand(V, r, scale, tol):
    """Reorthogonalise r against V (twice), normalise and append; None on breakdown."""
    r = reorth(r, V)
    nr = np.linalg.norm(r)
    if nr == 0.0 or nr <= tol * scale:
        return None, nr
    return np.column_stack([V, r / nr]), nr


# ---------------------------------------------------------------- Solve-OF

def gks(A, AT, Lop, LTop, b, ell, iters, tol=1e-10):
    """Generalized Krylov subspace method for min ||A x - b||^2 + lam ||L x||^2 with lam
    chosen by GCV at every iteration (Alg. 3 with p = q = 2: constant weights).

    Returns (x, info): info has the final basis V, the lam sequence and the basis size.
    """
    V, _, _ = gkb(A, AT, b, ell, tol)
    info = {"gamma": [], "k": V.shape[1], "V": V}
    if V.shape[1] == 0:
        return np.zeros(AT(b).size), info
    scale = np.linalg.norm(AT(b))
    AV = np.column_stack([A(V[:, j]) for j in range(V.shape[1])])
    LV = np.column_stack([Lop(V[:, j]) for j in range(V.shape[1])])
    x = np.zeros(V.shape[0])
    grow = True
    for k in range(iters):
        pp = ProjectedProblem(AV, LV, b)
        lam, _ = choose_lambda_gcv(pp)
        z = pp.solve(lam)
        x = V @ z
        info["gamma"].append(lam)
        if k == iters - 1 or not grow:
            continue
        r = AT(AV @ z - b) + lam * LTop(LV @ z)
        Vn, _ = expand(V, r, scale, tol)
        if Vn is None:
            grow = False
            continue
        V = Vn
        AV = np.column_stack([AV, A(V[:, -1])])
        LV = np.column_stack([LV, Lop(V[:, -1])])
    info["k"], info["V"] = V.shape[1], V
    return x, info


def mm_gks(A, AT, Lop, LTop, b, ell, iters, eps, tol=1e-10, lam_fixed=None):
    """MM-GKS (App. A) for min ||A x - b||_1 + lam ||L x||_1, both norms smoothed to
    sum_i sqrt(t_i^2 + eps^2): at iteration k the weights w = ((.)^2 + eps^2)^(-1/2) of the
    fidelity residual A x^(k) - b and of L x^(k) (x^(0) = 0) define the quadratic majorant
    ||W_f^(1/2) (A x - b)||^2 + lam ||W_L^(1/2) L x||^2, minimised over range(V) with lam by
    GCV (or lam_fixed); the majorant's normal-equation residual at the new x,
    A^T W_f (A x - b) + lam L^T W_L L x, is orthogonalised, normalised and appended.
    The weights rescale that residual from one iteration to the next, so the growth of
    the subspace ends when the orthogonalised residual is at most tol times its norm
    before the orthogonalisation (the direction is already in range(V)).

    Returns (x, info) like gks."""
    V, _, _ = gkb(A, AT, b, ell, tol)
    info = {"gamma": [], "k": V.shape[1], "V": V}
    if V.shape[1] == 0:
        return np.zeros(AT(b).size), info
    AV = np.column_stack([A(V[:, j]) for j in range(V.shape[1])])
    LV = np.column_stack([Lop(V[:, j]) for j in range(V.shape[1])])
    x = np.zeros(V.shape[0])
    grow = True
    for k in range(iters):
        wf = 1.0 / np.sqrt((A(x) - b) ** 2 + eps * eps)
        wl = 1.0 / np.sqrt(Lop(x) ** 2 + eps * eps)
        sf, sl = np.sqrt(wf), np.sqrt(wl)
        pp = ProjectedProblem(sf[:, None] * AV, sl[:, None] * LV, sf * b)
        lam = lam_fixed if lam_fixed is not None else choose_lambda_gcv(pp)[0]
        z = pp.solve(lam)
        x = V @ z
        info["gamma"].append(lam)
        if k == iters - 1 or not grow:
            continue
        r = AT(wf * (AV @ z - b)) + lam * LTop(wl * (LV @ z))
        Vn, _ = expand(V, r, np.linalg.norm(r), tol)
        if Vn is None:
            grow = False
            continue
        V = Vn
        AV = np.column_stack([AV, A(V[:, -1])])
        LV = np.column_stack([LV, Lop(V[:, -1])])
    info["k"], info["V"] = V.shape[1], V
    return x, info


def solve_of_pair(ux, uy, ut, prm: Params):
    """Alg. 2 for one pair: min ||Upsilon s + u_t||_p^p + gamma ||(L (+) L) s||_q^q with
    p = q = 2 (GKS) or, when prm.of_pq == 1, p = q = 1 (MM-GKS).

    ux, uy, ut: (ny, nx) fields of App. C. Returns (s (2, ny, nx), info).
    """
    ny, nx = ut.shape
    ns = nx * ny
    b = -ut.ravel()
    if not np.any(b):
        return np.zeros((2, ny, nx)), {"gamma": [], "k": 0}
    fx, fy = ux.ravel(), uy.ravel()

    def A(s):
        return fx * s[:ns] + fy * s[ns:]

    def AT(r):
        return np.concatenate([fx * r, fy * r])

    def Lop(s):
        return ops.vgrad(s.reshape(1, 2, ny, nx)).ravel()

    def LTop(g):
        return ops.vgradT(g.reshape(1, 2, 2, ny, nx)).ravel()

    if prm.of_pq == 1:
        s, info = mm_gks(A, AT, Lop, LTop, b, prm.of_ell, prm.of_iters, prm.eps, prm.breakdown_tol)
    else:
        s, info = gks(A, AT, Lop, LTop, b, prm.of_ell, prm.of_iters, prm.breakdown_tol)
    return s.reshape(2, ny, nx), info


def _of_pair_job(args):
    ux, uy, ut, prm = args
    return solve_of_pair(ux, uy, ut, prm)[0]


def solve_of(u, prm: Params, pool=None):
    """Solve-OF on every consecutive pair of u (nt, ny, nx) -> s (nt-1, 2, ny, nx)."""
    ux, uy, ut = ops.of_fields(u, prm.of_dr)
    jobs = [(ux[p], uy[p], ut[p], prm) for p in range(ut.shape[0])]
    if pool is not None:
        res = pool.map(_of_pair_job, jobs)
    else:
        res = [_of_pair_job(j) for j in jobs]
    return np.stack(res) if res else np.zeros((0, 2) + u.shape[1:])


# ---------------------------------------------------------------- MMGKS-OF

def time_diff(x):
    """L_t of Table 2 (AnisoTV, eq. (L) along time): forward differences between
    consecutive frames, (nt, ny, nx) -> (nt-1, ny, nx), no boundary row."""
    return x[1:] - x[:-1]


def time_diffT(r):
    """The transpose of time_diff: (nt-1, ny, nx) -> (nt, ny, nx)."""
    out = np.zeros((r.shape[0] + 1,) + r.shape[1:])
    out[1:] += r
    out[:-1] -= r
    return out


class Theta:
    """Theta = [Psi; Mhat(s, s')] (Sec. 4.1.1) for fixed velocities; with temporal,
    Theta = [Psi; L_t; Mhat(s, s')], the AnisoTV-OF regulariser (D1-OF of Table 2:
    spatial and temporal first differences plus the motion term, all in the l1 norm)."""

    def __init__(self, shape, s, sr, temporal=False, warp_round=False):
        self.shape = shape  # (nt, ny, nx)
        self.s, self.sr = s, sr
        self.temporal = bool(temporal)
        self.flow = ops.flow_round if warp_round else ops.flow
        self.flowT = ops.flowT_round if warp_round else ops.flowT

    def __call__(self, x):
        x = x.reshape(self.shape)
        parts = [ops.grad(x).ravel()]
        if self.temporal:
            parts.append(time_diff(x).ravel())
        parts.append(self.flow(x, self.s, self.sr).ravel())
        return np.concatenate(parts)

    def T(self, y):
        nt, ny, nx = self.shape
        npsi, nlt = 2 * nt * ny * nx, ((nt - 1) * ny * nx if self.temporal else 0)
        g = y[:npsi].reshape(nt, 2, ny, nx)
        out = ops.gradT(g)
        if self.temporal:
            out = out + time_diffT(y[npsi:npsi + nlt].reshape(nt - 1, ny, nx))
        r = y[npsi + nlt:].reshape(2, nt - 1, ny, nx)
        return (out + self.flowT(r, self.s, self.sr)).ravel()


@dataclass
class Result:
    u: np.ndarray
    s: np.ndarray
    sr: np.ndarray
    report: list = field(default_factory=list)


def mmgks_of(geom: ops.Geometry, b, prm: Params, n_outer, u0=None, s_init=None, pool=None,
             objective=False, hook=None):
    """Alg. 1 (MMGKS-OF). Returns Result(u (nt,ny,nx), s, s', report).

    s_init: velocities to start from (default 0); with prm.tau == 0 they are
    kept fixed for the whole run (used by the majorisation test).
    objective: also record J(u^{k+1}) = ||Hu-b||^2 + 2 lam sum sqrt((Theta u)^2 + eps^2)
    with the lam of that iteration (the functional the quadratic Q majorises).
    hook: optional callable(k, V, r) given the normal-equation residual before it is
    reorthogonalised (for tests).
    """
    shape = (geom.nt, geom.ny, geom.nx)
    npairs = geom.nt - 1
    b = np.asarray(b, dtype=np.float64).ravel()

    def H(x):
        return ops.project(geom, x.reshape(shape))

    def HT(y):
        return ops.backproject(geom, y).ravel()

    V, _, _ = gkb(H, HT, b, prm.ell, prm.breakdown_tol)
    scale = np.linalg.norm(HT(b))
    HV = np.column_stack([H(V[:, j]) for j in range(V.shape[1])])
    u = np.zeros(geom.n) if u0 is None else np.asarray(u0, dtype=np.float64).ravel().copy()
    s = np.zeros((npairs, 2, geom.ny, geom.nx)) if s_init is None \
        else np.asarray(s_init, dtype=np.float64).copy()
    sr = ops.reverse_flow(s)
    out = Result(u=u, s=s, sr=sr)
    grow = True
    eps2 = prm.eps * prm.eps
    for k in range(n_outer):
        rec = {"k": k}
        if prm.tau > 0 and k % prm.tau == 0:
            if prm.of_scale > 1:  # on downsampled frames, velocities upscaled (Sec. 4.1.5)
                s = ops.upsample_velocity(solve_of(ops.downsample(u.reshape(shape), prm.of_scale), prm, pool),
                                          prm.of_scale)
            else:
                s = solve_of(u.reshape(shape), prm, pool)
            sr = ops.reverse_flow(s)
        th = Theta(shape, s, sr, prm.temporal_tv, prm.warp_round)
        nu = th(u)
        w = 1.0 / np.sqrt(nu * nu + eps2)
        P = np.sqrt(w)
        ThV = np.column_stack([P * th(V[:, j]) for j in range(V.shape[1])])
        pp = ProjectedProblem(HV, ThV, b)
        if prm.image_rule == RULE_DP:
            lam, flag = choose_lambda_dp(pp, (prm.eta * prm.noise_norm) ** 2)
        elif prm.image_rule == RULE_GCV:
            lam, flag = choose_lambda_gcv(pp)
        else:
            lam, flag = prm.lam_fixed, 0
        z = pp.solve(lam)
        u = V @ z
        HVz = HV @ z
        rec.update(lam=lam, flag=flag, basis=V.shape[1], resid=float(np.linalg.norm(HVz - b)))
        if objective:
            nu1 = th(u)
            rec["J"] = float(np.sum((HVz - b) ** 2) + 2.0 * lam * np.sum(np.sqrt(nu1 * nu1 + eps2)))
        if k < n_outer - 1 and grow:
            r = HT(HVz - b) + lam * th.T(w * th(u))
            if hook is not None:
                hook(k, V, r)
            Vn, nr = expand(V, r, scale, prm.breakdown_tol)
            rec["rnorm"] = float(nr)
            if Vn is None:
                grow = False
            else:
                V = Vn
                HV = np.column_stack([HV, H(V[:, -1])])
        out.report.append(rec)
    out.u = u.reshape(shape)
    out.s, out.sr = s, sr
    return out
