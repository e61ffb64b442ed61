// K11: the small projected problem of MMGKS / GKS, in FP64, one block per
// problem (Sec. 4.1.1 eq. (QR)-(minKryov2), Sec. 4.1.3 DP and GCV).
//
// Given the Gram matrices G_A = (A V)^T (A V), G_L = (L V)^T (L V) and
// g = (A V)^T b of the current basis (R_A^T R_A = G_A and R_L^T R_L = G_L for
// the R factors of eq. (QR)), the block
//   1. factors M = G_A + rho G_L = R^T R (Cholesky), rho = tr G_A / tr G_L;
//   2. diagonalises C = R^-T G_A R^-1 = W diag(theta) W^T (parallel cyclic
//      Jacobi), so that with X = R^-1 W:  X^T G_A X = diag(theta),
//      X^T G_L X = diag(1 - theta)/rho  (the generalized singular values of
//      (R_A, R_L));
//   3. evaluates, for any lam, the filter factors f_i = theta_i/(theta_i +
//      (lam/rho)(1 - theta_i)), the projected residual
//      ||R_A z - Q_A^T b||^2 = sum_i chat_i^2 (1 - f_i)^2 with
//      chat_i^2 = (X^T g)_i^2 / theta_i, and trace(I - S) = sum_i (1 - f_i);
//   4. picks lam: DP solves ||A V z - b||^2 = (eta delta)^2 on the bracket
//      [1e-12, 1e12] rho by 256-way multisection in log10 lam; GCV minimises
//      G = sum chat^2 (1-f)^2 / (sum (1-f))^2 on a 200-point log grid and
//      refines around the grid minimum by repeated 256-point grids;
//   5. returns z = X diag(1/(theta + (lam/rho)(1 - theta))) X^T g.
#include "solver.cuh"

#include <cfloat>

namespace mof {

namespace {

constexpr int ST = 256;
constexpr int GRID_POINTS = 200;
constexpr double BRACKET_DECADES = 12.0;
constexpr double THETA_TINY = 1e-14;
constexpr int JACOBI_MAX_SWEEPS = 40;
constexpr int REFINE_ROUNDS = 7;
constexpr int DP_ROUNDS = 8;

struct Spec {
    int K;
    double rho, bb, rho0sq;
    const double *theta, *c2;
};

// sum_i chat_i^2 (1 - f_i)^2 and sum_i (1 - f_i) at lam = 10^t
__device__ __forceinline__ void filters(const Spec &S, double t, double &num, double &den) {
    const double mu = exp10(t) / S.rho;
    num = 0.0;
    den = 0.0;
    for (int i = 0; i < S.K; ++i) {
        const double th = S.theta[i];
        const double d = th + mu * (1.0 - th);
        const double omf = d > 0.0 ? mu * (1.0 - th) / d : 1.0;
        num += S.c2[i] * omf * omf;
        den += omf;
    }
}

__device__ __forceinline__ double gcv_at(const Spec &S, double t) {
    double num, den;
    filters(S, t, num, den);
    const double g = num / (den * den);
    return g == g ? g : DBL_MAX;
}

__device__ __forceinline__ double dp_at(const Spec &S, double t, double target2) {
    double num, den;
    filters(S, t, num, den);
    return num + S.rho0sq - target2;
}

// block argmin of (v, i): smallest v, ties to the smallest i
__device__ void block_argmin(double v, int i, double *sv, int *si, double &vbest, int &ibest) {
    const int tid = threadIdx.x;
    sv[tid] = v;
    si[tid] = i;
    __syncthreads();
    for (int s = ST / 2; s > 0; s >>= 1) {
        if (tid < s) {
            const double vo = sv[tid + s];
            const int io = si[tid + s];
            if (vo < sv[tid] || (vo == sv[tid] && io < si[tid])) {
                sv[tid] = vo;
                si[tid] = io;
            }
        }
        __syncthreads();
    }
    vbest = sv[0];
    ibest = si[0];
    __syncthreads();
}

}  // namespace

__global__ void __launch_bounds__(ST) k_small_solve(SmallArgs a) {
    extern __shared__ double sm[];
    __shared__ double s_rho, s_piv, s_rho0sq, s_lo, s_hi, s_t, s_va;
    __shared__ int s_fail, s_flag, s_conv;
    __shared__ double sv[ST];
    __shared__ int si[ST];
    const int b = blockIdx.x, tid = threadIdx.x;
    const int ld = a.ld;
    const int K = min(a.K[b], ld);
    double *z = a.z + (long long)b * ld;
    for (int i = tid; i < ld; i += ST) z[i] = 0.0;
    if (K <= 0 || (a.active && !a.active[b])) {
        if (tid == 0) {
            a.lam[b] = 0.0;
            a.flag[b] = 0;
        }
        return;
    }
    const int Kp = K + (K & 1);  // padded to even for the round-robin Jacobi
    const int lds = ld + 2;       // shared-memory leading dimension (>= Kp)
    double *M = sm;               // Kp x Kp, later C
    double *Ri = M + lds * lds;   // R^-1
    double *T = Ri + lds * lds;   // G_A R^-1, later X
    double *W = T + lds * lds;    // eigenvectors
    double *theta = W + lds * lds;
    double *gh = theta + (ld + 2);
    double *c2 = gh + (ld + 2);
    double *rc = c2 + (ld + 2);
    double *rs = rc + (ld + 2);
    int *perm = (int *)(rs + (ld + 2));
    const double *GA = a.GA + (long long)b * ld * ld;
    const double *GL = a.GL + (long long)b * ld * ld;
    const double *g = a.g + (long long)b * ld;
#define AT(P, i, j) P[(i) * lds + (j)]

    if (tid == 0) {
        double tA = 0.0, tL = 0.0;
        for (int i = 0; i < K; ++i) {
            tA += GA[i * ld + i];
            tL += GL[i * ld + i];
        }
        s_rho = (tA > 0.0 && tL > 0.0) ? tA / tL : 1.0;
        s_fail = 0;
    }
    __syncthreads();
    const double rho = s_rho;
    for (int e = tid; e < K * K; e += ST) {
        const int i = e / K, j = e % K;
        AT(M, i, j) = GA[i * ld + j] + rho * GL[i * ld + j];
    }
    __syncthreads();
    // Cholesky, upper: M = R^T R, R stored in the upper triangle of M
    for (int j = 0; j < K; ++j) {
        if (tid == 0) {
            const double d = AT(M, j, j);
            if (!(d > 0.0) || !isfinite(d)) s_fail = 1;
            s_piv = d > 0.0 ? sqrt(d) : 1.0;
            AT(M, j, j) = s_piv;
        }
        __syncthreads();
        const double piv = s_piv;
        for (int k = j + 1 + tid; k < K; k += ST) AT(M, j, k) /= piv;
        __syncthreads();
        const int rem = K - j - 1;
        for (int e = tid; e < rem * rem; e += ST) {
            const int k = j + 1 + e / rem, l = j + 1 + e % rem;
            if (l >= k) AT(M, k, l) -= AT(M, j, k) * AT(M, j, l);
        }
        __syncthreads();
    }
    if (s_fail) {
        if (tid == 0) {
            atomicOr(a.err, 1);
            a.lam[b] = 0.0;
            a.flag[b] = 0;
        }
        return;
    }
    // R^-1 by back substitution, one column per thread
    for (int c = tid; c < K; c += ST) {
        for (int i = 0; i < K; ++i) AT(Ri, i, c) = 0.0;
        AT(Ri, c, c) = 1.0 / AT(M, c, c);
        for (int i = c - 1; i >= 0; --i) {
            double s = 0.0;
            for (int k = i + 1; k <= c; ++k) s += AT(M, i, k) * AT(Ri, k, c);
            AT(Ri, i, c) = -s / AT(M, i, i);
        }
    }
    __syncthreads();
    // T = G_A R^-1
    for (int e = tid; e < K * K; e += ST) {
        const int i = e / K, j = e % K;
        double s = 0.0;
        for (int k = 0; k <= j; ++k) s += GA[i * ld + k] * AT(Ri, k, j);
        AT(T, i, j) = s;
    }
    __syncthreads();
    // C = R^-T T (symmetric), into M; padded row/column zero
    for (int e = tid; e < Kp * Kp; e += ST) {
        const int i = e / Kp, j = e % Kp;
        double s = 0.0;
        if (i < K && j < K)
            for (int k = 0; k <= i; ++k) s += AT(Ri, k, i) * AT(T, k, j);
        AT(M, i, j) = s;
        AT(W, i, j) = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    // symmetrise (rounding)
    for (int e = tid; e < K * K; e += ST) {
        const int i = e / K, j = e % K;
        if (i < j) {
            const double v = 0.5 * (AT(M, i, j) + AT(M, j, i));
            AT(M, i, j) = v;
            AT(M, j, i) = v;
        }
    }
    for (int i = tid; i < Kp; i += ST) perm[i] = i;
    __syncthreads();
    // parallel cyclic Jacobi with round-robin pairing
    const int half = Kp / 2;
    for (int sweep = 0; sweep < JACOBI_MAX_SWEEPS; ++sweep) {
        if (tid == 0) {
            double off = 0.0, dia = 0.0;
            for (int i = 0; i < K; ++i)
                for (int j = 0; j < K; ++j) {
                    const double v = AT(M, i, j);
                    if (i == j) dia += v * v;
                    else off += v * v;
                }
            s_conv = !(off > 1e-30 * dia);
        }
        __syncthreads();
        if (s_conv) break;
        for (int round = 0; round < Kp - 1; ++round) {
            if (tid < half) {
                int p = perm[tid], q = perm[Kp - 1 - tid];
                double c = 1.0, s = 0.0;
                if (p < K && q < K) {
                    const double apq = AT(M, p, q);
                    if (apq != 0.0) {
                        const double th = (AT(M, q, q) - AT(M, p, p)) / (2.0 * apq);
                        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        s = t * c;
                    }
                }
                rc[tid] = c;
                rs[tid] = s;
            }
            __syncthreads();
            // columns: A <- A J, W <- W J
            for (int e = tid; e < half * Kp; e += ST) {
                const int pr = e / Kp, r = e % Kp;
                const int p = perm[pr], q = perm[Kp - 1 - pr];
                const double c = rc[pr], s = rs[pr];
                if (s != 0.0) {
                    const double ap = AT(M, r, p), aq = AT(M, r, q);
                    AT(M, r, p) = c * ap - s * aq;
                    AT(M, r, q) = s * ap + c * aq;
                    const double wp = AT(W, r, p), wq = AT(W, r, q);
                    AT(W, r, p) = c * wp - s * wq;
                    AT(W, r, q) = s * wp + c * wq;
                }
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int e = tid; e < half * Kp; e += ST) {
                const int pr = e / Kp, r = e % Kp;
                const int p = perm[pr], q = perm[Kp - 1 - pr];
                const double c = rc[pr], s = rs[pr];
                if (s != 0.0) {
                    const double ap = AT(M, p, r), aq = AT(M, q, r);
                    AT(M, p, r) = c * ap - s * aq;
                    AT(M, q, r) = s * ap + c * aq;
                }
            }
            __syncthreads();
            if (tid == 0) {  // rotate players 1..Kp-1
                const int last = perm[Kp - 1];
                for (int i = Kp - 1; i > 1; --i) perm[i] = perm[i - 1];
                perm[1] = last;
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < K; i += ST) theta[i] = fmin(fmax(AT(M, i, i), 0.0), 1.0);
    __syncthreads();
    // X = R^-1 W into T
    for (int e = tid; e < K * K; e += ST) {
        const int i = e / K, j = e % K;
        double s = 0.0;
        for (int k = i; k < K; ++k) s += AT(Ri, i, k) * AT(W, k, j);
        AT(T, i, j) = s;
    }
    __syncthreads();
    for (int i = tid; i < K; i += ST) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += AT(T, k, i) * g[k];
        gh[i] = s;
        c2[i] = theta[i] > THETA_TINY ? s * s / theta[i] : 0.0;
    }
    __syncthreads();
    if (tid == 0) {
        double kept = 0.0;
        for (int i = 0; i < K; ++i) kept += c2[i];
        s_rho0sq = a.bb[b] - kept;
        s_lo = log10(rho) - BRACKET_DECADES;
        s_hi = log10(rho) + BRACKET_DECADES;
        s_flag = 0;
    }
    __syncthreads();
    Spec S{K, rho, a.bb[b], s_rho0sq, theta, c2};
    double t_sel;
    if (a.rule == MOF_RULE_DP) {
        double lo = s_lo, hi = s_hi;
        if (tid == 0) {
            if (dp_at(S, lo, a.target2) >= 0.0) s_flag = 1;
            else if (dp_at(S, hi, a.target2) <= 0.0) s_flag = 2;
        }
        __syncthreads();
        if (s_flag == 1) t_sel = lo;
        else if (s_flag == 2) t_sel = hi;
        else {
            for (int r = 0; r < DP_ROUNDS; ++r) {
                const double tj = lo + (tid + 1) * (hi - lo) / (ST + 1);
                const double f = dp_at(S, tj, a.target2);
                double vb;
                int ib;
                block_argmin(f > 0.0 ? 0.0 : 1.0, f > 0.0 ? tid : ST, sv, si, vb, ib);
                const double nlo = ib == 0 ? lo : lo + ib * (hi - lo) / (ST + 1);
                const double nhi = ib >= ST ? hi : lo + (ib + 1) * (hi - lo) / (ST + 1);
                lo = nlo;
                hi = nhi;
            }
            t_sel = 0.5 * (lo + hi);
        }
    } else if (a.rule == MOF_RULE_GCV) {
        const double lo = s_lo, hi = s_hi;
        const double step = (hi - lo) / (GRID_POINTS - 1);
        const double v = tid < GRID_POINTS ? gcv_at(S, lo + tid * step) : DBL_MAX;
        double vgrid;
        int ig;
        block_argmin(v, tid, sv, si, vgrid, ig);
        double a0 = lo + max(ig - 1, 0) * step, b0 = lo + min(ig + 1, GRID_POINTS - 1) * step;
        double tbest = lo + ig * step, vbest = vgrid;
        for (int r = 0; r < REFINE_ROUNDS; ++r) {
            const double tj = a0 + tid * (b0 - a0) / (ST - 1);
            double vr;
            int ir;
            block_argmin(gcv_at(S, tj), tid, sv, si, vr, ir);
            const double ts = a0 + ir * (b0 - a0) / (ST - 1);
            if (vr < vbest) {
                vbest = vr;
                tbest = ts;
            }
            const double na = a0 + max(ir - 1, 0) * (b0 - a0) / (ST - 1);
            const double nb = a0 + min(ir + 1, ST - 1) * (b0 - a0) / (ST - 1);
            a0 = na;
            b0 = nb;
        }
        t_sel = tbest;
    } else {
        t_sel = log10(fmax(a.lam_fixed, 1e-300));
    }
    const double lam = a.rule == MOF_RULE_FIXED ? a.lam_fixed : exp10(t_sel);
    const double mu = lam / rho;
    // z = X diag(1/(theta + mu (1 - theta))) gh
    for (int i = tid; i < K; i += ST) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) {
            const double d = theta[k] + mu * (1.0 - theta[k]);
            if (d > 0.0) s += AT(T, i, k) * gh[k] / d;
        }
        z[i] = s;
        if (!isfinite(s)) atomicOr(a.err, 2);
    }
    if (tid == 0) {
        a.lam[b] = lam;
        a.flag[b] = s_flag;
    }
#undef AT
}

mof_status launch_small_solve(const SmallArgs &a, cudaStream_t st) {
    const int ld = a.ld;
    const size_t lds = (size_t)ld + 2;
    const size_t smem = sizeof(double) * (4 * lds * lds + 5 * lds) + sizeof(int) * lds;
    static size_t configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        MOF_CUDA(cudaFuncSetAttribute(k_small_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = smem;
    }
    k_small_solve<<<a.B, ST, smem, st>>>(a);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

}  // namespace mof
