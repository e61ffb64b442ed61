// K11: the small projected problem of MMGKS / GKS, in FP64, one block per
// problem (Sec. 4.1.1 eq. (QR)-(minKryov2), Sec. 4.1.3 DP and GCV).
//
// Given the Gram matrices G_A = (A V)^T (A V), G_L = (L V)^T (L V) and
// g = (A V)^T b of the current basis (R_A^T R_A = G_A and R_L^T R_L = G_L for
// the R factors of eq. (QR)), the block
//   1. factors M = G_A + rho G_L = R^T R (Cholesky, FP64), rho = tr G_A / tr G_L,
//      and forms C = R^-T G_A R^-1 and h = R^-T g (FP64);
//   2. diagonalises C: cyclic Jacobi sweeps in FP32 give approximate
//      eigenvectors W; two Newton-Schulz steps make them orthonormal in FP64
//      (W <- W (3I - W^T W)/2), and cyclic Jacobi sweeps in FP64 on W^T C W,
//      which start near diagonal and converge quadratically, finish the
//      decomposition to FP64 accuracy; with the eigenvalues theta_i in [0, 1]
//      and eigenvectors W, X = R^-1 W satisfies X^T G_A X = diag(theta),
//      X^T G_L X = diag(1 - theta)/rho (the generalized singular values of
//      (R_A, R_L)); the FP64 sweeps rotate the one vector W^T h they need
//      instead of accumulating W;
//   3. with ghat = X^T g, chat_i^2 = ghat_i^2 / theta_i and the filter factors
//      f_i = theta_i / (theta_i + mu (1 - theta_i)), mu = lam / rho, has
//      ||R_A z - Q_A^T b||^2 = sum chat_i^2 (1 - f_i)^2 and
//      trace(I - S) = sum (1 - f_i), with closed-form derivatives in lam;
//   4. picks lam on the bracket 10^[log10 rho - 12, log10 rho + 12]:
//      DP: the root of ||A V z - b||^2 = (eta delta)^2 (monotone in lam) by
//      safeguarded Newton steps in log10 lam; GCV: the minimum of a 200-point
//      log grid (ties to the smaller lam), refined inside its two grid
//      neighbours by safeguarded Newton steps on dG/dlog10(lam) = 0, kept only
//      if it improves on the grid value;
//   5. returns z = R^-1 (C + mu (I - C))^-1 h, the solution of
//      (G_A + lam G_L) z = g, by an FP64 Cholesky solve in the R basis.
// Each Jacobi round updates every 2x2 block (pair i rows, pair j columns) of
// the matrix from its old values in one pass, so a round costs two barriers.
#include "solver.cuh"

#include <atomic>
#include <cfloat>

namespace mof {

namespace {

constexpr int ST = 256;
constexpr int GRID_POINTS = 200;
constexpr int NEWTON_MAX = 60;
constexpr double BRACKET_DECADES = 12.0;
constexpr double THETA_TINY = 1e-14;
constexpr int JACOBI32_MAX_SWEEPS = 12;
constexpr int JACOBI64_MAX_SWEEPS = 10;
constexpr double LN10 = 2.302585092994045684;

struct Spec {
    int K;
    double rho, rho0sq;
    const double *theta, *c2;
};

// sums over i (lane-strided) of the lam-functions and their mu-derivatives:
// s[0] = N = sum c2 g^2, s[1] = N', s[2] = N'', s[3] = D = sum g, s[4] = D', s[5] = D''
// with g_i = mu a_i / d_i = 1 - f_i, a_i = 1 - theta_i, d_i = theta_i + mu a_i.
__device__ __forceinline__ void lam_sums(const Spec &S, double mu, int i0, int step, double s[6]) {
    for (int k = 0; k < 6; ++k) s[k] = 0.0;
    for (int i = i0; i < S.K; i += step) {
        const double th = S.theta[i], a = 1.0 - th, d = th + mu * a;
        if (!(d > 0.0)) {
            s[3] += 1.0;
            continue;
        }
        const double inv = 1.0 / d;
        const double g = mu * a * inv;
        const double g1 = a * th * inv * inv;
        const double g2 = -2.0 * a * g1 * inv;
        const double c = S.c2[i];
        s[0] += c * g * g;
        s[1] += 2.0 * c * g * g1;
        s[2] += 2.0 * c * (g1 * g1 + g * g2);
        s[3] += g;
        s[4] += g1;
        s[5] += g2;
    }
}

// N = sum c2 g^2 and D = sum g only (the grid scan)
__device__ __forceinline__ double gcv_plain(const Spec &S, double mu) {
    double N = 0.0, D = 0.0;
    for (int i = 0; i < S.K; ++i) {
        const double th = S.theta[i], a = 1.0 - th, d = th + mu * a;
        const double g = d > 0.0 ? mu * a / d : 1.0;
        N += S.c2[i] * g * g;
        D += g;
    }
    const double v = N / (D * D);
    return v == v ? v : DBL_MAX;
}

__device__ __forceinline__ void warp_lam_sums(const Spec &S, double t, double s[6]) {
    const double mu = exp10(t) / S.rho;
    lam_sums(S, mu, threadIdx.x & 31, 32, s);
#pragma unroll
    for (int k = 0; k < 6; ++k) s[k] = warp_sum(s[k]);
}

__device__ __forceinline__ double gcv_of(const double s[6]) {
    const double g = s[0] / (s[3] * s[3]);
    return g == g ? g : DBL_MAX;
}

// first and second derivative of G = N / D^2 with respect to t = log10(lam)
__device__ __forceinline__ void gcv_dt(const double s[6], double mu, double &d1, double &d2) {
    const double N = s[0], N1 = s[1], N2 = s[2], D = s[3], D1 = s[4], D2 = s[5];
    const double G1 = N1 / (D * D) - 2.0 * N * D1 / (D * D * D);
    const double G2 =
        N2 / (D * D) - 4.0 * N1 * D1 / (D * D * D) - 2.0 * N * D2 / (D * D * D) + 6.0 * N * D1 * D1 / (D * D * D * D);
    d1 = G1 * mu * LN10;
    d2 = (G2 * mu * mu + G1 * mu) * LN10 * LN10;
}

// round-robin tournament: player at position j in round r (positions 0..Kp-1)
__device__ __forceinline__ int rr_player(int j, int r, int Kp) {
    int v = j - 1 + r;
    if (v >= Kp - 1) v -= Kp - 1;
    return j == 0 ? 0 : 1 + v;
}

// Rotation (c, s) that zeroes a_pq of the 2x2 block [[a_pp, a_pq], [a_pq, a_qq]]:
// t = tan(phi) from the classical formula, c = 1/sqrt(1 + t^2), s = t c. For
// the FP64 sweeps the angle itself is computed in FP32 and c, s in FP64 from
// it: the rotation stays orthogonal to FP64 accuracy, and an angle accurate
// to FP32 still shrinks a_pq by ~1e-7 per visit once the matrix is near
// diagonal (the quadratic phase these sweeps run in).
__device__ __forceinline__ void rot_angle(float app, float aqq, float apq, float &c, float &s) {
    const float th = (aqq - app) / (2.0f * apq);
    const float t = (th >= 0.0f ? 1.0f : -1.0f) / (fabsf(th) + sqrtf(th * th + 1.0f));
    c = rsqrtf(t * t + 1.0f);
    s = t * c;
}
__device__ __forceinline__ void rot_angle(double app, double aqq, double apq, double &c, double &s) {
    const float th = (float)(aqq - app) / (2.0f * (float)apq);
    const double t = (double)((th >= 0.0f ? 1.0f : -1.0f) / (fabsf(th) + sqrtf(th * th + 1.0f)));
    c = rsqrt(fma(t, t, 1.0));
    s = t * c;
}

// Cyclic two-sided Jacobi sweeps on the symmetric Kp x Kp matrix A (padded
// rows/columns beyond K are zero) with eigenvector accumulation W <- W J
// (W may be null) and/or the rotations applied to one vector v <- J^T v (v may be null),
// until a sweep applies no rotation (|a_pq| <= rel * sqrt(|a_pp a_qq|) or
// |a_pq| <= rel_abs * max_i |a_ii|) or max_sweeps. Every warp computes the
// round's rotations itself (pair index = lane) and takes the others' by
// shuffle; a barrier separates the pivot reads from the block updates and
// another ends the round. All threads must call.
template <typename T>
__device__ void jacobi(T *A, int lda, T *W, int ldw, T *v, int K, int Kp, int max_sweeps, T rel, T rel_abs, double *red) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int half = Kp / 2;
    double dm = 0.0;
    for (int i = tid; i < K; i += ST) dm = fmax(dm, fabs((double)A[i * lda + i]));
    for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    if (lane == 0) red[wid] = dm;
    __syncthreads();
    dm = 0.0;
    for (int w = 0; w < ST / 32; ++w) dm = fmax(dm, red[w]);
    __syncthreads();
    const T floor_abs = rel_abs * (T)dm;
    const T tiny = (T)(sizeof(T) == 8 ? 1e-300 : 1e-30);
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        int any_in_sweep = 0;
        for (int round = 0; round < Kp - 1; ++round) {
            const int pl = rr_player(lane, round, Kp), ql = rr_player(Kp - 1 - lane, round, Kp);
            T c = 1, s = 0;
            if (lane < half && pl < K && ql < K) {
                const T apq = A[pl * lda + ql], app = A[pl * lda + pl], aqq = A[ql * lda + ql];
                if (fabs(apq) > rel * sqrt(fabs(app * aqq)) && fabs(apq) > floor_abs && fabs(apq) > tiny)
                    rot_angle(app, aqq, apq, c, s);
            }
            if (!__any_sync(0xffffffffu, s != (T)0)) continue;  // identical decision in every warp
            any_in_sweep = 1;
            __syncthreads();  // every warp has read this round's pivots before any block is rewritten
            for (int j = wid; j < half; j += ST / 32) {
                const int pj = rr_player(j, round, Kp), qj = rr_player(Kp - 1 - j, round, Kp);
                const T cj = __shfl_sync(0xffffffffu, c, j), sj = __shfl_sync(0xffffffffu, s, j);
                if (lane < half) {
                    const T a = A[pl * lda + pj], b = A[pl * lda + qj], cc = A[ql * lda + pj], d = A[ql * lda + qj];
                    const T a1 = c * a - s * cc, b1 = c * b - s * d, c1 = s * a + c * cc, d1 = s * b + c * d;
                    A[pl * lda + pj] = cj * a1 - sj * b1;
                    A[pl * lda + qj] = sj * a1 + cj * b1;
                    A[ql * lda + pj] = cj * c1 - sj * d1;
                    A[ql * lda + qj] = sj * c1 + cj * d1;
                }
            }
            if (W && lane < half && s != (T)0)
                for (int r = wid; r < Kp; r += ST / 32) {  // W <- W J on the columns of pair `lane`
                    const T wp = W[r * ldw + pl], wq = W[r * ldw + ql];
                    W[r * ldw + pl] = c * wp - s * wq;
                    W[r * ldw + ql] = s * wp + c * wq;
                }
            if (v && wid == 0 && lane < half && s != (T)0) {  // v <- J^T v
                const T vp = v[pl], vq = v[ql];
                v[pl] = c * vp - s * vq;
                v[ql] = s * vp + c * vq;
            }
            __syncthreads();
        }
        if (!any_in_sweep) break;
    }
}

}  // namespace

__global__ void __launch_bounds__(ST) k_small_solve(SmallArgs a) {
    extern __shared__ double sm[];
    __shared__ double s_rho, s_piv, s_rho0sq, s_t, s_vgrid;
    __shared__ double s_red[ST / 32];
    __shared__ int s_fail, s_flag, s_ig, s_idx[ST / 32];
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
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
    const int Kp = K + (K & 1);
    const int lds = ld + 2;       // FP64 leading dimension (>= Kp)
    const int ldf = ld + 3;       // FP32 leading dimension
    double *M = sm;               // Cholesky factor R (upper), later X^T C X
    double *Ri = M + lds * lds;   // R^-1
    double *C = Ri + lds * lds;   // G_A, then C = R^-T G_A R^-1
    double *T = C + lds * lds;    // scratch: G_A R^-1, Newton-Schulz products, C X
    double *X = T + lds * lds;    // eigenvector estimate
    double *E = X + lds * lds;    // G_L, then scratch
    double *vec = E + lds * lds;  // vectors, lds each
    double *theta = vec, *gh = vec + lds, *c2 = vec + 2 * lds, *h = vec + 3 * lds, *y = vec + 4 * lds;
    float *Af = reinterpret_cast<float *>(T);  // FP32 Jacobi matrices alias T and E (free then)
    float *Wf = reinterpret_cast<float *>(E);
    const double *GA = a.GA + (long long)b * ld * ld;
    const double *GL = a.GL + (long long)b * ld * ld;
    const double *g = a.g + (long long)b * ld;
#define AT(P, i, j) P[(i) * lds + (j)]
#define AF(P, i, j) P[(i) * ldf + (j)]

    // ---------------------------------------------- 1. Cholesky, C, h (FP64)
    for (int e = tid; e < K * K; e += ST) {
        const int i = e / K, j = e - (e / K) * K;
        AT(C, i, j) = GA[i * ld + j];
        AT(E, i, j) = GL[i * ld + j];
    }
    for (int i = tid; i < K; i += ST) y[i] = g[i];
    __syncthreads();
    if (tid < 32) {
        double tA = 0.0, tL = 0.0;
        for (int i = lane; i < K; i += 32) {
            tA += AT(C, i, i);
            tL += AT(E, i, i);
        }
        tA = warp_sum(tA);
        tL = warp_sum(tL);
        if (lane == 0) {
            s_rho = (tA > 0.0 && tL > 0.0) ? tA / tL : 1.0;
            s_fail = 0;
        }
    }
    __syncthreads();
    const double rho = s_rho;
    for (int e = tid; e < K * K; e += ST) {
        const int i = e / K, j = e - (e / K) * K;
        AT(M, i, j) = AT(C, i, j) + rho * AT(E, i, j);
    }
    __syncthreads();
    for (int j = 0; j < K; ++j) {
        if (tid == 0) {
            const double d = AT(M, j, j);
            if (!(d > 0.0) || !isfinite(d)) s_fail = 1;
            s_piv = d > 0.0 ? sqrt(d) : 1.0;
            AT(M, j, j) = s_piv;
        }
        __syncthreads();
        const double inv = 1.0 / s_piv;
        for (int k = j + 1 + tid; k < K; k += ST) AT(M, j, k) *= inv;
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
    for (int e = tid; e < K * K; e += ST) {  // T = G_A R^-1
        const int i = e / K, j = e - (e / K) * K;
        double s = 0.0;
        for (int k = 0; k <= j; ++k) s += AT(C, i, k) * AT(Ri, k, j);
        AT(T, i, j) = s;
    }
    for (int i = tid; i < K; i += ST) {  // h = R^-T g
        double s = 0.0;
        for (int k = 0; k <= i; ++k) s += AT(Ri, k, i) * y[k];
        h[i] = s;
    }
    __syncthreads();
    for (int e = tid; e < K * K; e += ST) {  // C = R^-T T (upper triangle, mirrored)
        const int i = e / K, j = e - (e / K) * K;
        if (i > j) continue;
        double s = 0.0;
        for (int k = 0; k <= i; ++k) s += AT(Ri, k, i) * AT(T, k, j);
        AT(C, i, j) = s;
        AT(C, j, i) = s;
    }
    __syncthreads();

    // ---------------------------------------------- 2a. FP32 Jacobi on C
    for (int e = tid; e < Kp * Kp; e += ST) {
        const int i = e / Kp, j = e - (e / Kp) * Kp;
        AF(Af, i, j) = (i < K && j < K) ? (float)AT(C, i, j) : 0.0f;
        AF(Wf, i, j) = i == j ? 1.0f : 0.0f;
    }
    __syncthreads();
    jacobi<float>(Af, ldf, Wf, ldf, (float *)nullptr, K, Kp, JACOBI32_MAX_SWEEPS, 1e-6f, 1e-7f, s_red);

    // ---------------------------------------------- 2b. FP64: orthonormalise, then Jacobi
    for (int e = tid; e < K * K; e += ST) {
        const int i = e / K, j = e - (e / K) * K;
        AT(X, i, j) = (double)AF(Wf, i, j);
    }
    __syncthreads();
    for (int step = 0; step < 2; ++step) {  // Newton-Schulz: X <- X (3I - X^T X) / 2
        for (int e = tid; e < K * K; e += ST) {
            const int i = e / K, j = e - (e / K) * K;
            if (i > j) continue;
            double s = 0.0;
            for (int k = 0; k < K; ++k) s += AT(X, k, i) * AT(X, k, j);
            AT(E, i, j) = s;
            AT(E, j, i) = s;
        }
        __syncthreads();
        for (int e = tid; e < K * K; e += ST) {
            const int i = e / K, j = e - (e / K) * K;
            double s = 0.0;
            for (int k = 0; k < K; ++k) s += AT(X, i, k) * ((k == j ? 3.0 : 0.0) - AT(E, k, j));
            AT(T, i, j) = 0.5 * s;
        }
        __syncthreads();
        for (int e = tid; e < K * K; e += ST) {
            const int i = e / K, j = e - (e / K) * K;
            AT(X, i, j) = AT(T, i, j);
        }
        __syncthreads();
    }
    for (int e = tid; e < K * K; e += ST) {  // T = C X
        const int i = e / K, j = e - (e / K) * K;
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += AT(C, i, k) * AT(X, k, j);
        AT(T, i, j) = s;
    }
    __syncthreads();
    for (int e = tid; e < Kp * Kp; e += ST) {  // M = X^T C X (padded row/column zero, X padded by I)
        const int i = e / Kp, j = e - (e / Kp) * Kp;
        if (i > j) continue;
        double s = 0.0;
        if (j < K)
            for (int k = 0; k < K; ++k) s += AT(X, k, i) * AT(T, k, j);
        AT(M, i, j) = s;
        AT(M, j, i) = s;
        if (j == K) {
            AT(X, i, j) = (i == j) ? 1.0 : 0.0;
            AT(X, j, i) = (i == j) ? 1.0 : 0.0;
        }
    }
    __syncthreads();
    for (int i = tid; i < Kp; i += ST) {  // gh = X^T h, then rotated along with M
        double s = 0.0;
        if (i < K)
            for (int k = 0; k < K; ++k) s += AT(X, k, i) * h[k];
        gh[i] = s;
    }
    __syncthreads();
    jacobi<double>(M, lds, (double *)nullptr, lds, gh, K, Kp, JACOBI64_MAX_SWEEPS, 1e-16, 1e-18, s_red);
    for (int i = tid; i < K; i += ST) {
        theta[i] = fmin(fmax(AT(M, i, i), 0.0), 1.0);
        c2[i] = theta[i] > THETA_TINY ? gh[i] * gh[i] / theta[i] : 0.0;
    }
    __syncthreads();

    // ---------------------------------------------- 3-4. lambda
    if (tid < 32) {
        double kept = 0.0;
        for (int i = lane; i < K; i += 32) kept += c2[i];
        kept = warp_sum(kept);
        if (lane == 0) {
            s_rho0sq = a.bb[b] - kept;
            s_flag = 0;
        }
    }
    __syncthreads();
    const Spec S{K, rho, s_rho0sq, theta, c2};
    const double lo = log10(rho) - BRACKET_DECADES, hi = log10(rho) + BRACKET_DECADES;
    if (a.rule == MOF_RULE_GCV) {
        const double step = (hi - lo) / (GRID_POINTS - 1);
        double vb = DBL_MAX;
        int ib = tid;
        if (tid < GRID_POINTS) vb = gcv_plain(S, exp10(lo + tid * step) / rho);
        for (int o = 16; o > 0; o >>= 1) {  // argmin, ties to the smaller index
            const double vo = __shfl_xor_sync(0xffffffffu, vb, o);
            const int io = __shfl_xor_sync(0xffffffffu, ib, o);
            if (vo < vb || (vo == vb && io < ib)) {
                vb = vo;
                ib = io;
            }
        }
        if (lane == 0) {
            s_red[wid] = vb;
            s_idx[wid] = ib;
        }
        __syncthreads();
        if (tid == 0) {
            double bv = s_red[0];
            int bi = s_idx[0];
            for (int w = 1; w < ST / 32; ++w) {
                if (s_red[w] < bv || (s_red[w] == bv && s_idx[w] < bi)) {
                    bv = s_red[w];
                    bi = s_idx[w];
                }
            }
            s_vgrid = bv;
            s_ig = bi;
        }
        __syncthreads();
        if (wid == 0) {
            // safeguarded Newton on dG/dt inside [t_{i-1}, t_{i+1}]
            const int ig = s_ig;
            double A0 = lo + max(ig - 1, 0) * step, B0 = lo + min(ig + 1, GRID_POINTS - 1) * step;
            double t = lo + ig * step, s[6], d1, d2;
            for (int it = 0; it < NEWTON_MAX; ++it) {
                warp_lam_sums(S, t, s);
                gcv_dt(s, exp10(t) / rho, d1, d2);
                if (d1 > 0.0) B0 = t;
                else if (d1 < 0.0) A0 = t;
                else break;
                double tn = (d2 > 0.0) ? t - d1 / d2 : 0.5 * (A0 + B0);
                if (!(tn > A0 && tn < B0)) tn = 0.5 * (A0 + B0);
                const double dt = fabs(tn - t);
                t = tn;
                if (dt <= 1e-10 * fmax(1.0, fabs(t)) || B0 - A0 <= 1e-10 * fmax(1.0, fabs(t))) break;
            }
            warp_lam_sums(S, t, s);
            if (gcv_of(s) > s_vgrid) t = lo + ig * step;
            if (lane == 0) s_t = t;
        }
        __syncthreads();
    } else if (a.rule == MOF_RULE_DP) {
        if (wid == 0) {
            double s[6], t;
            warp_lam_sums(S, lo, s);
            const double flo = s[0] + S.rho0sq - a.target2;
            warp_lam_sums(S, hi, s);
            const double fhi = s[0] + S.rho0sq - a.target2;
            int flag = 0;
            if (flo >= 0.0) {
                flag = 1;
                t = lo;
            } else if (fhi <= 0.0) {
                flag = 2;
                t = hi;
            } else {
                // safeguarded Newton on F(t) = N(mu(t)) + rho0^2 - target^2 (increasing in t)
                double A0 = lo, B0 = hi;
                t = 0.5 * (lo + hi);
                for (int it = 0; it < NEWTON_MAX; ++it) {
                    warp_lam_sums(S, t, s);
                    const double mu = exp10(t) / rho;
                    const double F = s[0] + S.rho0sq - a.target2;
                    const double F1 = s[1] * mu * LN10;
                    if (F > 0.0) B0 = t;
                    else A0 = t;
                    double tn = F1 > 0.0 ? t - F / F1 : 0.5 * (A0 + B0);
                    if (!(tn > A0 && tn < B0)) tn = 0.5 * (A0 + B0);
                    const double dt = fabs(tn - t);
                    t = tn;
                    if (dt <= 1e-15 * fmax(1.0, fabs(t)) || B0 - A0 <= 1e-15 * fmax(1.0, fabs(t))) break;
                }
            }
            if (lane == 0) {
                s_t = t;
                s_flag = flag;
            }
        }
        __syncthreads();
    } else {
        if (tid == 0) s_t = 0.0;
        __syncthreads();
    }
    const double lam = a.rule == MOF_RULE_FIXED ? a.lam_fixed : exp10(s_t);
    const double mu = lam / rho;

    // ---------------------------------------------- 5. z = R^-1 (C + mu (I - C))^-1 h
    // (G_A + lam G_L = R^T (C + mu (I - C)) R and g = R^T h)
    for (int e = tid; e < K * K; e += ST) {
        const int i = e / K, j = e - (e / K) * K;
        AT(M, i, j) = (1.0 - mu) * AT(C, i, j) + (i == j ? mu : 0.0);
    }
    for (int i = tid; i < K; i += ST) y[i] = h[i];
    __syncthreads();
    for (int j = 0; j < K; ++j) {  // Cholesky, upper, in M
        if (tid == 0) {
            const double d = AT(M, j, j);
            if (!(d > 0.0) || !isfinite(d)) s_fail = 1;
            s_piv = d > 0.0 ? sqrt(d) : 1.0;
            AT(M, j, j) = s_piv;
        }
        __syncthreads();
        const double inv = 1.0 / s_piv;
        for (int k = j + 1 + tid; k < K; k += ST) AT(M, j, k) *= inv;
        __syncthreads();
        const int rem = K - j - 1;
        for (int e = tid; e < rem * rem; e += ST) {
            const int k = j + 1 + e / rem, l = j + 1 + e % rem;
            if (l >= k) AT(M, k, l) -= AT(M, j, k) * AT(M, j, l);
        }
        __syncthreads();
    }
    if (wid == 0) {  // forward (R^T w = h) and backward (R y = w) substitution, one warp
        for (int i = 0; i < K; ++i) {
            double s = 0.0;
            for (int k = lane; k < i; k += 32) s += AT(M, k, i) * y[k];
            s = warp_sum(s);
            if (lane == 0) y[i] = (y[i] - s) / AT(M, i, i);
            __syncwarp();
        }
        for (int i = K - 1; i >= 0; --i) {
            double s = 0.0;
            for (int k = i + 1 + lane; k < K; k += 32) s += AT(M, i, k) * y[k];
            s = warp_sum(s);
            if (lane == 0) y[i] = (y[i] - s) / AT(M, i, i);
            __syncwarp();
        }
    }
    __syncthreads();
    for (int i = tid; i < K; i += ST) {
        double s = 0.0;
        for (int k = i; k < K; ++k) s += AT(Ri, i, k) * y[k];
        z[i] = s;
        if (!isfinite(s) || s_fail) atomicOr(a.err, 2);
    }
    if (tid == 0) {
        a.lam[b] = lam;
        a.flag[b] = s_flag;
    }
#undef AT
#undef AF
}

static size_t small_smem(int ld) {
    const size_t lds = (size_t)ld + 2;
    return sizeof(double) * (6 * lds * lds + 5 * lds);
}

mof_status prepare_small_solve(int ld) {
    // the limit only ever grows: smaller problems launched later still fit
    static std::atomic<size_t> configured{48 * 1024};
    const size_t smem = small_smem(ld);
    size_t cur = configured.load();
    while (smem > cur) {
        MOF_CUDA(cudaFuncSetAttribute(k_small_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (configured.compare_exchange_weak(cur, smem)) break;
    }
    return MOF_OK;
}

mof_status launch_small_solve(const SmallArgs &a, cudaStream_t st) {
    const size_t smem = small_smem(a.ld);
    ::mof::count_launch(), k_small_solve<<<a.B, ST, smem, st>>>(a);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

}  // namespace mof
