// K11: the small projected problem of MMGKS / GKS, in FP64, one block per
// problem (Sec. 4.1.1 eq. (QR)-(minKryov2), Sec. 4.1.3 DP and GCV).
//
// Given the Gram matrices G_A = (A V)^T (A V), G_L = (L V)^T (L V) and
// g = (A V)^T b of the current basis (R_A^T R_A = G_A and R_L^T R_L = G_L for
// the R factors of eq. (QR)), the block
//   1. factors M = G_A + rho G_L = R^T R (Cholesky, FP64), rho = tr G_A / tr G_L,
//      and forms C = R^-T G_A R^-1 and h = R^-T g by two triangular solves;
//   2. diagonalises C: cyclic one-sided Jacobi sweeps in FP32 (four warps,
//      each holding a quarter of every column) give approximate
//      eigenvectors W; one third-order Newton-Schulz step makes them
//      orthonormal in FP64 (W <- W (I - E/2 + 3E^2/8), E = W^T W - I), and
//      cyclic Jacobi sweeps in FP64 on W^T C W, which start near diagonal,
//      finish the decomposition (usually in one sweep: the sweeps stop once no
//      off-diagonal entry exceeds 1e-12 max|c_ii|) while rotating the one vector
//      W^T h they need; with the eigenvalues theta_i in [0, 1] and the
//      eigenvectors, X = R^-1 W satisfies X^T G_A X = diag(theta),
//      X^T G_L X = diag(1 - theta)/rho (the generalized singular values of
//      (R_A, R_L));
//   3. with ghat = X^T g, chat_i^2 = ghat_i^2 / theta_i and the filter factors
//      f_i = theta_i / (theta_i + mu (1 - theta_i)), mu = lam / rho, has
//      ||R_A z - Q_A^T b||^2 = sum chat_i^2 (1 - f_i)^2 and
//      trace(I - S) = sum (1 - f_i), with closed-form derivatives in lam;
//   4. picks lam on the bracket 10^[log10 rho - 12, log10 rho + 12]:
//      GCV: the first minimum of a 200-point log grid (ties to the smaller
//      lam), every point evaluated in FP64 (one thread per point), then
//      refined between its two grid neighbours by
//      safeguarded Newton steps on dG/dlog10(lam) = 0 (FP32 steps, then FP64
//      steps, which stop after a Newton step below 1e-6 -- the next would be
//      below ~1e-12 -- or once the derivative is at its rounding level), kept
//      only if it improves on the grid value; where the five FP64 values agree
//      to 1e-13 the neighbourhood is flat to rounding (the plateau G takes
//      as lam -> 0 when every theta_i > 0) and the grid point stands;
//      DP: the root of ||A V z - b||^2 = (eta delta)^2 (monotone in lam); the
//      bracket ends decide the no-root flags in FP64, an FP32 grid locates the
//      sign change (its cell is confirmed in FP64), and safeguarded Newton
//      steps in log10 lam (FP32, then FP64) converge to the root;
//   5. returns z = R^-1 (C + mu (I - C))^-1 h, the solution of
//      (G_A + lam G_L) z = g, by an FP64 Cholesky solve in the R basis.
//
// GB300 executes FP64 at about 2 fused multiply-adds per clock per SM, and a
// warp's FP64 instruction costs the same with one lane active as with 32, so
// the block does its FP64 arithmetic with full warps wherever the work is
// parallel (triangular updates over all threads, symmetric products over the
// upper triangle), keeps the serial parts (pivots, rotation angles,
// substitutions, Newton steps) in one warp, and evaluates in FP32 what a
// later FP64 step corrects (the Jacobi warm start, the lambda grids).
#include "solver.cuh"

#include <atomic>
#include <cfloat>

namespace mof {

namespace {

constexpr int ST = 256;
constexpr int NW = ST / 32;
constexpr int GRID_POINTS = 200;
constexpr int NEWTON_MAX = 60;
constexpr int NEWTON32_MAX = 30;
constexpr int NREF = 5;  // FP64 re-evaluated grid points around the FP32 minimum
constexpr double BRACKET_DECADES = 12.0;
constexpr double THETA_TINY = 1e-14;
constexpr int JACOBI32_MAX_SWEEPS = 12;
constexpr int JACOBI64_MAX_SWEEPS = 10;
constexpr int JW = 4;  // warps of the FP32 one-sided Jacobi
constexpr int RW = 32 / JW;
constexpr double LN10 = 2.302585092994045684;

// ------------------------------------------------------------ index helpers
// The n(n+1)/2 pairs (r, c), r <= c < n, of an upper triangle enumerated as a
// ceil(n/2) x (n+1) rectangle whose row q holds triangle rows q and n-1-q.
__device__ __forceinline__ int tri_count(int n) { return ((n + 1) / 2) * (n + 1); }
__device__ __forceinline__ bool tri_pair(int e, int n, int &r, int &c) {
    const int q = e / (n + 1), x = e - q * (n + 1);
    if (x < n - q) {
        r = q;
        c = q + x;
        return true;
    }
    r = n - 1 - q;
    if (r == q) return false;  // middle row of an odd n: already enumerated
    c = r + (x - (n - q));
    return true;
}

// round-robin tournament: player at position j in round r (positions 0..Kp-1)
__device__ __forceinline__ int rr_player(int j, int r, int Kp) {
    int v = j - 1 + r;
    if (v >= Kp - 1) v -= Kp - 1;
    return j == 0 ? 0 : 1 + v;
}

// ------------------------------------------------------------ reductions
// Sums over the warp of two values, each returned to every lane; 5 FP64
// additions per lane instead of 10.
__device__ __forceinline__ void warp_sum2(double &a, double &b) {
    const bool hi = (threadIdx.x & 16) != 0;
    double y = (hi ? b : a) + __shfl_xor_sync(0xffffffffu, hi ? a : b, 16);
    for (int o = 8; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
    a = __shfl_sync(0xffffffffu, y, 0);
    b = __shfl_sync(0xffffffffu, y, 16);
}
// Sums over the warp of six values with 8 FP64 additions per lane instead of
// 30: each shuffle level halves the number of distinct partial sums a lane
// carries; the totals end in lanes 0, 16, 8, 24, 4, 20 and are broadcast.
__device__ __forceinline__ void warp_sum6(double s[6]) {
    const int lane = threadIdx.x & 31;
    const bool h = (lane & 16) != 0, g = (lane & 8) != 0, f = (lane & 4) != 0;
    const double r0 = __shfl_xor_sync(0xffffffffu, h ? s[0] : s[1], 16);
    const double r1 = __shfl_xor_sync(0xffffffffu, h ? s[2] : s[3], 16);
    const double r2 = __shfl_xor_sync(0xffffffffu, h ? s[4] : s[5], 16);
    const double a = (h ? s[1] : s[0]) + r0, b = (h ? s[3] : s[2]) + r1;
    double c = (h ? s[5] : s[4]) + r2;
    const double x = (g ? b : a) + __shfl_xor_sync(0xffffffffu, g ? a : b, 8);
    c += __shfl_xor_sync(0xffffffffu, c, 8);
    double y = (f ? c : x) + __shfl_xor_sync(0xffffffffu, f ? x : c, 4);
    y += __shfl_xor_sync(0xffffffffu, y, 2);
    y += __shfl_xor_sync(0xffffffffu, y, 1);
    s[0] = __shfl_sync(0xffffffffu, y, 0);
    s[1] = __shfl_sync(0xffffffffu, y, 16);
    s[2] = __shfl_sync(0xffffffffu, y, 8);
    s[3] = __shfl_sync(0xffffffffu, y, 24);
    s[4] = __shfl_sync(0xffffffffu, y, 4);
    s[5] = __shfl_sync(0xffffffffu, y, 20);
}

// ------------------------------------------------------------ dense kernels
// Upper Cholesky in place: on return row j of A holds R[j][j..K) with
// A = R^T R (only the upper triangle of A is referenced) and
// invd[j] = 1 / R[j][j]. One barrier per column: warp 0 factors the pivot
// row, which it brought up to date itself in the previous column, while the
// other warps finish the previous column's trailing update. A non-positive or
// non-finite pivot sets *fail. All threads call; ends with a barrier.
__device__ void chol_upper(double *A, int lds, int K, double *invd, int *fail) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int j = 0; j < K; ++j) {
        if (wid == 0) {
            const double d = A[j * lds + j];
            const bool ok = d > 0.0 && isfinite(d);
            const double rs = ok ? rsqrt(d) : 1.0;
            for (int k = j + lane; k < K; k += 32) A[j * lds + k] = (k == j) ? d * rs : A[j * lds + k] * rs;
            if (lane == 0) {
                invd[j] = rs;
                if (!ok) *fail = 1;
            }
        }
        __syncthreads();
        if (wid == 0) {
            const int k = j + 1;
            if (k < K) {
                const double ajk = A[j * lds + k];
                for (int l = k + lane; l < K; l += 32) A[k * lds + l] -= ajk * A[j * lds + l];
            }
            __syncwarp();
        } else {
            const int n = K - j - 2;  // rows j+2 .. K-1
            if (n > 0) {
                const int cnt = tri_count(n);
                for (int e = tid - 32; e < cnt; e += ST - 32) {
                    int r, c;
                    if (!tri_pair(e, n, r, c)) continue;
                    const int k = j + 2 + r, l = j + 2 + c;
                    A[k * lds + l] -= A[j * lds + k] * A[j * lds + l];
                }
            }
        }
    }
    __syncthreads();
}

// Y <- R^-T Y for the K x nc block Y (row stride ldy): forward substitution
// in column-oriented form with the division by R[i][i] deferred to the end,
// so the update by row i needs U[i][k] = R[i][k] / R[i][i] (k > i) only. One
// barrier per row; all threads call; ends with a barrier.
__device__ void trsm_rt(const double *U, int ldu, const double *invd, double *Y, int ldy, int K, int nc) {
    const int tid = threadIdx.x;
    for (int i = 0; i + 1 < K; ++i) {
        const int cnt = (K - 1 - i) * nc;
        for (int e = tid; e < cnt; e += ST) {
            const int k = i + 1 + e / nc, j = e - (e / nc) * nc;
            Y[k * ldy + j] -= U[i * ldu + k] * Y[i * ldy + j];
        }
        __syncthreads();
    }
    for (int e = tid; e < K * nc; e += ST) {
        const int i = e / nc, j = e - (e / nc) * nc;
        Y[i * ldy + j] *= invd[i];
    }
    __syncthreads();
}

// Y <- Y R^-1 for the nr x K block Y: column-oriented solve of Z R = Y with
// deferred scaling. One barrier per column; all threads call.
__device__ void trsm_r(const double *U, int ldu, const double *invd, double *Y, int ldy, int nr, int K) {
    const int tid = threadIdx.x;
    for (int j = 0; j + 1 < K; ++j) {
        const int w = K - 1 - j, cnt = nr * w;
        for (int e = tid; e < cnt; e += ST) {
            const int r = e / w, l = j + 1 + (e - (e / w) * w);
            Y[r * ldy + l] -= Y[r * ldy + j] * U[j * ldu + l];
        }
        __syncthreads();
    }
    for (int e = tid; e < nr * K; e += ST) {
        const int r = e / K, j = e - (e / K) * K;
        Y[r * ldy + j] *= invd[j];
    }
    __syncthreads();
}

// O = op(A) op(B) for K x K operands (op = transpose when the flag is set).
// With sym, only the upper triangle is computed and mirrored. Ends with a barrier.
__device__ void gemm_kk(double *O, const double *A, bool tA, const double *B, bool tB, int K, int lds, bool sym) {
    const int tid = threadIdx.x;
    const int cnt = sym ? tri_count(K) : K * K;
    for (int e = tid; e < cnt; e += ST) {
        int i, j;
        if (sym) {
            if (!tri_pair(e, K, i, j)) continue;
        } else {
            i = e / K;
            j = e - i * K;
        }
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += (tA ? A[k * lds + i] : A[i * lds + k]) * (tB ? B[j * lds + k] : B[k * lds + j]);
        O[i * lds + j] = s;
        if (sym) O[j * lds + i] = s;
    }
    __syncthreads();
}

// Triangular solve in one warp, column-oriented; lane k holds entries k and
// k + 32 of the right-hand side (K <= 64). R is upper, given by its rows, and
// invd = 1 / diag(R). forward = true solves R^T x = x, else R x = x.
__device__ void warp_trsv(const double *R, int lds, const double *invd, double &x0, double &x1, int K, bool forward) {
    const int lane = threadIdx.x & 31;
    for (int s = 0; s < K; ++s) {
        const int i = forward ? s : K - 1 - s;
        const double own = (i >> 5) ? x1 : x0;
        const double xi = __shfl_sync(0xffffffffu, own, i & 31) * invd[i];
        if (lane == (i & 31)) {
            if (i >> 5) x1 = xi;
            else x0 = xi;
        }
        if (forward) {  // x_k -= R[i][k] x_i for k > i
            if (lane > i && lane < K) x0 -= R[i * lds + lane] * xi;
            if (lane + 32 > i && lane + 32 < K) x1 -= R[i * lds + lane + 32] * xi;
        } else {  // x_k -= R[k][i] x_i for k < i
            if (lane < i) x0 -= R[lane * lds + i] * xi;
            if (lane + 32 < i) x1 -= R[(lane + 32) * lds + i] * xi;
        }
    }
}

// ------------------------------------------------------------ Jacobi
// Rotation (c, s) that zeroes a_pq of [[a_pp, a_pq], [a_pq, a_qq]]: tan(phi)
// by the classical formula in FP32, from the FP64 difference a_qq - a_pp.
// For the FP64 sweeps the FP32 pair is renormalised in FP64 with the series
// 1/sqrt(1 + d) = 1 - d/2 + 3d^2/8 (|d| < 1e-6), so the rotation is orthogonal
// to FP64 accuracy; an angle accurate to FP32 still shrinks a_pq by ~1e-7 per
// visit, which is what the FP64 sweeps (started near diagonal) need.
__device__ __forceinline__ void rot_from(float th, float &c0, float &s0) {
    const float t = (th >= 0.0f ? 1.0f : -1.0f) / (fabsf(th) + sqrtf(fmaf(th, th, 1.0f)));
    c0 = rsqrtf(fmaf(t, t, 1.0f));
    s0 = t * c0;
}
__device__ __forceinline__ void rot_angle(float app, float aqq, float apq, float &c, float &s) {
    rot_from((aqq - app) / (2.0f * apq), c, s);
}
__device__ __forceinline__ void rot_angle(double app, double aqq, double apq, double &c, double &s) {
    float c0, s0;
    rot_from((float)(aqq - app) / (2.0f * (float)apq), c0, s0);
    const double cd = c0, sd = s0;
    const double dl = fma(cd, cd, sd * sd) - 1.0;
    const double r = fma(dl, fma(0.375, dl, -0.5), 1.0);
    c = cd * r;
    s = sd * r;
}

template <typename T>
struct JacobiShared {
    T c[2][32], s[2][32];
    int any[2];
};

// Cyclic two-sided Jacobi on the symmetric Kp x Kp matrix A (rows/columns
// beyond K are zero padding) with eigenvector accumulation W <- W J (W may be
// null) and the rotations applied to one vector v <- J^T v (v may be null).
// Each round of the round-robin ordering rotates Kp/2 disjoint pairs: warp 0
// decides and computes the rotations and rotates v, then all threads update
// the 2x2 blocks (pair i rows, pair j columns) of the upper block triangle
// from their old values and mirror them, and the rows of W. A pair rotates
// while |a_pq| > rel sqrt(|a_pp a_qq|) and |a_pq| > rel_abs max_i |a_ii|; the
// sweeps stop when a parallel scan after a sweep finds no such pair, or after
// max_sweeps. The rotation buffers alternate between rounds, so a round costs
// one barrier when it rotates nothing and two otherwise. All threads call.
template <typename T>
__device__ void jacobi(T *A, int lda, T *W, int ldw, T *v, int K, int Kp, int max_sweeps, float rel, float rel_abs,
                       JacobiShared<T> &sh, float *redf) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int half = Kp / 2;
    float dm = 0.0f;
    for (int i = tid; i < K; i += ST) dm = fmaxf(dm, fabsf((float)A[i * lda + i]));
    dm = warp_maxf(dm);
    if (lane == 0) redf[wid] = dm;
    __syncthreads();
    dm = 0.0f;
    for (int w = 0; w < NW; ++w) dm = fmaxf(dm, redf[w]);
    const float floor_abs = rel_abs * dm;
    int buf = 0;
    const int nblk = tri_count(half);
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        for (int round = 0; round < Kp - 1; ++round, buf ^= 1) {
            if (wid == 0) {
                T c = 1, s = 0;
                bool rot = false;
                if (lane < half) {
                    const int pl = rr_player(lane, round, Kp), ql = rr_player(Kp - 1 - lane, round, Kp);
                    if (pl < K && ql < K) {
                        const T apq = A[pl * lda + ql], app = A[pl * lda + pl], aqq = A[ql * lda + ql];
                        const float fpq = fabsf((float)apq);
                        rot = fpq > rel * sqrtf(fabsf((float)app * (float)aqq)) && fpq > floor_abs && fpq > 1e-35f;
                        if (rot) rot_angle(app, aqq, apq, c, s);
                        if (rot && v) {
                            const T vp = v[pl], vq = v[ql];
                            v[pl] = c * vp - s * vq;
                            v[ql] = s * vp + c * vq;
                        }
                    }
                    sh.c[buf][lane] = c;
                    sh.s[buf][lane] = rot ? s : (T)0;
                }
                const int any = __any_sync(0xffffffffu, rot);
                if (lane == 0) sh.any[buf] = any;
            }
            __syncthreads();
            if (!sh.any[buf]) continue;
            for (int e = tid; e < nblk; e += ST) {
                int bi, bj;
                if (!tri_pair(e, half, bi, bj)) continue;
                const T ci = sh.c[buf][bi], si = sh.s[buf][bi], cj = sh.c[buf][bj], sj = sh.s[buf][bj];
                if (si == (T)0 && sj == (T)0) continue;
                const int pi = rr_player(bi, round, Kp), qi = rr_player(Kp - 1 - bi, round, Kp);
                const int pj = rr_player(bj, round, Kp), qj = rr_player(Kp - 1 - bj, round, Kp);
                const T a = A[pi * lda + pj], b = A[pi * lda + qj], cc = A[qi * lda + pj], d = A[qi * lda + qj];
                const T a1 = ci * a - si * cc, b1 = ci * b - si * d, c1 = si * a + ci * cc, d1 = si * b + ci * d;
                const T na = cj * a1 - sj * b1, nb = sj * a1 + cj * b1, nd = sj * c1 + cj * d1;
                const T nc = (bi == bj) ? nb : cj * c1 - sj * d1;  // exact symmetry of a diagonal block
                A[pi * lda + pj] = na;
                A[pi * lda + qj] = nb;
                A[qi * lda + pj] = nc;
                A[qi * lda + qj] = nd;
                if (bi != bj) {
                    A[pj * lda + pi] = na;
                    A[qj * lda + pi] = nb;
                    A[pj * lda + qi] = nc;
                    A[qj * lda + qi] = nd;
                }
            }
            if (W) {
                for (int e = tid; e < Kp * half; e += ST) {  // W <- W J on the columns of each pair
                    const int r = e / half, j = e - (e / half) * half;
                    const T s = sh.s[buf][j];
                    if (s == (T)0) continue;
                    const T c = sh.c[buf][j];
                    const int pl = rr_player(j, round, Kp), ql = rr_player(Kp - 1 - j, round, Kp);
                    const T wp = W[r * ldw + pl], wq = W[r * ldw + ql];
                    W[r * ldw + pl] = c * wp - s * wq;
                    W[r * ldw + ql] = s * wp + c * wq;
                }
            }
            __syncthreads();
        }
        // does any pair still exceed the rotation threshold?
        int more = 0;
        for (int e = tid; e < K * K; e += ST) {
            const int p = e / K, q = e - (e / K) * K;
            if (q <= p) continue;
            const float fpq = fabsf((float)A[p * lda + q]);
            if (fpq > rel * sqrtf(fabsf((float)A[p * lda + p] * (float)A[q * lda + q])) && fpq > floor_abs &&
                fpq > 1e-35f)
                more = 1;
        }
        if (!__syncthreads_or(more)) break;
    }
}

__device__ __forceinline__ void jw_bar() { asm volatile("bar.sync 1, %0;" ::"r"(JW * 32) : "memory"); }

// The partner of column l in round r of the round-robin ordering of Kp
// (even, <= 32) columns; columns l >= Kp pair with themselves.
__device__ __forceinline__ int rr_partner(int l, int r, int Kp) {
    if (l >= Kp) return l;
    int pos = 0;
    if (l > 0) {
        pos = (l - 1 - r) % (Kp - 1);
        if (pos < 0) pos += Kp - 1;
        pos += 1;
    }
    return rr_player(Kp - 1 - pos, r, Kp);
}

// FP32 one-sided (Hestenes) Jacobi in registers, K <= 32, by warps 0..JW-1:
// lane i of every warp holds column i of the symmetric positive semi-definite
// C and of the accumulated rotation V, warp w the rows [w RW, (w + 1) RW). In
// each round of the round-robin ordering (partners from the table ptab) a lane
// takes its partner's entries by shuffles; the warps' partial dot products and
// squared norms are summed through shared memory in a fixed order (one named
// barrier per round, the buffer alternating between rounds), so every warp,
// and both lanes of a pair, take the same rotation from the same numbers, and
// each lane updates its own column (lower index p: c x_p - s x_q, higher q:
// s x_p + c x_q). At convergence the columns of C V are orthogonal, so V
// diagonalises C^2 and therefore C. The warm start needs eigenvectors to FP32
// accuracy only; V is written to X (FP64, K x K).
__device__ void jacobi1_warps(const double *C, int lds, int K, double *X, int max_sweeps, float tol,
                              float2 (*xch)[JW][32], const unsigned char (*ptab)[32]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float a[RW], v[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const int k = w * RW + r;
        a[r] = (lane < K && k < K) ? (float)C[k * lds + lane] : 0.0f;
        v[r] = (k == lane && lane < K) ? 1.0f : 0.0f;
    }
    const int Kp = K + (K & 1);
    // pairs whose dot product is below floor_g (set by ||C||_F^2, invariant under the
    // rotations) are left alone: their directions carry eigenvalues too small for FP32
    // to resolve, and the FP64 stage handles them
    float f2 = 0.0f;
#pragma unroll
    for (int r = 0; r < RW; ++r) f2 = fmaf(a[r], a[r], f2);
    f2 = warp_sumf(f2);
    xch[1][w][lane] = make_float2(f2, 0.0f);
    jw_bar();
    float f2t = 0.0f;
    for (int u = 0; u < JW; ++u) f2t += xch[1][u][lane].x;
    const float floor_g = 1e-14f * f2t, tol2 = tol * tol;
    int buf = 0;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        bool any = false;
        for (int round = 0; round < Kp - 1; ++round, buf ^= 1) {
            const int partner = ptab[round][lane];
            const int src = partner < 32 ? partner : lane;
            float pa[RW];
            float g = 0.0f, nrm = 0.0f;
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                pa[r] = __shfl_sync(0xffffffffu, a[r], src);
                g = fmaf(a[r], pa[r], g);
                nrm = fmaf(a[r], a[r], nrm);
            }
            xch[buf][w][lane] = make_float2(g, nrm);
            jw_bar();
            g = 0.0f;
            nrm = 0.0f;
#pragma unroll
            for (int u = 0; u < JW; ++u) {
                const float2 t = xch[buf][u][lane];
                g += t.x;
                nrm += t.y;
            }
            const float pn = __shfl_sync(0xffffffffu, nrm, src);
            const bool low = lane < partner;
            const float alpha = low ? nrm : pn, beta = low ? pn : nrm;  // norms^2 of the lower, higher column
            const bool rot = lane < K && partner < K && g * g > tol2 * (alpha * beta) && fabsf(g) > floor_g &&
                             fabsf(g) > 1e-30f;
            float c = 1.0f, sp = 0.0f;  // own' = c own + sp partner
            if (rot) {
                // tangent of the rotation angle: 2 g sign(d) / (|d| + sqrt(d^2 + 4 g^2)), d = beta - alpha
                const float dd = beta - alpha, g2 = 2.0f * g;
                const float r2 = fmaf(dd, dd, g2 * g2);
                const float t = __fdividef(dd >= 0.0f ? g2 : -g2, fabsf(dd) + r2 * rsqrtf(r2));
                c = rsqrtf(fmaf(t, t, 1.0f));
                sp = low ? -t * c : t * c;
                any = true;
            }
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                const float pv = __shfl_sync(0xffffffffu, v[r], src);
                a[r] = fmaf(sp, pa[r], c * a[r]);
                v[r] = fmaf(sp, pv, c * v[r]);
            }
        }
        if (!__any_sync(0xffffffffu, any)) break;  // the same decision in every warp
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const int k = w * RW + r;
        if (lane < K && k < K) X[k * lds + lane] = (double)v[r];
    }
}

// ------------------------------------------------------------ lambda functions
struct Spec {
    int K;
    double rho, rho0sq;
    const double *theta, *c2;
};
// FP32 copies of theta, 1 - theta and c2 (scaled by 1 / sum c2) for the scans
struct SpecF {
    int K;
    const float *th, *a, *c2;
};

// per-lane terms (lanes stride over i) of the lam-functions and their
// mu-derivatives: s[0] = N = sum c2 g^2, s[1] = N', s[2] = N'', s[3] = D = sum g,
// s[4] = D', s[5] = D'' with g_i = mu a_i / d_i = 1 - f_i, a_i = 1 - theta_i,
// d_i = theta_i + mu a_i.
template <typename R, typename SP>
__device__ __forceinline__ void lam_terms6(const SP &S, R mu, R s[6]) {
    for (int k = 0; k < 6; ++k) s[k] = R(0);
    for (int i = threadIdx.x & 31; i < S.K; i += 32) {
        R th, a, c;
        if constexpr (sizeof(R) == 8) {
            th = S.theta[i];
            a = 1.0 - th;
            c = S.c2[i];
        } else {
            th = S.th[i];
            a = S.a[i];
            c = S.c2[i];
        }
        const R d = th + mu * a;
        if (!(d > R(0))) {
            s[3] += R(1);
            continue;
        }
        const R inv = R(1) / d;
        const R g = mu * a * inv, g1 = a * th * inv * inv, g2 = R(-2) * a * g1 * inv;
        s[0] += c * g * g;
        s[1] += R(2) * c * g * g1;
        s[2] += R(2) * c * (g1 * g1 + g * g2);
        s[3] += g;
        s[4] += g1;
        s[5] += g2;
    }
}
// N and N' only (DP)
template <typename R, typename SP>
__device__ __forceinline__ void lam_terms_n(const SP &S, R mu, R &N, R &N1) {
    N = R(0);
    N1 = R(0);
    for (int i = threadIdx.x & 31; i < S.K; i += 32) {
        R th, a, c;
        if constexpr (sizeof(R) == 8) {
            th = S.theta[i];
            a = 1.0 - th;
            c = S.c2[i];
        } else {
            th = S.th[i];
            a = S.a[i];
            c = S.c2[i];
        }
        const R d = th + mu * a;
        if (!(d > R(0))) continue;
        const R inv = R(1) / d;
        const R g = mu * a * inv, g1 = a * th * inv * inv;
        N += c * g * g;
        N1 += R(2) * c * g * g1;
    }
}
// N and D only (GCV values)
__device__ __forceinline__ void lam_terms_nd(const Spec &S, double mu, double &N, double &D) {
    N = 0.0;
    D = 0.0;
    for (int i = threadIdx.x & 31; i < S.K; i += 32) {
        const double th = S.theta[i], a = 1.0 - th, d = th + mu * a;
        const double g = d > 0.0 ? mu * a / d : 1.0;
        N += S.c2[i] * g * g;
        D += g;
    }
}
__device__ __forceinline__ double gcv_value(double N, double D) {
    const double g = N / (D * D);
    return g == g ? g : DBL_MAX;
}
// one thread's FP32 grid value: GCV (N / D^2) or the DP function N - delta
__device__ __forceinline__ void grid_nd(const SpecF &S, float mu, float &N, float &D) {
    N = 0.0f;
    D = 0.0f;
    for (int i = 0; i < S.K; ++i) {
        const float ai = S.a[i], d = fmaf(mu, ai, S.th[i]);
        const float gg = d > 0.0f ? __fdividef(mu * ai, d) : 1.0f;
        N = fmaf(S.c2[i] * gg, gg, N);
        D += gg;
    }
}
template <typename R>
__device__ __forceinline__ R warp_sum_t(R v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// first and second derivative of G = N / D^2 with respect to t = log10(lam)
template <typename R>
__device__ __forceinline__ void gcv_dt(const R s[6], R mu, R &d1, R &d2) {
    const R N = s[0], N1 = s[1], N2 = s[2], D = s[3], D1 = s[4], D2 = s[5];
    const R iD = R(1) / D, iD2 = iD * iD;
    const R G1 = N1 * iD2 - R(2) * N * D1 * iD2 * iD;
    const R G2 = N2 * iD2 - R(4) * N1 * D1 * iD2 * iD - R(2) * N * D2 * iD2 * iD + R(6) * N * D1 * D1 * iD2 * iD2;
    const R ln10 = R(LN10);
    d1 = G1 * mu * ln10;
    d2 = (G2 * mu * mu + G1 * mu) * ln10 * ln10;
}

// size of the two terms whose difference is dG/dt: |dG/dt| below a small
// multiple of it is rounding noise
template <typename R>
__device__ __forceinline__ R gcv_dt_scale(const R s[6], R mu) {
    const R iD = R(1) / s[3];
    return (fabs(s[1]) + fabs(R(2) * s[0] * s[4] * iD)) * iD * iD * mu * R(LN10);
}

// safeguarded Newton step for a root of an increasing function f (f1 = f')
// inside [A, B], which the sign of f shrinks
template <typename R>
__device__ __forceinline__ R newton_step(R t, R f, R f1, R &A, R &B) {
    if (f > R(0)) B = t;
    else if (f < R(0)) A = t;
    R tn = (f1 > R(0)) ? t - f / f1 : R(0.5) * (A + B);
    if (!(tn > A && tn < B)) tn = R(0.5) * (A + B);
    return tn;
}

}  // namespace

__global__ void __launch_bounds__(ST, 1) k_small_solve(SmallArgs a) {
    extern __shared__ double sm[];
    __shared__ double s_rho, s_rho0sq, s_t, s_scale;
    __shared__ double s_grid[GRID_POINTS];
    __shared__ float s_redf[NW];
    __shared__ int s_fail, s_flag, s_idx[NW], s_end[4];
    __shared__ JacobiShared<float> jf;
    __shared__ JacobiShared<double> jd;
    __shared__ float2 s_xch[2][JW][32];
    __shared__ unsigned char s_ptab[31][32];
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
    if (Kp <= 32)  // partners of the FP32 Jacobi rounds
        for (int e = tid; e < (Kp - 1) * 32; e += ST) s_ptab[e >> 5][e & 31] = (unsigned char)rr_partner(e & 31, e >> 5, Kp);
    const int lds = (ld + 1) | 1;  // FP64 leading dimension: odd, >= Kp and >= K + 1
    const int ldf = ld + 3;        // FP32 leading dimension
    double *Rm = sm;               // Cholesky rows of M = G_A + rho G_L (kept for z)
    double *Cm = Rm + lds * lds;   // [G_A | g] -> [R^-T G_A | h] -> C = R^-T G_A R^-1 (kept for z)
    double *Um = Cm + lds * lds;   // R rows over their diagonal; then X^T C X; then C + mu (I - C)
    double *Xm = Um + lds * lds;   // eigenvector estimate
    double *Tm = Xm + lds * lds;   // scratch (FP32 Jacobi matrix first)
    double *Em = Tm + lds * lds;   // scratch (FP32 eigenvectors first)
    double *vec = Em + lds * lds;
    double *theta = vec, *gh = vec + lds, *c2 = vec + 2 * lds, *invd = vec + 3 * lds, *hv = vec + 4 * lds;
    float *fvec = reinterpret_cast<float *>(vec + 5 * lds);  // 3 x lds floats within 2 x lds doubles
    float *thf = fvec, *af = fvec + lds, *c2f = fvec + 2 * lds;
    float *Af = reinterpret_cast<float *>(Tm);
    float *Wf = reinterpret_cast<float *>(Em);
    const double *GA = a.GA + (long long)b * ld * ld;
    const double *GL = a.GL + (long long)b * ld * ld;
    const double *g = a.g + (long long)b * ld;
#define AT(P, i, j) P[(i) * lds + (j)]
#define AF(P, i, j) P[(i) * ldf + (j)]

    // ---------------------------------------------- 1. Cholesky of M, C and h (FP64)
    if (wid == 0) {
        double tA = 0.0, tL = 0.0;
        for (int i = lane; i < K; i += 32) {
            tA += GA[i * ld + i];
            tL += GL[i * ld + i];
        }
        warp_sum2(tA, tL);
        if (lane == 0) {
            s_rho = (tA > 0.0 && tL > 0.0) ? tA / tL : 1.0;
            s_fail = 0;
            s_flag = 0;
        }
    }
    __syncthreads();
    const double rho = s_rho;
    for (int e = tid; e < K * K; e += ST) {
        const int i = e / K, j = e - (e / K) * K;
        const double ga = GA[i * ld + j];
        AT(Cm, i, j) = ga;
        AT(Rm, i, j) = ga + rho * GL[i * ld + j];
    }
    for (int i = tid; i < K; i += ST) AT(Cm, i, K) = g[i];
    __syncthreads();
    chol_upper(Rm, lds, K, invd, &s_fail);
    if (s_fail) {
        if (tid == 0) {
            atomicOr(a.err, 1);
            a.lam[b] = 0.0;
            a.flag[b] = 0;
        }
        return;
    }
    for (int e = tid; e < K * K; e += ST) {
        const int i = e / K, k = e - (e / K) * K;
        if (k > i) AT(Um, i, k) = AT(Rm, i, k) * invd[i];
    }
    __syncthreads();
    trsm_rt(Um, lds, invd, Cm, lds, K, K + 1);  // [G_A | g] <- R^-T [G_A | g]
    for (int i = tid; i < K; i += ST) hv[i] = AT(Cm, i, K);
    trsm_r(Um, lds, invd, Cm, lds, K, K);  // C = (R^-T G_A) R^-1
    for (int e = tid; e < K * K; e += ST) {  // exact symmetry
        const int i = e / K, j = e - (e / K) * K;
        if (j > i) {
            const double s = 0.5 * (AT(Cm, i, j) + AT(Cm, j, i));
            AT(Cm, i, j) = s;
            AT(Cm, j, i) = s;
        }
    }
    __syncthreads();

    double lam = a.lam_fixed;
    if (a.rule != MOF_RULE_FIXED) {
        // ------------------------------------------ 2a. FP32 Jacobi on C
        if (K <= 32) {  // registers only
            if (wid < JW) jacobi1_warps(Cm, lds, K, Xm, JACOBI32_MAX_SWEEPS, 1e-6f, s_xch, s_ptab);
            __syncthreads();
        } else {
            for (int e = tid; e < Kp * Kp; e += ST) {
                const int i = e / Kp, j = e - (e / Kp) * Kp;
                AF(Af, i, j) = (i < K && j < K) ? (float)AT(Cm, i, j) : 0.0f;
                AF(Wf, i, j) = i == j ? 1.0f : 0.0f;
            }
            __syncthreads();
            jacobi<float>(Af, ldf, Wf, ldf, (float *)nullptr, K, Kp, JACOBI32_MAX_SWEEPS, 1e-6f, 1e-7f, jf, s_redf);
            for (int e = tid; e < K * K; e += ST) {
                const int i = e / K, j = e - (e / K) * K;
                AT(Xm, i, j) = (double)AF(Wf, i, j);
            }
            __syncthreads();
        }

        // ------------------------------------------ 2b. FP64: orthonormalise, congruence
        gemm_kk(Tm, Xm, true, Xm, false, K, lds, true);  // X0^T X0 (the FP32 matrix is done with)
        for (int i = tid; i < K; i += ST) AT(Tm, i, i) -= 1.0;  // E = X0^T X0 - I
        __syncthreads();
        gemm_kk(Em, Tm, false, Tm, false, K, lds, true);  // E^2 (the FP32 eigenvectors are in Xm)
        for (int e = tid; e < K * K; e += ST) {           // P = I - E/2 + 3 E^2/8
            const int i = e / K, j = e - (e / K) * K;
            AT(Em, i, j) = (i == j ? 1.0 : 0.0) - 0.5 * AT(Tm, i, j) + 0.375 * AT(Em, i, j);
        }
        __syncthreads();
        gemm_kk(Tm, Xm, false, Em, false, K, lds, false);  // X = X0 P
        for (int e = tid; e < K * K; e += ST) {
            const int i = e / K, j = e - (e / K) * K;
            AT(Xm, i, j) = AT(Tm, i, j);
        }
        __syncthreads();
        gemm_kk(Tm, Cm, false, Xm, false, K, lds, false);  // T = C X
        gemm_kk(Um, Xm, true, Tm, false, K, lds, true);    // X^T C X
        for (int i = tid; i < Kp; i += ST) {               // gh = X^T h; zero padding of an odd size
            double s = 0.0;
            if (i < K)
                for (int k = 0; k < K; ++k) s += AT(Xm, k, i) * hv[k];
            gh[i] = s;
            if (K & 1) {
                AT(Um, i, K) = 0.0;
                AT(Um, K, i) = 0.0;
            }
        }
        __syncthreads();

        // ------------------------------------------ 2c. FP64 Jacobi polish
        jacobi<double>(Um, lds, (double *)nullptr, lds, gh, K, Kp, JACOBI64_MAX_SWEEPS, 1e-16f, 1e-12f, jd, s_redf);
        for (int i = tid; i < K; i += ST) {
            theta[i] = fmin(fmax(AT(Um, i, i), 0.0), 1.0);
            c2[i] = theta[i] > THETA_TINY ? gh[i] * gh[i] / theta[i] : 0.0;
        }
        __syncthreads();

        // ------------------------------------------ 3-4. lambda
        if (wid == 0) {
            double kept = 0.0, unused = 0.0;
            for (int i = lane; i < K; i += 32) kept += c2[i];
            warp_sum2(kept, unused);
            if (lane == 0) {
                s_rho0sq = a.bb[b] - kept;
                s_scale = kept > 0.0 ? 1.0 / kept : 1.0;
            }
        }
        __syncthreads();
        for (int i = tid; i < K; i += ST) {
            thf[i] = (float)theta[i];
            af[i] = (float)(1.0 - theta[i]);
            c2f[i] = (float)(c2[i] * s_scale);
        }
        __syncthreads();
        const Spec S{K, rho, s_rho0sq, theta, c2};
        const SpecF SF{K, thf, af, c2f};
        const double lrho = log10(rho);
        const double lo = lrho - BRACKET_DECADES, hi = lrho + BRACKET_DECADES;
        const double step = (hi - lo) / (GRID_POINTS - 1);
        if (a.rule == MOF_RULE_GCV) {
            // GCV at every grid point in FP64 and its first minimum (ties to the smaller
            // lambda), as the grid search defines it; a scan in lower precision can pick another
            // of two nearly equal minima. One thread per point, its terms summed in order: a
            // warp's FP64 instruction occupies the pipe as long with one active lane as with 32,
            // so lanes over points take far fewer FP64 instructions than lanes over the terms
            // with a reduction (and one exp10 per point instead of one per lane)
            for (int gi = tid; gi < GRID_POINTS; gi += ST) {
                const double mu = exp10(lo + gi * step) / rho;
                double N = 0.0, D = 0.0;
                for (int i = 0; i < S.K; ++i) {
                    const double th = S.theta[i], am = 1.0 - th, d = th + mu * am;
                    const double g = d > 0.0 ? mu * am / d : 1.0;
                    N += S.c2[i] * g * g;
                    D += g;
                }
                s_grid[gi] = gcv_value(N, D);
            }
            __syncthreads();
            if (wid == 0) {
                double bv = DBL_MAX;
                int ig = GRID_POINTS;
                for (int gi = lane; gi < GRID_POINTS; gi += 32)
                    if (s_grid[gi] < bv) {
                        bv = s_grid[gi];
                        ig = gi;
                    }
                for (int o = 16; o > 0; o >>= 1) {
                    const double bo = __shfl_xor_sync(0xffffffffu, bv, o);
                    const int io = __shfl_xor_sync(0xffffffffu, ig, o);
                    if (bo < bv || (bo == bv && io < ig)) {
                        bv = bo;
                        ig = io;
                    }
                }
                if (ig >= GRID_POINTS) ig = 0;
                bv = s_grid[ig];
                double vmax = bv;  // the flatness test over the NREF points around the minimum
                for (int w = -(NREF / 2); w <= NREF / 2; ++w) vmax = fmax(vmax, s_grid[min(max(ig + w, 0), GRID_POINTS - 1)]);
                const bool flat = vmax - bv <= 1e-13 * bv;
                // safeguarded Newton on dG/dt = 0 inside [t_{i-1}, t_{i+1}]: FP32 steps
                // (in t - log10 rho) to a starting point, then FP64 steps on the full cell pair
                const double A0 = lo + max(ig - 1, 0) * step, B0 = lo + min(ig + 1, GRID_POINTS - 1) * step;
                float tf = (float)(ig * step - BRACKET_DECADES);
                float Af0 = (float)(A0 - lrho), Bf0 = (float)(B0 - lrho);
                for (int it = 0; it < (flat ? 0 : NEWTON32_MAX); ++it) {
                    float s[6], d1, d2;
                    const float mu = exp10f(tf);
                    lam_terms6<float>(SF, mu, s);
                    for (int k = 0; k < 6; ++k) s[k] = warp_sum_t(s[k]);
                    gcv_dt<float>(s, mu, d1, d2);
                    if (d1 == 0.0f || !(d1 == d1)) break;
                    if (fabsf(d1) <= 1e-5f * gcv_dt_scale<float>(s, mu)) break;  // at the rounding level
                    const float tn = newton_step<float>(tf, d1, d2, Af0, Bf0);
                    const float dt = fabsf(tn - tf);
                    tf = tn;
                    if (dt <= 1e-6f || Bf0 - Af0 <= 1e-6f) break;
                }
                double t = lrho + (double)tf, A1 = A0, B1 = B0;
                if (!(t > A1 && t < B1)) t = lo + ig * step;
                for (int it = 0; it < (flat ? 0 : NEWTON_MAX); ++it) {
                    double s6[6], d1, d2;
                    const double mu = exp10(t) / rho;
                    lam_terms6<double>(S, mu, s6);
                    warp_sum6(s6);
                    gcv_dt<double>(s6, mu, d1, d2);
                    if (d1 == 0.0) break;
                    if (fabs(d1) <= 1e-12 * gcv_dt_scale<double>(s6, mu)) break;  // at the rounding level
                    const bool pure = d2 > 0.0 && t - d1 / d2 > A1 && t - d1 / d2 < B1;
                    const double tn = newton_step<double>(t, d1, d2, A1, B1);
                    const double dt = fabs(tn - t);
                    t = tn;
                    if (dt <= 1e-10 * fmax(1.0, fabs(t)) || B1 - A1 <= 1e-10 * fmax(1.0, fabs(t))) break;
                    if (pure && dt <= 1e-6 * fmax(1.0, fabs(t))) break;  // quadratic: the next step is ~1e-12
                }
                if (flat) {
                    t = lo + ig * step;
                } else {
                    double N, D;
                    lam_terms_nd(S, exp10(t) / rho, N, D);
                    warp_sum2(N, D);
                    if (gcv_value(N, D) > bv) t = lo + ig * step;
                }
                if (lane == 0) s_t = t;
            }
            __syncthreads();
        } else {  // DP on F(t) = N(mu(t)) + rho0^2 - (eta delta)^2, increasing in t
            if (wid < 2) {  // the bracket ends, in FP64
                double N, N1;
                lam_terms_n<double>(S, exp10(wid ? hi : lo) / rho, N, N1);
                warp_sum2(N, N1);
                const double F = N + S.rho0sq - a.target2;
                if (lane == 0) s_end[wid] = wid ? (F <= 0.0) : (F >= 0.0);
            }
            __syncthreads();
            const int flag = s_end[0] ? 1 : (s_end[1] ? 2 : 0);
            if (flag == 0) {
                const float delta = (float)((a.target2 - S.rho0sq) * s_scale);
                // FP32 grid: the first point with F >= 0
                int first = GRID_POINTS;
                if (tid < GRID_POINTS) {
                    float N, D;
                    grid_nd(SF, exp10f((float)(-BRACKET_DECADES + tid * step)), N, D);
                    if (N - delta >= 0.0f) first = tid;
                }
                for (int o = 16; o > 0; o >>= 1) first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
                if (lane == 0) s_idx[wid] = first;
                __syncthreads();
                int k = GRID_POINTS;
                for (int w = 0; w < NW; ++w) k = min(k, s_idx[w]);
                // the sign change within (t_{k-2}, t_{k+1}), confirmed in FP64
                const double A1 = lo + max(k - 2, 0) * step, B1 = lo + min(k + 1, GRID_POINTS - 1) * step;
                if (wid < 2) {
                    double N, N1;
                    lam_terms_n<double>(S, exp10(wid ? B1 : A1) / rho, N, N1);
                    warp_sum2(N, N1);
                    const double F = N + S.rho0sq - a.target2;
                    if (lane == 0) s_end[2 + wid] = wid ? (F > 0.0) : (F < 0.0);
                }
                __syncthreads();
                if (wid == 0) {
                    const bool cell = s_end[2] && s_end[3];
                    double A0 = cell ? A1 : lo, B0 = cell ? B1 : hi;
                    float tf = (float)(0.5 * (A0 + B0) - lrho), Af0 = (float)(A0 - lrho), Bf0 = (float)(B0 - lrho);
                    for (int it = 0; it < NEWTON32_MAX; ++it) {
                        float N, N1;
                        const float mu = exp10f(tf);
                        lam_terms_n<float>(SF, mu, N, N1);
                        N = warp_sum_t(N);
                        N1 = warp_sum_t(N1);
                        const float tn = newton_step<float>(tf, N - delta, N1 * mu * (float)LN10, Af0, Bf0);
                        const float dt = fabsf(tn - tf);
                        tf = tn;
                        if (dt <= 1e-6f || Bf0 - Af0 <= 1e-6f) break;
                    }
                    double t = lrho + (double)tf;
                    if (!(t > A0 && t < B0)) t = 0.5 * (A0 + B0);
                    for (int it = 0; it < NEWTON_MAX; ++it) {
                        const double mu = exp10(t) / rho;
                        double N, N1;
                        lam_terms_n<double>(S, mu, N, N1);
                        warp_sum2(N, N1);
                        const double tn = newton_step<double>(t, N + S.rho0sq - a.target2, N1 * mu * LN10, A0, B0);
                        const double dt = fabs(tn - t);
                        t = tn;
                        if (dt <= 1e-15 * fmax(1.0, fabs(t)) || B0 - A0 <= 1e-15 * fmax(1.0, fabs(t))) break;
                    }
                    if (lane == 0) s_t = t;
                }
            } else if (tid == 0) {
                s_t = flag == 1 ? lo : hi;
            }
            if (tid == 0) s_flag = flag;
            __syncthreads();
        }
        lam = exp10(s_t);
    }
    const double mu = lam / rho;

    // ---------------------------------------------- 5. z = R^-1 (C + mu (I - C))^-1 h
    // (G_A + lam G_L = R^T (C + mu (I - C)) R and g = R^T h)
    for (int e = tid; e < K * K; e += ST) {
        const int i = e / K, j = e - (e / K) * K;
        if (j >= i) AT(Um, i, j) = (1.0 - mu) * AT(Cm, i, j) + (i == j ? mu : 0.0);
    }
    __syncthreads();
    double *invs = gh;  // 1 / diagonal of the Cholesky factor of C + mu (I - C)
    chol_upper(Um, lds, K, invs, &s_fail);
    if (wid == 0) {
        double x0 = lane < K ? hv[lane] : 0.0, x1 = lane + 32 < K ? hv[lane + 32] : 0.0;
        warp_trsv(Um, lds, invs, x0, x1, K, true);   // Rs^T w = h
        warp_trsv(Um, lds, invs, x0, x1, K, false);  // Rs y = w
        warp_trsv(Rm, lds, invd, x0, x1, K, false);  // R z = y
        const bool bad = (lane < K && !isfinite(x0)) || (lane + 32 < K && !isfinite(x1));
        if (lane < K) z[lane] = x0;
        if (lane + 32 < K) z[lane + 32] = x1;
        if (__any_sync(0xffffffffu, bad) || s_fail) {
            if (lane == 0) atomicOr(a.err, 2);
        }
        if (lane == 0) {
            a.lam[b] = lam;
            a.flag[b] = s_flag;
        }
    }
#undef AT
#undef AF
}

static size_t small_smem(int ld) {
    const size_t lds = (size_t)((ld + 1) | 1);
    return sizeof(double) * (6 * lds * lds + 7 * lds);
}

mof_status prepare_small_solve(int ld) {
    // the limit only ever grows: smaller problems launched later still fit (set
    // from the first call on: static and dynamic shared memory together exceed
    // the default 48 KB before the dynamic part alone does)
    static std::atomic<size_t> configured{0};
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
