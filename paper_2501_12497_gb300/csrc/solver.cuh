// Internal interfaces of the Krylov layer and the solver (krylov.cu,
// small.cu, solver.cu).
#pragma once

#include "common.cuh"

namespace mof {

// ------------------------------------------------------ per-problem scratch
// Small buffers of the stand-alone operator entry points, allocated on first
// use and kept until mof_problem_destroy.
enum ScratchKind { SCR_IMAGE = 0, SCR_RADIUS = 1, SCR_DEST = 2, SCR_FLOWROWS = 3, SCR_COUNT = 4 };
mof_status apply_scratch(mof_problem *p, ScratchKind kind, void **out);
void free_workspace(mof_problem *p);

// ------------------------------------------------------------ Krylov bases
template <typename real>
struct BasisRef {
    real *V;          // [B][Kmax][N]
    long long N;      // vector length
    int Kmax;
    int B;            // number of independent problems
    const int *K;     // device [B]: current basis size
    const int *act;   // device [B] or null: problems with act[b] == 0 are skipped
};

// Up to three right-hand vectors of one batched multi-dot.
template <typename real>
struct DotVecs {
    const real *x[3];
    long long stride[3];  // between problems
};
// Output addressing of one dot result i (i < K[b]) of problem b:
//   out[b*bstride + i*istride + col*jstride], col = K[b]-1 if last_col else 0.
struct DotOut {
    double *out;
    long long bstride;
    int istride;
    int jstride;
    int last_col;
    double sign;
};
struct DotOuts {
    DotOut o[3];
};

long long krylov_chunks(long long N);
// doubles of Krylov::partial needed per problem of length N and basis capacity Kmax
long long krylov_partial_doubles(long long N, int Kmax);

template <typename real>
struct Krylov {
    double *partial = nullptr;  // scratch [B][chunks][Kmax] (sized by the owner: krylov_partial_doubles)
    int *err = nullptr;         // device error word (|= 4: a bounded wait ran out), may be null
    double *aux = nullptr;      // scratch [2][B] of append (slot, 1/||x||), sized by the owner
    // out[b][j] = sign * <V[b][j], x[b]>, j < K[b]
    void dots(const BasisRef<real> &B, const real *x, long long xstride, double *out, long long ostride, double sign,
              cudaStream_t st) const;
    // dots of every basis vector with nv (1..3) vectors in one pass over V; exact: error-free
    // accumulation of FP32 products (for Grams whose projected residual cancels)
    void multidot(const BasisRef<real> &B, int nv, const DotVecs<real> &xs, const DotOuts &outs, cudaStream_t st,
                  bool exact = false) const;
    // out[b] = sum_j V[b][j] c[b][j]
    void combine(const BasisRef<real> &B, const double *c, long long cstride, real *out, long long ostride,
                 cudaStream_t st) const;
    // out[b] = sum_j V[b][j] c[b][j] - x[b]; optionally ||out[b]||^2 -> nrm2_out[b]
    void combine_minus(const BasisRef<real> &B, const double *c, long long cstride, const real *x, long long xstride,
                       real *out, long long ostride, double *nrm2_out, cudaStream_t st) const;
    // out[b] = x[b] - sum_j V[b][j] c[b][j]; optionally ||out[b]||^2 -> nrm2_out[b]
    void subtract(const BasisRef<real> &B, const double *c, long long cstride, const real *x, long long xstride, real *out,
                  long long ostride, double *nrm2_out, cudaStream_t st) const;
    void norm2(const real *x, long long N, long long xstride, int nb, double *out, cudaStream_t st,
               bool exact = false) const;
    // x[b] <- (I - V V^T)^2 x[b] (classical Gram-Schmidt twice); ||x||^2 -> nrm2_out
    void reorth(const BasisRef<real> &B, real *x, long long xstride, double *coef, double *nrm2_out, cudaStream_t st) const;
    // the same with the first projection's coefficients V^T x supplied by the caller from an
    // exact identity (c1 [B][Kmax]; null when they are zero, as for a Golub-Kahan residual),
    // so that only the second projection streams V for its dot products
    // kcap (> 0): a bound on every K[b] known to the caller, which sizes the fused pass's
    // shared-memory tile (a larger K[b] sets bit 8 of err)
    void reorth_second(const BasisRef<real> &B, real *x, long long xstride, const double *c1, double *coef,
                       double *nrm2_out, cudaStream_t st, int kcap = 0) const;
    // x[b] <- x[b] - V[b] c[b] and out[b] = V[b]^T x[b] in one pass over V (false: not
    // applicable to this layout, nothing enqueued)
    // nparts (may be null): also the chunk partials of ||x'[b]||^2, after the dot partials in
    // partial (at partial + B.B * nparts * Kmax), their number per problem in *nparts
    bool sub_dot(const BasisRef<real> &B, const double *c, long long cstride, real *x, long long xstride, double *out,
                 cudaStream_t st, int kcap = 0, int *nparts = nullptr) const;
    // x[b] <- x[b] - V[b] c[b], the per-block partials of ||x[b]||^2 left in partial;
    // returns their number per problem (for append_parts)
    int subtract_parts(const BasisRef<real> &B, const double *c, long long cstride, const real *x, long long xstride,
                       real *out, long long ostride, cudaStream_t st) const;
    // reorth_second with the final norm left as partials (returns their number per problem)
    int reorth_second_parts(const BasisRef<real> &B, real *x, long long xstride, const double *c1, double *coef,
                            cudaStream_t st, int kcap = 0) const;
    // append with ||x||^2 summed from the nparts partials of the preceding update (written to
    // nrm2_out), and sqrt(||x||^2) written to sq1 / sq2 (may be null) for problems still growing
    // (parts: where the partials are, default the start of partial)
    void append_parts(const BasisRef<real> &B, int *Kmut, const real *x, long long xstride, int nparts, double *nrm2_out,
                      const double *scale, double tol, int *grow, int *appended, real *stage, double *sq1, double *sq2,
                      cudaStream_t st, const double *parts = nullptr) const;
    // V[b][K[b]] = x[b]/||x[b]||, K[b]++ unless ||x[b]|| <= tol*scale[b] (then grow[b] = 0);
    // scale may be null (only ||x|| > 0 required); stage[b] (may be null) receives the new vector
    void append(const BasisRef<real> &B, int *Kmut, const real *x, long long xstride, const double *nrm2,
                const double *scale, double tol, int *grow, int *appended, real *stage, cudaStream_t st) const;
};

// Solve-OF (p = q = 2) GKS step after the projection coefficients d: the graph Laplacian q of
// the residual x, then one pass over the basis forming x' = x - V d (in x) with the dot
// products that give the new vector's Gram columns, the append decision, the new columns of
// G_A, G_L, g and Mg, and the append of x'/||x'|| (krylov.cu, k_of_proj_gram_pass).
// partial: [B][chunks][3 Kmax + 4] doubles; res: [B][3 Kmax + 4]; q: [B][2 ns] scratch.
long long of_pass_chunks(long long ns, int elem_bytes);
int of_pass_stride(int Kmax);
template <typename real> bool of_pass_applicable(long long ns, const void *V, const void *x);
template <typename real>
mof_status launch_of_proj_gram_pass(const BasisRef<real> &B, int *Kmut, long long ns, int nx, int ny, const double *d, real *x,
                                    real *q, const real *AtB, const real *ux, const real *uy, double *partial,
                                    double *res, int *err, int kcap, const double *scale, double tol, int *grow,
                                    double *GA, double *GL, double *g, double *Mg, double *nrm2_out, int *appended,
                                    double *aux, cudaStream_t st);

// Bound of the device waits on tile copies for the current device (polls; < 0: the
// default); used by mof_debug_set_wait_limit.
mof_status set_wait_polls(long long polls);

// ------------------------------------------------------ small FP64 solver
// One projected problem per block: min ||A V z - b||^2 + lam ||L V z||^2
// given G_A = (AV)^T(AV), G_L = (LV)^T(LV), g = (AV)^T b, bb = ||b||^2.
struct SmallArgs {
    const double *GA;      // [B][ld][ld]
    const double *GL;      // [B][ld][ld]
    const double *g;       // [B][ld]
    const double *bb;      // [B]
    const int *K;          // [B] problem dimension
    const int *active;     // [B] (null = all active); inactive -> z = 0, lam = 0
    int ld;                // leading dimension (Kmax)
    int B;
    int rule;              // MOF_RULE_*
    double target2;        // DP: (eta delta)^2
    double lam_fixed;
    double *lam;           // [B] out
    double *z;             // [B][ld] out
    int *flag;             // [B] out: DP flag
    int *err;              // error word (|= 1: factorisation failed, 2: non-finite)
};
mof_status launch_small_solve(const SmallArgs &a, cudaStream_t st);
// Raise the kernel's dynamic shared-memory limit for leading dimension ld
// (done before any graph capture).
mof_status prepare_small_solve(int ld);

}  // namespace mof
