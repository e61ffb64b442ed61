// Internal declarations of libmof: the problem object, per-angle tables,
// error plumbing and small device helpers shared by the kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "mof.h"

namespace mof {

// ----------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
mof_status fail(mof_status st, const char *fmt, ...);
mof_status cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define MOF_CUDA(call)                                                               \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) return ::mof::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define MOF_TRY(expr)                       \
    do {                                    \
        mof_status s_ = (expr);             \
        if (s_ != MOF_OK) return s_;        \
    } while (0)

// Kernel-launch counter (every launch site calls count_launch()); graph
// replays add the number of kernel nodes they execute.
void count_launch();
void count_launches_add(long long k);
long long launches_so_far();

// Launch-error check after a kernel launch.
#define MOF_LAUNCH_CHECK() MOF_CUDA(cudaGetLastError())

// ------------------------------------------------------- per-angle tables
// Host-computed (FP64) parameters of one projection angle. The FP32
// kernels evaluate affine coordinates base + j * step with the step split
// into a 12-significant-bit head (exact products with |j| < 4096) and a
// tail, so that the fractional interpolation weight keeps ~1e-7 absolute
// accuracy at any grid size (see affine_frac below).
struct AngleParams {
    double c, s;        // cos, sin
    // Ray-driven (Joseph) march, in the frame of the stepping axis:
    //   f(j) = k * f0_k + f0_c + j * df   (fractional index along the fast axis)
    double f0_k;        // d f0 / d bin
    double f0_c;        // constant part
    double df;          // step of f per step index
    float df_hi, df_lo; // split of df
    float wstep;        // h / max(|c|, |s|): path length per step
    int rows;           // 1: step over rows y (|c| >= |s|), fast axis x; 0: transposed
    // Pixel-driven footprint: bin coordinate t(i, j) = t0 + i * tA + j * tB
    double t0, tA, tB;
    float tA_hi, tA_lo, tB_hi, tB_lo;
    float rfoot;        // half-width of the footprint in bins: mu h / db
    float wfoot;        // footprint height h / mu
    int frame;          // frame this angle belongs to
    int pad_;
    double wstep_d, rfoot_d, wfoot_d;  // the same three in FP64 (FP64 kernels)
    // FP32 ray set-up without FP64: f0(k) = f0c_i + f0c_f + k (f0k_hi + f0k_lo),
    // f0k_hi with 12 significant bits (k * f0k_hi exact for k < 4096)
    int f0c_i;
    float f0c_f, f0k_hi, f0k_lo;
    float inv_rfoot;    // 1 / rfoot
    float df_f;         // df rounded to FP32 (step-range bounds only)
};

// Fan beam (flat detector): one Joseph march per ray (view a, bin k), stored per
// ray because the rays of one view are not parallel. The crossing of step j is
// f(j) = f0 + j df along the fast axis (x when rows = 1, else y), each step
// weighted h / max(|cos|, |sin|) = h sqrt(1 + df^2) for the ray. Steps whose
// crossing lies beyond (-1, nfast) by a margin touch no pixel, so the forward
// march may skip them and the transpose needs no step range.
template <typename real> struct FanRay;
template <> struct __align__(16) FanRay<float> {
    int ibr;             // 2 floor(f0) + rows
    float fb;            // f0 - floor(f0)
    float df_hi, df_lo;  // df split, df_hi with 12 significant bits
};
template <> struct FanRay<double> {
    double f0, df, wstep;
    int rows, jlo, jhi, pad_;
};
// Per view, for the pixel-driven transpose: q = p - S = (x h + qx0, y h + qy0) is the
// pixel centre seen from the source; its bin coordinate is
// scale (q . f) / (q . e) + (nb - 1)/2, e the central ray direction, f the detector axis.
struct FanView {
    float qx0, qy0, ex, ey, fx, fy;
};
// Margin, in bins, of the transpose's FP32 search for the bins a pixel can reach (the host
// rejects geometries whose rounding bound exceeds half of it)
constexpr double FAN_PAD_BINS = 0.02;

}  // namespace mof

struct mof_problem {
    int nx = 0, ny = 0, nt = 0, nb = 0, precision = MOF_FP32;
    double h = 1.0, db = 1.0;
    long long ns = 0, n = 0, m = 0, nv = 0;
    int A = 0;                          // total number of angles
    std::vector<int> na, aoff;          // host: angles per frame, offsets (nt+1)
    mof::AngleParams *d_ang = nullptr;  // device [A]
    int *d_aoff = nullptr;              // device [nt+1] first angle of each frame
    int device = 0;
    void *ws = nullptr;                 // solver workspace (solver.cu)
    int timing = 0;
    void *timer = nullptr;              // kernel-class timer (solver.cu)
    int warp_mode = 0;                  // M(s): 0 bilinear, 1 rounding and clipping (Sec. 3)
    int fan = 0;                        // 1: fan beam with a flat detector
    double rs = 0, rd = 0;              // source and detector distances from the centre
    float fan_scale = 0;                // (rs + rd) / db
    void *d_fanray = nullptr;           // device FanRay<real>[A * nb] (fan only)
    mof::FanView *d_fanview = nullptr;  // device [A] (fan only)
};

namespace mof {

// Operator launchers (ops_*.cu). Templated on the element type; `stream` is
// the caller's stream. All return MOF_OK or a launch error.
// per_frame: one launch per frame (the plain execution form), else one for the sequence
template <typename real> mof_status launch_project(const mof_problem *p, const real *u, real *uT_scratch, real *b, cudaStream_t st, bool per_frame = false);
template <typename real> mof_status launch_backproject(const mof_problem *p, const real *b, real *u, cudaStream_t st, bool per_frame = false);
template <typename real> mof_status launch_grad(const mof_problem *p, int nf, const real *u, real *g, cudaStream_t st);
template <typename real> mof_status launch_gradT(const mof_problem *p, int nf, const real *g, real *u, cudaStream_t st);
template <typename real> mof_status launch_flow(const mof_problem *p, const real *u, const real *s, const real *sr, real *r, cudaStream_t st);
// Velocity VJP of Mhat(s, s') u: gs, gsr = (d r / d s)^T gr, (d r / d s')^T gr.
template <typename real> mof_status launch_flow_ds(const mof_problem *p, const real *u, const real *s, const real *sr, const real *gr, real *gs, real *gsr, cudaStream_t st);
// Per-tile displacement bounds of the warp transposes' gathers: bnd_* hold
// (nt-1) * tile_bound_ints ints (4 per 32x8 tile, 16-byte aligned).
int tiles_count(const mof_problem *p);
long long tile_bound_ints(const mof_problem *p);
template <typename real> mof_status launch_tile_bounds(const mof_problem *p, const real *s, const real *sr, int *bnd_s, int *bnd_sr, cudaStream_t st);
template <typename real> mof_status launch_flowT(const mof_problem *p, const real *r, const real *s, const real *sr, const int *bnd_s, const int *bnd_sr, real *u, cudaStream_t st);
template <typename real> mof_status launch_of_fields(const mof_problem *p, const real *u, int dr, real *ux, real *uy, real *ut, cudaStream_t st);
// Rescaling for Solve-OF (Sec. 4.1.5): uc = a x a block means of every frame of u;
// s = a * bilinear interpolation of the coarse velocities sc at the fine pixel centres.
template <typename real> mof_status launch_downsample(const mof_problem *p, int a, const real *u, real *uc, cudaStream_t st);
template <typename real> mof_status launch_upsample_velocity(const mof_problem *p, int a, const real *sc, real *s, cudaStream_t st);
template <typename real> mof_status launch_flow_lin(const mof_problem *p, const real *ux, const real *uy, const real *ut, const real *s, real *r, cudaStream_t st);
template <typename real> mof_status launch_flow_linT(const mof_problem *p, const real *ux, const real *uy, const real *r, real *gs, cudaStream_t st);
template <typename real> mof_status launch_reverse_flow(const mof_problem *p, const real *s, int *bnd_scratch, int *dest_scratch, real *sr, cudaStream_t st);
// Weighted regulariser normal operator: y = y_add + scale * Theta^T W Theta x,
// W from uk; q_scratch holds 2*(nt-1)*ns weighted flow rows. lam_dev (may be
// null) multiplies `scale` by *lam_dev.
// temporal: 1 adds L_t^T w_t L_t x (the temporal differences of D1-OF), 0 is M-OF
template <typename real> mof_status launch_reg_normal(const mof_problem *p, int temporal, const real *x, const real *uk, const real *s, const real *sr,
                                                      const int *bnd_s, const int *bnd_sr, double eps, double scale, const double *lam_dev,
                                                      const real *y_add, real *q_scratch, real *y, cudaStream_t st);

// ----------------------------------------------------------- device helpers
template <typename T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_maxf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// floor and fraction of base + j * (hi + lo), base = ibase + fbase with
// fbase in [0, 1): j * hi is exact for |j| < 4096, so the fraction carries
// only the rounding of a sum of O(1) terms.
__device__ __forceinline__ void affine_frac(int ibase, float fbase, float hi, float lo, int j,
                                            int &ifl, float &frac) {
    const float pj = (float)j * hi;  // exact
    const float pf = floorf(pj);
    const float r = fbase + (pj - pf) + (float)j * lo;
    const float rf = floorf(r);
    ifl = ibase + (int)pf + (int)rf;
    frac = r - rf;
}

// Error-free FP32 accumulation of a dot product ("double-float"): hi + lo carries the
// running sum with the rounding error of every product (TwoProduct by an FMA) and of
// every addition (Knuth's TwoSum) kept in lo, so a chunk's partial is accurate to a few
// units of 2^-48 of the sum of |terms|, independent of cancellation. The _rn intrinsics
// keep the compiler from contracting or reordering the steps.
struct DFAcc {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = __fmaf_rn(a, b, -p);
        const float s = __fadd_rn(hi, p);
        const float bp = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(err, e));
    }
    // add x with its rounding error kept in lo (TwoSum): a running sum of short FP32
    // partials that does not grow its error with the number of partials
    __device__ __forceinline__ void add(float x) {
        const float s = __fadd_rn(hi, x);
        const float bp = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
        hi = s;
        lo = __fadd_rn(lo, err);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

}  // namespace mof
