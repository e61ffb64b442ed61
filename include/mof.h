/*
 * mof.h -- C ABI of the GB300 MMGKS-OF library (libmof.so).
 *
 * MMGKS-OF (arXiv 2501.12497) reconstructs an image sequence u from
 * per-frame tomographic data b by alternating an optical-flow motion
 * estimate (Alg. 2, "Solve-OF") with one majorization-minimization
 * generalized-Krylov step on ||H u - b||^2 + lambda ||Theta u||_1,
 * Theta = [Psi; Mhat(s, s')] (Alg. 1, Sec. 4.1.1). This header exposes the
 * operators of that method and the solver.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Array arguments are DEVICE pointers owned by the caller and borrowed for
 *    the duration of the call (the library keeps no reference), except where
 *    a parameter is documented as a host pointer. Element type is float for a
 *    problem created with MOF_FP32 and double for MOF_FP64.
 *  - Every call that takes `stream` enqueues its work on that CUDA stream
 *    (cudaStream_t passed as void*; NULL = the legacy default stream) and
 *    returns without synchronising, unless documented otherwise.
 *  - Argument errors are detected on the host and returned synchronously;
 *    nothing is enqueued then. The text of the last error of the calling
 *    thread is available from mof_last_error().
 *  - Layouts (x fastest, all contiguous):
 *      image sequence  u[nt][ny][nx]        (Sec. 2.1: vec of column-stacked
 *                                            frames; pixel row index y*nx + x)
 *      sinogram        b[sum_t na[t]][nb]   (frame t's na[t] angles in order)
 *      velocities      s[nt-1][2][ny][nx]   (component 0 = s_x, 1 = s_y);
 *                      s[p] maps frame p to frame p+1 (M(s(p)) u_{p+1} ~ u_p)
 *      reverse flow    sr[nt-1][2][ny][nx]  (sr[p] = s'(p+1), on frame p+1)
 *      gradient        g[nf][2][ny][nx]     (d=0: u(x+1)-u(x), d=1: u(y+1)-u(y),
 *                                            last column/row identically 0)
 *      flow residual   r[2][nt-1][ny][nx]   (r[0] = Mbar rows, r[1] = Mbar' rows)
 *      OF fields       ux, uy, ut [nt-1][ny][nx]
 *      velocity grad.  gs[nt-1][2 comp][2 dir][ny][nx]
 *  - Geometry: 2D parallel beam. Pixel centres x_i = (i - (nx-1)/2) h,
 *    y_j = (j - (ny-1)/2) h; bin centres sigma_k = (k - (nb-1)/2) db; the ray
 *    (theta, k) is { x cos(theta) + y sin(theta) = sigma_k }.
 */
#ifndef MOF_H
#define MOF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MOF_OK = 0,
    MOF_EINVAL = 1,        /* bad argument (null pointer, size, value) */
    MOF_ENOMEM = 2,        /* device or host allocation failed */
    MOF_ECUDA = 3,         /* a CUDA runtime call failed (text in mof_last_error) */
    MOF_ENUMERIC = 4,      /* non-finite value or failed factorisation detected on device */
    MOF_ETIMEOUT = 5,      /* a bounded device wait expired */
    MOF_EUNSUPPORTED = 6   /* valid but not supported by this build */
} mof_status;

typedef enum { MOF_FP32 = 0, MOF_FP64 = 1 } mof_precision;

typedef enum { MOF_RULE_DP = 0, MOF_RULE_GCV = 1, MOF_RULE_FIXED = 2 } mof_rule;

/* Geometry of one problem (Sec. 2.1: H = blockdiag(H^1, ..., H^nt)).
 * na and angles are HOST arrays, read during mof_problem_create only. */
typedef struct {
    int nx, ny, nt;        /* frame width, height, number of frames (nt >= 2) */
    int nb;                /* detector bins per angle */
    const int *na;         /* [nt] angles of each frame (>= 1) */
    const double *angles;  /* [sum na] projection angles in radians */
    double pixel_size;     /* h > 0 */
    double bin_size;       /* db > 0 */
} mof_geometry;

typedef struct mof_problem mof_problem;

/* Parameters of Alg. 1 / Alg. 2. mof_default_params fills the defaults. */
typedef struct {
    int ell;               /* initial GKB subspace of the image step (Sec. 5: 10) */
    int tau;               /* Solve-OF every tau outer iterations (Sec. 4.1.5); 0 = never */
    int of_iters;          /* GKS iterations per Solve-OF (Sec. 5: 20) */
    int of_ell;            /* GKB start of Solve-OF (10) */
    int of_dr;             /* box half-width Delta r of App. C (1) */
    int image_rule;        /* mof_rule for lambda of the image step (DP when delta known) */
    double eps;            /* l1 smoothing epsilon of Alg. 1 (1e-3) */
    double eta;            /* DP safety factor (Sec. 4.1.3: 1.01) */
    double noise_norm;     /* delta = ||e||, required by MOF_RULE_DP */
    double lam_fixed;      /* lambda for MOF_RULE_FIXED */
    double breakdown_tol;  /* <= 0: 1e-10 (FP64) / 1e-6 (FP32) relative breakdown threshold */
    int of_streams;        /* execution only: the GKS iterations of Solve-OF run the frame pairs in
                              this many groups on separate streams, so that one group's small
                              FP64 solves overlap another group's bandwidth-bound kernels; the
                              result does not depend on it. 0 = automatic: one group per pair,
                              up to 64 groups; at most 64 */
    int of_scale;          /* Solve-OF on frames downsampled by this factor a (Sec. 4.1.5, Sec. 5:
                              a = 2 or 4 to reach frames under 50x50): a x a block means, the
                              velocities interpolated bilinearly back to the full grid and
                              multiplied by a. 1 = full resolution; a must divide nx and ny */
    int temporal_tv;       /* 1: D1-OF (AnisoTV-OF, Table 2): Theta = [Psi; L_t; Mhat] with L_t the
                              forward differences between consecutive frames, all rows in the
                              same l1 norm; 0 (default): M-OF, Theta = [Psi; Mhat] */
    int of_pq;             /* norms of Solve-OF (Sec. 4.1.2): 2 (default, the paper's experiments)
                              p = q = 2 by GKS; 1: p = q = 1 by MM-GKS (App. A) with IRLS weights
                              ((.)^2 + eps^2)^(-1/2) on the flow residual and on (L+L) s, recomputed
                              from the current velocity (zero at the start) every iteration; the
                              subspace stops growing when the orthogonalised residual is at most
                              breakdown_tol times its norm before the orthogonalisation */
    int plain;             /* execution form (results equal up to rounding): 0 (default) the
                              batched form, every outer iteration replayed from a CUDA graph and
                              the frame pairs of Solve-OF in concurrent groups; 1 the plain
                              unbatched per-frame form, every kernel launched from the host as it
                              comes, Solve-OF one frame pair after another on one stream and the
                              projector and its adjoint one frame per launch (the reference point
                              the batched form is measured against) */
} mof_solver_params;

/* One record per outer iteration k of mof_solve (host struct). */
typedef struct {
    double lambda;         /* regularisation parameter chosen at iteration k */
    double resid;          /* ||H u^(k+1) - b|| */
    double rnorm;          /* ||r^(k+1)|| before normalisation (0 if not expanded) */
    int basis;             /* dimension l+k of the image-step subspace used */
    int flag;              /* DP: 0 root, 1 no root (residual > target), 2 (< target) */
    int of_basis_min;      /* smallest Solve-OF basis over pairs (0 if no OF this k) */
    int of_basis_max;      /* largest Solve-OF basis over pairs */
} mof_report;

void mof_default_params(mof_solver_params *p);

/* Create a problem: validates the geometry, uploads the angle tables.
 * precision: MOF_FP32 (operators in FP32, Krylov bookkeeping and small
 * solves in FP64) or MOF_FP64 (everything FP64). Uses the current device.
 * On success *out owns its device memory until mof_problem_destroy. */
mof_status mof_problem_create(const mof_geometry *g, int precision, mof_problem **out);
void mof_problem_destroy(mof_problem *p);

/* Create a fan-beam problem (Sec. 5.1: the experiments' 2D flat fan-beam
 * geometry): for the view at angle theta the source is the point
 * -source_distance (-sin theta, cos theta) and the detector the line at
 * detector_distance on the other side of the centre, perpendicular to
 * (-sin theta, cos theta); bin k is its point at sigma_k = (k - (nb-1)/2)
 * bin_size along (cos theta, sin theta), and its ray the line from the source
 * through that point. mof_apply_A integrates each ray by the same Joseph rule
 * as the parallel rays (its own direction, step h / max(|cos|, |sin|));
 * mof_apply_AT is its exact transpose (pixel-driven gather). Every other
 * entry point is unchanged. Distances are in the units of pixel_size.
 * Returns MOF_EINVAL unless source_distance exceeds half the frame diagonal
 * plus two pixels and detector_distance >= 0, and MOF_EUNSUPPORTED when the
 * rounding bound of the transpose's FP32 search for a pixel's bins,
 * 12 u (1 + t)^2 S + 2 u nb bins with u = 2^-24, S = (source_distance +
 * detector_distance) / bin_size and t = (nb / 2 + 1) / S, exceeds half its
 * margin of 0.02 bins (S up to about 14000 for a narrow fan, about 7000 when
 * the detector's half width is 0.4 (source_distance + detector_distance));
 * holds a ray table of 16 (FP32) or 40 (FP64) bytes per data value on the
 * device. */
mof_status mof_problem_create_fan(const mof_geometry *g, double source_distance, double detector_distance,
                                  int precision, mof_problem **out);

/* Sizes: n = nx*ny*nt pixels, m = nb * sum(na) data values,
 * nv = (nt-1)*2*nx*ny values of one velocity field. Any pointer may be NULL. */
mof_status mof_problem_sizes(const mof_problem *p, long long *n, long long *m, long long *nv);

/* b = H u: per frame, per angle and bin, Joseph's line integral along the
 * ray (Sec. 2.1 block-diagonal H; entry a = (h/mu) max(0, 1 - |sigma - p|/(mu h)),
 * p = x cos + y sin, mu = max(|cos|, |sin|)). Ray-driven. u: n, b: m. */
mof_status mof_apply_A(mof_problem *p, const void *u, void *b, void *stream);

/* u = H^T b: the exact transpose of mof_apply_A (same entries), pixel-driven
 * gather (Sec. 4.1.1: H^T in the normal-equation residual). b: m, u: n. */
mof_status mof_apply_AT(mof_problem *p, const void *b, void *u, void *stream);

/* g = Psi u, forward differences along x and y of every frame
 * (eq. (L), Psi = blockdiag(L, ..., L)). u: n, g: 2n. */
mof_status mof_apply_grad(mof_problem *p, const void *u, void *g, void *stream);

/* u = Psi^T g (exact transpose; padded zero rows ignore g there). */
mof_status mof_apply_gradT(mof_problem *p, const void *g, void *u, void *stream);

/* Encoding of the warp M(s) (Sec. 3, the two constructions of the motion
 * operator) used by every operator and solve on p from now on: mode 0
 * (default), bilinear interpolation at r + s(r) clipped to the image; mode 1,
 * rounding and clipping, M(s) picks the one pixel clamp(r + round(s(r))),
 * halves rounded away from zero. In mode 1 the velocity VJP
 * (mof_apply_flow_ds) is zero. Returns MOF_EINVAL for any other mode. */
mof_status mof_set_warp(mof_problem *p, int mode);

/* r = Mhat(s, s') u (Sec. 3, bilinear-warp encoding of M(s); Sec. 4:
 * Mhat = [Mbar; Mbar']):  r[0][p] = u_p - M(s_p) u_{p+1},
 * r[1][p] = u_{p+1} - M(sr_p) u_p. M(s) samples its argument at r + s(r),
 * clipped to the image, with bilinear weights (or by rounding, see
 * mof_set_warp). u: n, s, sr: nv, r: 2*(nt-1)*nx*ny. */
mof_status mof_apply_flow(mof_problem *p, const void *u, const void *s, const void *sr,
                          void *r, void *stream);

/* u = Mhat(s, s')^T r (exact transpose of mof_apply_flow). Deterministic: the
 * terms of each output pixel are summed exactly in 64-bit fixed point (scaled per
 * 64x16 tile by the tile's largest term), then rounded once; a non-finite value
 * among a tile's terms makes that tile's outputs NaN. */
mof_status mof_apply_flowT(mof_problem *p, const void *r, const void *s, const void *sr,
                           void *u, void *stream);

/* Vector-Jacobian product of the flow residual r = Mhat(s, s') u (mof_apply_flow,
 * Sec. 2.3) with respect to the velocities: for a cotangent gr (layout of r),
 *   gs[t]  = -gr[0][t] * grad_s  B(u_{t+1}; x + s_t),
 *   gsr[t] = -gr[1][t] * grad_s' B(u_t;     x + sr_t),
 * with B the clipped bilinear sample: on the forward pass's cell,
 * dB/dsx = (1-wy)(f01-f00) + wy(f11-f10), dB/dsy = (1-wx)(f10-f00) + wx(f11-f01),
 * zero along an axis where the sample point is clipped (x + s < 0 or
 * x + s >= n-1), the derivative from the right where x + s is an integer.
 * u: n; s, sr: nv; gr: 2 (nt-1) ns; gs, gsr: nv (outputs). The image VJP of r
 * is mof_apply_flowT; the projector's is mof_apply_AT. Used as the backward
 * pass of the differentiable operators of the binding. */
mof_status mof_apply_flow_ds(mof_problem *p, const void *u, const void *s, const void *sr, const void *gr,
                             void *gs, void *gsr, void *stream);

/* App. C derivative fields of every pair (u_p, u_{p+1}), box half-width dr,
 * image flipped about its edges:  ux = box-averaged central x-difference of
 * u_p, uy likewise in y, ut = box average of u_{p+1} - u_p. u: n; outputs (nt-1)*nx*ny. */
mof_status mof_of_fields(mof_problem *p, const void *u, int dr, void *ux, void *uy, void *ut,
                         void *stream);

/* Rescaling for Solve-OF (Sec. 4.1.5: Solve-OF on smaller frames, velocities upscaled; the
 * paper does not name the operators):
 * uc = the a x a block means of every frame of u. a >= 1 must divide nx and ny.
 * u: n values, uc: nt * (ny/a) * (nx/a) values (the same layout at the coarse size). */
mof_status mof_downsample(mof_problem *p, int a, const void *u, void *uc, void *stream);

/* s = a * (bilinear interpolation of the coarse velocities sc at the fine pixel centres),
 * the coarse coordinate of fine pixel x being (x + 1/2)/a - 1/2 clamped to the coarse grid
 * (so that velocities in coarse pixels become fine pixels). a as for mof_downsample.
 * sc: (nt-1) * 2 * (ny/a) * (nx/a) values, s: nv values. */
mof_status mof_upsample_velocity(mof_problem *p, int a, const void *sc, void *s, void *stream);

/* r = Upsilon s + u_t per pair (Sec. 2.2: the pointwise row [u_x u_y]).
 * s: nv, r: (nt-1)*nx*ny. */
mof_status mof_apply_flow_lin(mof_problem *p, const void *ux, const void *uy, const void *ut,
                              const void *s, void *r, void *stream);

/* gs = Upsilon^T r per pair: gs[p][0] = ux r, gs[p][1] = uy r. */
mof_status mof_apply_flow_linT(mof_problem *p, const void *ux, const void *uy, const void *r,
                               void *gs, void *stream);

/* gs = (L (+) L) s: forward-difference gradient of each velocity component
 * (Sec. 2.2, the discrete gradient of the velocity regulariser). gs: 2*nv. */
mof_status mof_apply_vgrad(mof_problem *p, const void *s, void *gs, void *stream);

/* s = (L (+) L)^T gs. */
mof_status mof_apply_vgradT(mof_problem *p, const void *gs, void *s, void *stream);

/* sr = reverse flow from s by the remark of Sec. 3: the pixel r of frame p
 * moves to round(r + s_p(r)) (half away from zero, clipped) in frame p+1 and
 * carries -s_p(r) there; arrivals are averaged, pixels without arrivals get 0. */
mof_status mof_reverse_flow(mof_problem *p, const void *s, void *sr, void *stream);

/* y = Theta^T W Theta x with Theta = [Psi; Mhat(s, s')] and IRLS weights
 * W = diag(((Theta uk)^2 + eps^2)^(-1/2)) recomputed from uk (Alg. 1:
 * P^2 with P = diag((nu^2 + eps^2)^(-1/4)), nu = Theta u^(k)). x, uk, y: n.
 * The terms of each output pixel are summed as in mof_apply_flowT. */
mof_status mof_apply_reg_normal(mof_problem *p, const void *x, const void *uk, const void *s,
                                const void *sr, double eps, void *y, void *stream);

/* Solve-OF (Alg. 2, p = q = 2) on every consecutive pair of u at once:
 * GKB start of prm->of_ell steps from -u_t, then prm->of_iters GKS
 * iterations on min ||Upsilon s + u_t||^2 + gamma ||(L (+) L) s||^2 with
 * gamma chosen by GCV every iteration. Pairs whose u_t is zero get s = 0.
 * u: n, s: nv. Synchronises `stream` before returning (reads status). */
mof_status mof_solve_of(mof_problem *p, const mof_solver_params *prm, const void *u, void *s,
                        void *stream);

/* MMGKS-OF (Alg. 1) for n_outer outer iterations from u^(0) = 0, s^(0) = 0
 * (ell + n_outer <= 60 and of_ell + of_iters <= 64; larger: MOF_EUNSUPPORTED).
 * b: m (device). u_out: n. s_out, sr_out: nv each, may be NULL (the flow
 * used by the last iteration). report: HOST array of n_outer records, may
 * be NULL. The library allocates its workspace (Krylov bases, Gram
 * matrices) on first use and keeps it until mof_problem_destroy.
 * Synchronises `stream` before returning; device-detected numerical errors
 * return MOF_ENUMERIC. */
mof_status mof_solve(mof_problem *p, const mof_solver_params *prm, int n_outer, const void *b,
                     void *u_out, void *s_out, void *sr_out, mof_report *report, void *stream);

/* mof_solve with HOST input and output buffers (b: m, u_out: n, s_out and
 * sr_out: nv or NULL); copies in and out on `stream` inside the call. Host
 * buffers may be pageable or pinned; pinned buffers overlap better. */
mof_status mof_solve_host(mof_problem *p, const mof_solver_params *prm, int n_outer,
                          const void *b_host, void *u_host, void *s_host, void *sr_host,
                          mof_report *report, void *stream);

/* Batched MMGKS-OF (Alg. 1) over `count` independent problems, each created
 * on its own and of any size and precision: problems[i] with params[i] (its
 * own noise level), device arrays b[i] (m_i) -> u_out[i] (n_i), s_out[i]
 * (nv_i; s_out or any entry may be NULL), reports[i] (HOST, n_outer records;
 * reports or any entry may be NULL). Each problem's outer iterations run on
 * the problem's own streams, enqueued outer iteration by outer iteration
 * across the batch, so the GPU works on many problems at once; every problem's
 * result is the one mof_solve gives it (bit for bit). A problem may appear
 * only once. Argument errors are returned before anything is enqueued;
 * otherwise the call returns after all problems finished, with the first
 * problem's error (its batch index in mof_last_error). */
mof_status mof_solve_batch(mof_problem *const *problems, int count, const mof_solver_params *params, int n_outer,
                           const void *const *b, void *const *u_out, void *const *s_out,
                           mof_report *const *reports, void *stream);

/* Autotuner of the execution parameter of_streams (the number of frame-pair
 * groups Solve-OF runs on separate streams): times n_probe outer iterations of
 * the batch (mof_solve_batch; count = 1 tunes a single problem) for each
 * candidate in {1, 2, 4, 8, 16, 32, 64} (at most the number of frame pairs), each after an
 * untimed run that captures its graphs, and writes the fastest into every
 * params[i].of_streams (and its time in milliseconds into *best_ms, may be
 * NULL). u_scratch[i] (n_i, device) receives the probes' images. The result of
 * a solve does not depend on of_streams, so tuning changes speed only. */
mof_status mof_autotune(mof_problem *const *problems, int count, mof_solver_params *params, int n_probe,
                        const void *const *b, void *const *u_scratch, double *best_ms, void *stream);

/* Per-kernel-class device time of the last mof_solve when timing was
 * enabled with mof_set_timing(p, 1): fills up to `cap` entries of names
 * (static strings), milliseconds and launch counts; returns the number of
 * classes in *count. Timing records CUDA events around each launch on the
 * solver's stream. */
mof_status mof_set_timing(mof_problem *p, int enable);
mof_status mof_get_timing(const mof_problem *p, int cap, const char **names, double *ms,
                          long long *launches, int *count);

/* Bound of the device waits on tile copies (library plumbing; the paper has no
 * counterpart). The fused reorthogonalisation pass stages its tiles with bulk
 * copies that complete on a shared-memory barrier, and each CTA polls that barrier
 * at most `polls` times (default 2^22; polls < 0 restores it) before it records a
 * timeout in the problem's device error word, waits with the default bound for its
 * own copies to land, and returns; the next synchronising call (the end of
 * mof_solve, mof_solve_of, ...) returns MOF_ETIMEOUT. Applies to the current device
 * and to launches made after the call (the device is synchronised first). For tests
 * of the timeout path: polls = 0 makes every such wait give up at once. */
mof_status mof_debug_set_wait_limit(long long polls);

/* Measured FP32 ceilings of the current device (library plumbing; the paper has no
 * counterpart), the roofline of the projector pair, whose Joseph taps are FP32 and
 * L1-load work rather than DRAM traffic: *fma_tflops the FP32 FMA rate (2 flops per
 * FMA) of a kernel of independent FMA chains, *l1_gloads_per_s the rate of 4-byte
 * loads served by L1 (billions per second). Best of five timed launches each; takes
 * about a second; allocates and frees its own small buffers. */
mof_status mof_measure_fp32_peaks(double *fma_tflops, double *l1_gloads_per_s);

/* Number of CUDA kernels this library has launched in the process so far
 * (all threads, all problems); differences bracket a region of interest. */
long long mof_kernel_launches(void);

/* ---- allocation-free variant (library plumbing; the paper has no counterpart) ----
 *
 * Mhat^T r exactly as mof_apply_flowT (same kernels, bit-identical result,
 * Sec. 2.3), but without allocating: mof_apply_flowT takes its scratch (the
 * per-tile bounds of the integer displacements of s and s' that tell each
 * output tile which sources can reach it) from the problem's workspace, which the library
 * allocates on first use; this call takes it from a fixed device array owned
 * by the library, one per device, of MOF_FLOWT_NOALLOC_MAX_INTS ints (16 MiB).
 * It is for callers that cannot allocate device memory at call time: a
 * process running against a fixed device-memory budget, where the first-use
 * allocation could fail with MOF_ENOMEM in the middle of a run, or a
 * latency-critical loop, where cudaMalloc may synchronise the device.
 *  - Size limit: the problem needs 8 (nt-1) (ceil(nx/64) ceil(ny/16) + 1) ints
 *    (four per 64x16 tile and four for the field's reach, for each of s and s');
 *    a problem needing more than MOF_FLOWT_NOALLOC_MAX_INTS returns
 *    MOF_EUNSUPPORTED and enqueues nothing.
 *  - Initial state: each call writes the part of the array it uses before
 *    reading it (the tile bounds are overwritten, the reach is set to zero
 *    and then raised); the caller initialises nothing.
 *  - Set-up: the first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, return code checked: MOF_ECUDA on failure) and
 *    caches it; make that first call before any stream capture begins. Every
 *    call must be made with the problem's device current (MOF_EINVAL
 *    otherwise). The cached address does not survive cudaDeviceReset: do not
 *    use this entry point on a device that was reset in the same process.
 *  - Concurrency: the array is shared by every problem and stream of the
 *    device. Calls whose kernels overlap in time (different streams, or
 *    different host threads without ordering) race on it and give undefined
 *    results; order them, e.g. on one stream.
 * Arguments, layouts and the other errors as mof_apply_flowT. */
#define MOF_FLOWT_NOALLOC_MAX_INTS (1 << 22)
mof_status mof_apply_flowT_noalloc(mof_problem *p, const void *r, const void *s, const void *sr,
                                   void *u, void *stream);

/* Text of the last error on the calling thread ("" if none). */
const char *mof_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MOF_H */
