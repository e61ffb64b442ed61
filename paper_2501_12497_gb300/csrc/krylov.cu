// K10: batched Krylov vector operations on B independent bases
// (the outer image step has B = 1; Solve-OF has one basis per frame pair).
//
// A basis is stored as V[b][j][N] (vector j of problem b contiguous), with
// the current size K[b] in device memory, so kernel grids never depend on
// the basis size and a whole solver iteration can be replayed as a graph.
//
// Reductions (dot products, norms) are deterministic: products in the
// storage precision, summed in a fixed tree within a chunk of CHUNK
// elements, chunk partials written out and combined in FP64 in chunk order.
#include "common.cuh"
#include "solver.cuh"

#include <atomic>
#include <type_traits>

namespace mof {

constexpr int KT = 256;                    // threads per block
constexpr int KE = 8;                      // elements per thread per chunk (norms, scalar paths)
constexpr int CHUNK = KT * KE;             // elements per chunk of the scalar kernels
constexpr int DCH_BYTES = 16384;           // bytes of one staged right-hand chunk of the multi-dot
template <typename real>
constexpr int dch() { return DCH_BYTES / (int)sizeof(real); }  // elements per multi-dot chunk

long long krylov_chunks(long long N) { return (N + CHUNK - 1) / CHUNK; }
template <typename real>
long long mdot_chunks(long long N) { return (N + dch<real>() - 1) / dch<real>(); }

// block-wide sum of one value per thread into thread 0's return (FP64 across warps)
template <typename acc_t>
__device__ __forceinline__ double block_sum_to_double(acc_t v, double *sh) {
    if constexpr (sizeof(acc_t) == 4) v = warp_sumf(v);
    else v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = (double)v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < KT / 32; ++i) r += sh[i];
    __syncthreads();
    return r;
}

// partial[b][chunk][v][j] = sum_{i in chunk} V[b][j][i] * x_v[b][i], j < K[b], v < NV.
// EXACT (FP32 data only): error-free accumulation per lane (DFAcc), lanes summed in FP64;
// used for the Gram matrices whose projected residual subtracts nearly equal terms.
// The NV right-hand chunks are staged in shared memory; warp w streams the
// basis vectors j = w, w + 8, ... of the chunk (16-byte loads when VEC) and
// reduces each dot once.
template <typename real, int NV, bool VEC, bool EXACT = false>
__global__ void __launch_bounds__(KT) k_mdot(const real *__restrict__ V, long long N, int Kmax, const int *__restrict__ K,
                                             const int *__restrict__ act, DotVecs<real> xs, double *__restrict__ partial,
                                             int nchunk) {
    constexpr int DCH = dch<real>();
    __shared__ __align__(16) real sx[NV][DCH];
    const int b = blockIdx.y, chunk = blockIdx.x;
    if (act && !act[b]) return;
    const int Kb = min(K[b], Kmax);
    const long long c0 = (long long)chunk * DCH;
    const int len = (int)min((long long)DCH, N - c0);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const real *xb = xs.x[v] + b * xs.stride[v] + c0;
        for (int i = threadIdx.x; i < DCH; i += KT) sx[v][i] = i < len ? xb[i] : (real)0;
    }
    __syncthreads();
    const real *Vb = V + (long long)b * Kmax * N + c0;
    if constexpr (EXACT && sizeof(real) == 4) {
        for (int j = w; j < Kb; j += KT / 32) {
            const real *vj = Vb + (long long)j * N;
            DFAcc a[NV];
            for (int i = l; i < len; i += 32) {
                const float q = vj[i];
#pragma unroll
                for (int v = 0; v < NV; ++v) a[v].add_prod(q, sx[v][i]);
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const double t = warp_sum(a[v].value());
                if (l == 0) partial[(((long long)b * nchunk + chunk) * NV + v) * Kmax + j] = t;
            }
        }
        return;
    }
    for (int j = w; j < Kb; j += KT / 32) {
        const real *vj = Vb + (long long)j * N;
        if constexpr (VEC) {
            // FP32: each step's 16 products per right-hand side summed in FP32, the steps'
            // partials accumulated with their rounding errors (DFAcc::add), lanes in FP64
            DFAcc a[NV];
            const float4 *v4 = reinterpret_cast<const float4 *>(vj);
            const int n4 = len >> 2;
            int i = l;
#pragma unroll 1
            for (; i + 96 < n4; i += 128) {
                const float4 q0 = __ldcs(v4 + i), q1 = __ldcs(v4 + i + 32), q2 = __ldcs(v4 + i + 64), q3 = __ldcs(v4 + i + 96);
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const float4 *x4 = reinterpret_cast<const float4 *>(sx[v]);
                    const float4 y0 = x4[i], y1 = x4[i + 32], y2 = x4[i + 64], y3 = x4[i + 96];
                    float t = q0.x * y0.x + q0.y * y0.y + q0.z * y0.z + q0.w * y0.w;
                    t += q1.x * y1.x + q1.y * y1.y + q1.z * y1.z + q1.w * y1.w;
                    t += q2.x * y2.x + q2.y * y2.y + q2.z * y2.z + q2.w * y2.w;
                    t += q3.x * y3.x + q3.y * y3.y + q3.z * y3.z + q3.w * y3.w;
                    a[v].add(t);
                }
            }
            for (; i < n4; i += 32) {
                const float4 q = __ldcs(v4 + i);
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const float4 y = reinterpret_cast<const float4 *>(sx[v])[i];
                    a[v].add(q.x * y.x + q.y * y.y + q.z * y.z + q.w * y.w);
                }
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const double t = warp_sum(a[v].value());
                if (l == 0) partial[(((long long)b * nchunk + chunk) * NV + v) * Kmax + j] = t;
            }
        } else {
            real a[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) a[v] = 0;
            for (int i = l; i < len; i += 32) {
                const real q = vj[i];
#pragma unroll
                for (int v = 0; v < NV; ++v) a[v] += q * sx[v][i];
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                real t = a[v];
                if constexpr (sizeof(real) == 4) t = warp_sumf(t);
                else t = warp_sum(t);
                if (l == 0) partial[(((long long)b * nchunk + chunk) * NV + v) * Kmax + j] = (double)t;
            }
        }
    }
}

// out_v[b*bstride + i*istride + col*jstride] = sign * sum_chunk partial[b][chunk][v][i], i < K[b];
// col = K[b] - 1 when last_col, else 0. One warp per output (lanes stride
// over the chunks, then a fixed tree), blockIdx.y = problem.
constexpr int SUMT = 256;
__global__ void __launch_bounds__(SUMT) k_sum_chunks(const double *__restrict__ partial, int nchunk, int NV, int Kmax,
                                                     const int *__restrict__ K, const int *__restrict__ act, DotOuts outs) {
    const int b = blockIdx.y;
    if (act && !act[b]) return;
    const int Kb = min(K[b], Kmax);
    const int e = blockIdx.x * (SUMT / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (e >= NV * Kb) return;
    const int v = e / Kb, i = e - (e / Kb) * Kb;
    const DotOut &o = outs.o[v];
    if (!o.out) return;
    double s = 0.0;
#pragma unroll 8
    for (int c = lane; c < nchunk; c += 32) s += partial[(((long long)b * nchunk + c) * NV + v) * Kmax + i];
    s = warp_sum(s);
    if (lane == 0) {
        const long long col = o.last_col ? (long long)(Kb - 1) : 0;
        o.out[b * o.bstride + (long long)i * o.istride + col * o.jstride] = o.sign * s;
    }
}

// out[b] = sum_j V[b][j] c[b][j] (mode 0), x[b] - sum_j V[b][j] c[b][j] (mode 1),
// sum_j V[b][j] c[b][j] - x[b] (mode 2); optionally ||out[b]||^2 per block.
// One thread per 4 consecutive elements (16-byte loads when VEC), basis
// vectors streamed four at a time.
constexpr int CT = 256;
template <typename real, int MODE, bool VEC>
__global__ void __launch_bounds__(CT) k_combine(const real *__restrict__ V, long long N, int Kmax, const int *__restrict__ K,
                                                const int *__restrict__ act, const double *__restrict__ c, long long cstride,
                                                const real *__restrict__ x, long long xstride, real *__restrict__ out,
                                                long long ostride, double *__restrict__ nrm_partial, int nblk) {
    __shared__ real sc[64];
    __shared__ double sh[CT / 32];
    const int b = blockIdx.y;
    if (act && !act[b]) return;
    const int Kb = min(K[b], Kmax);
    for (int j = threadIdx.x; j < Kb; j += CT) sc[j] = (real)c[b * cstride + j];
    __syncthreads();
    const long long i4 = ((long long)blockIdx.x * CT + threadIdx.x) * 4;
    const real *Vb = V + (long long)b * Kmax * N;
    real n2 = 0;
    if (i4 < N) {
        real acc[4] = {0, 0, 0, 0};
        if (VEC && i4 + 3 < N) {
            int j = 0;
            for (; j + 3 < Kb; j += 4) {
                const float4 q0 = __ldcs(reinterpret_cast<const float4 *>(Vb + (long long)j * N + i4));
                const float4 q1 = __ldcs(reinterpret_cast<const float4 *>(Vb + (long long)(j + 1) * N + i4));
                const float4 q2 = __ldcs(reinterpret_cast<const float4 *>(Vb + (long long)(j + 2) * N + i4));
                const float4 q3 = __ldcs(reinterpret_cast<const float4 *>(Vb + (long long)(j + 3) * N + i4));
                const real c0 = sc[j], c1 = sc[j + 1], c2 = sc[j + 2], c3 = sc[j + 3];
                acc[0] += q0.x * c0 + q1.x * c1 + q2.x * c2 + q3.x * c3;
                acc[1] += q0.y * c0 + q1.y * c1 + q2.y * c2 + q3.y * c3;
                acc[2] += q0.z * c0 + q1.z * c1 + q2.z * c2 + q3.z * c3;
                acc[3] += q0.w * c0 + q1.w * c1 + q2.w * c2 + q3.w * c3;
            }
            for (; j < Kb; ++j) {
                const float4 q = __ldcs(reinterpret_cast<const float4 *>(Vb + (long long)j * N + i4));
                const real cj = sc[j];
                acc[0] += q.x * cj;
                acc[1] += q.y * cj;
                acc[2] += q.z * cj;
                acc[3] += q.w * cj;
            }
        } else {
            for (int j = 0; j < Kb; ++j) {
                const real cj = sc[j];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (i4 + e < N) acc[e] += Vb[(long long)j * N + i4 + e] * cj;
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const long long i = i4 + e;
            if (i < N) {
                const real v = MODE == 1 ? x[b * xstride + i] - acc[e] : (MODE == 2 ? acc[e] - x[b * xstride + i] : acc[e]);
                out[b * ostride + i] = v;
                n2 += v * v;
            }
        }
    }
    if (nrm_partial) {
        const double s = block_sum_to_double(n2, sh);
        if (threadIdx.x == 0) nrm_partial[(long long)b * nblk + blockIdx.x] = s;
    }
}

// ------------------------------------------------------------ fused CGS2 middle pass
// x'[b] = x[b] - V[b] c[b] and the chunk partials of V[b]^T x'[b] in one pass
// over V: a CTA owns one 1 KB chunk of every basis vector of its problem and
// of x, brought into shared memory by 1D bulk copies (TMA) that complete on
// an mbarrier; it forms x' for the chunk, writes it, and takes the dots from
// the same staged tile. Classical Gram-Schmidt twice then reads V three times
// instead of four. Products in the storage precision, summed per chunk in a
// fixed order (deterministic), chunks combined in FP64 by k_sum_chunks.
constexpr int SDT = 64;        // threads per CTA
constexpr int SD_BYTES = 1024; // bytes of one vector's chunk (small tiles: many CTAs per SM keep copies in flight)
template <typename real>
constexpr int sdch() { return SD_BYTES / (int)sizeof(real); }
constexpr long long MBAR_MAX_POLLS = 1LL << 22;

long long subdot_chunks(long long N, int elem_bytes) { return (N * elem_bytes + SD_BYTES - 1) / SD_BYTES; }
long long krylov_partial_doubles(long long N, int Kmax) {
    // multi-dot (<= 3 right-hand sides), norms and combines; fused pass, whose fixed-size
    // chunks hold the fewest elements (so are the most numerous) for FP64
    const long long a = krylov_chunks(N) * 3 * Kmax, b = subdot_chunks(N, 8) * (Kmax + 1);
    return a > b ? a : b;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// Bound of the first wait of a tile (polls of the mbarrier); mof_debug_set_wait_limit
// lowers it to make the timeout path run in tests. The wait after a timeout, which only
// keeps the CTA alive until its own copies have landed, always uses MBAR_MAX_POLLS.
__device__ long long g_wait_polls = MBAR_MAX_POLLS;

// poll the mbarrier phase with a bound; false when the bound ran out
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned phase, long long limit = MBAR_MAX_POLLS) {
    for (long long it = 0; it < limit; ++it) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <typename real>
__global__ void __launch_bounds__(SDT) k_sub_dot(const real *__restrict__ V, long long N, int Kmax, const int *__restrict__ K,
                                                 const int *__restrict__ act, const double *__restrict__ c, long long cstride,
                                                 const real *x, long long xstride, real *out, long long ostride,
                                                 double *__restrict__ partial, int nchunk, int *__restrict__ err, int kcap,
                                                 double *__restrict__ nrm_partial) {
    constexpr int CH = sdch<real>();
    constexpr int EPT = CH / SDT;  // elements per thread: 4 (FP32) or 2 (FP64), 16 bytes
    using vec_t = typename std::conditional<sizeof(real) == 4, float4, double2>::type;
    extern __shared__ __align__(128) unsigned char sd_smem[];
    real *sx = reinterpret_cast<real *>(sd_smem);  // [CH]
    real *sV = sx + CH;                            // [Kmax][CH]
    __shared__ real sc[64];
    __shared__ __align__(8) unsigned long long bar;
    const int b = blockIdx.y, chunk = blockIdx.x, tid = threadIdx.x;
    if (act && !act[b]) return;
    int Kb = min(K[b], Kmax);
    if (Kb > kcap) {  // the tile holds kcap vectors: a caller's bound was wrong
        if (tid == 0 && err) atomicOr(err, 8);
        Kb = kcap;
    }
    const long long c0 = (long long)chunk * CH;
    const int len = (int)min((long long)CH, N - c0);
    const unsigned bar_a = smem_u32(&bar);
    // the copies go out first (the thread that initialised the barrier issues them);
    // the coefficients are read while they are in flight
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const unsigned bytes = (unsigned)len * (unsigned)sizeof(real);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a), "r"(bytes * (unsigned)(Kb + 1))
                     : "memory");
        bulk_g2s(sx, x + b * xstride + c0, bytes, bar_a);
        const real *Vb = V + (long long)b * Kmax * N + c0;
        for (int j = 0; j < Kb; ++j) bulk_g2s(sV + (long long)j * CH, Vb + (long long)j * N, bytes, bar_a);
    }
    for (int j = tid; j < Kb; j += SDT) sc[j] = (real)c[b * cstride + j];
    __syncthreads();  // sc complete, and the barrier's initialisation visible to every thread
    if (!mbar_wait(bar_a, 0, g_wait_polls)) {
        if (tid == 0 && err) atomicOr(err, 4);
        mbar_wait(bar_a, 0);  // do not leave while copies may still land
        return;
    }
    // x' = x - V c on this thread's EPT consecutive elements
    const int i0 = tid * EPT;
    real acc[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) acc[e] = 0;
    for (int j = 0; j < Kb; ++j) {
        const vec_t q = *reinterpret_cast<const vec_t *>(sV + (long long)j * CH + i0);
        const real cj = sc[j];
        const real *qq = reinterpret_cast<const real *>(&q);
#pragma unroll
        for (int e = 0; e < EPT; ++e) acc[e] += qq[e] * cj;
    }
    {
        vec_t xv = *reinterpret_cast<const vec_t *>(sx + i0);
        real *xx = reinterpret_cast<real *>(&xv);
#pragma unroll
        for (int e = 0; e < EPT; ++e) xx[e] = (i0 + e < len) ? xx[e] - acc[e] : (real)0;
        *reinterpret_cast<vec_t *>(sx + i0) = xv;
        real *ob = out + b * ostride + c0;
        if (i0 + EPT <= len) {
            *reinterpret_cast<vec_t *>(ob + i0) = xv;
        } else {
#pragma unroll
            for (int e = 0; e < EPT; ++e)
                if (i0 + e < len) ob[i0 + e] = xx[e];
        }
        if (nrm_partial) {  // ||x'||^2 of the chunk (the padding is zero), FP64 across the warps
            real q = 0;
#pragma unroll
            for (int e = 0; e < EPT; ++e) q += xx[e] * xx[e];
            double dq;
            if constexpr (sizeof(real) == 4) dq = (double)warp_sumf(q);
            else dq = warp_sum(q);
            __shared__ double s_nq[SDT / 32];
            if ((tid & 31) == 0) s_nq[tid >> 5] = dq;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int wq = 0; wq < SDT / 32; ++wq) t += s_nq[wq];
                nrm_partial[(long long)b * nchunk + chunk] = t;
            }
        }
    }
    __syncthreads();
    // partial dots V_j^T x' of the chunk: warp w takes j = w, w + 4, ...
    const int w = tid >> 5, l = tid & 31;
    for (int j = w; j < Kb; j += SDT / 32) {
        real a = 0;
#pragma unroll
        for (int q = 0; q < CH / (32 * EPT); ++q) {
            const int i = (q * 32 + l) * EPT;
            const vec_t v = *reinterpret_cast<const vec_t *>(sV + (long long)j * CH + i);
            const vec_t y = *reinterpret_cast<const vec_t *>(sx + i);
            const real *vv = reinterpret_cast<const real *>(&v);
            const real *yy = reinterpret_cast<const real *>(&y);
#pragma unroll
            for (int e = 0; e < EPT; ++e)
                if (i + e < len) a += vv[e] * yy[e];
        }
        if constexpr (sizeof(real) == 4) a = warp_sumf(a);
        else a = warp_sum(a);
        if (l == 0) partial[((long long)b * nchunk + chunk) * Kmax + j] = (double)a;
    }
}

// ------------------------------------------------ Solve-OF: projection and new Gram column in one pass
// For every frame pair b (p = q = 2 GKS, one basis V of K vectors of [2][ns] values):
//   x' = r - V d                                (d = Mg^-1 V^T r, the projection coefficients)
//   y  = Ups^T Ups x'                           (pointwise: u_c (u_x x'_x + u_y x'_y))
//   dots  V^T x', V^T y, V^T q                  (q = L^T L r, the graph Laplacian of r, precomputed)
//   scalars ||x'||^2, x'^T y, x'^T q, x'^T Ups^T b
// A CTA owns OPX pixels of both components: TMA bulk copies stage, for each basis vector and for
// r and q and Ups^T b, the two 1 KB segments of those pixels, and the segments of u_x and u_y,
// completing on one mbarrier (bounded wait). The chunk partials (3 Kmax + 4 per chunk,
// FP32 16-element partials accumulated with their rounding errors, FP64 across lanes) are
// reduced by k_of_pass_reduce. With x' = r - V d the new vector is v = x' / ||x'|| and its Gram
// column follows from these without another pass over the basis (k_of_pass_finish):
//   G_A[i][v] = (V^T y)_i / ||x'||,   G_L[i][v] = ((V^T q)_i - (G_L d)_i) / ||x'||,
//   g[v] = x'^T Ups^T b / ||x'||,     G_A[v][v] = x'^T y / ||x'||^2,
//   G_L[v][v] = (x'^T q - d^T V^T q + d^T G_L d) / ||x'||^2,   Mg[i][v] = (V^T x')_i / ||x'||.
constexpr int OP_T = 128;  // threads per CTA
template <typename real>
constexpr int opx() { return 1024 / (int)sizeof(real); }  // pixels per CTA: 256 (FP32), 128 (FP64): 1 KB copies

long long of_pass_chunks(long long ns, int elem_bytes) { return (ns * elem_bytes + 1023) / 1024; }
int of_pass_stride(int Kmax) { return 3 * Kmax + 4; }

template <typename real>
__global__ void __launch_bounds__(OP_T) k_of_proj_gram_pass(const real *__restrict__ V, long long ns, int Kmax,
                                                           const int *__restrict__ K, const int *__restrict__ act,
                                                           const double *__restrict__ d, real *x, const real *__restrict__ q,
                                                           const real *__restrict__ AtB, const real *__restrict__ ux,
                                                           const real *__restrict__ uy, double *__restrict__ partial,
                                                           int nchunk, int *__restrict__ err, int kcap) {
    constexpr int PX = opx<real>(), CH = 2 * PX;  // elements of one vector in the tile
    constexpr int EPT = CH / OP_T;                // 4 (FP32) or 2 (FP64): 16 bytes per thread
    using vec_t = typename std::conditional<sizeof(real) == 4, float4, double2>::type;
    extern __shared__ __align__(128) unsigned char op_smem[];
    real *sx = reinterpret_cast<real *>(op_smem);  // [CH] r, then x'
    real *sq = sx + CH, *sa = sq + CH;             // [CH] q, Ups^T b
    real *sfx = sa + CH, *sfy = sfx + PX;           // [PX] u_x, u_y
    real *sy = sfy + PX;                            // [CH] y
    real *sV = sy + CH;                             // [kcap][CH]
    __shared__ real sd[64];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ double s_red[OP_T / 32][4];
    const int b = blockIdx.y, chunk = blockIdx.x, tid = threadIdx.x;
    if (act && !act[b]) return;
    int Kb = min(K[b], Kmax);
    if (Kb > kcap) {
        if (tid == 0 && err) atomicOr(err, 8);
        Kb = kcap;
    }
    const long long p0 = (long long)chunk * PX;
    const int len = (int)min((long long)PX, ns - p0);  // pixels of this chunk (a multiple of 16 bytes)
    const unsigned bar_a = smem_u32(&bar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const unsigned bytes = (unsigned)len * (unsigned)sizeof(real);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a),
                     "r"(bytes * (unsigned)(2 * Kb + 8))
                     : "memory");
        const long long N2 = 2 * ns;
        const real *xb = x + b * N2, *qb = q + b * N2, *ab = AtB + b * N2;
        bulk_g2s(sx, xb + p0, bytes, bar_a);
        bulk_g2s(sx + PX, xb + ns + p0, bytes, bar_a);
        bulk_g2s(sq, qb + p0, bytes, bar_a);
        bulk_g2s(sq + PX, qb + ns + p0, bytes, bar_a);
        bulk_g2s(sa, ab + p0, bytes, bar_a);
        bulk_g2s(sa + PX, ab + ns + p0, bytes, bar_a);
        bulk_g2s(sfx, ux + b * ns + p0, bytes, bar_a);
        bulk_g2s(sfy, uy + b * ns + p0, bytes, bar_a);
        const real *Vb = V + (long long)b * Kmax * N2;
        for (int j = 0; j < Kb; ++j) {
            bulk_g2s(sV + (long long)j * CH, Vb + (long long)j * N2 + p0, bytes, bar_a);
            bulk_g2s(sV + (long long)j * CH + PX, Vb + (long long)j * N2 + ns + p0, bytes, bar_a);
        }
    }
    for (int j = tid; j < Kb; j += OP_T) sd[j] = (real)d[(long long)b * Kmax + j];
    __syncthreads();
    if (!mbar_wait(bar_a, 0, g_wait_polls)) {
        if (tid == 0 && err) atomicOr(err, 4);
        mbar_wait(bar_a, 0);
        return;
    }
    // x' = r - V d on this thread's EPT consecutive elements (comp = i0 / PX)
    const int i0 = tid * EPT, pix0 = i0 % PX;
    {
        real acc[EPT];
#pragma unroll
        for (int e = 0; e < EPT; ++e) acc[e] = 0;
        for (int j = 0; j < Kb; ++j) {
            const vec_t v = *reinterpret_cast<const vec_t *>(sV + (long long)j * CH + i0);
            const real *vv = reinterpret_cast<const real *>(&v);
            const real dj = sd[j];
#pragma unroll
            for (int e = 0; e < EPT; ++e) acc[e] += vv[e] * dj;
        }
        vec_t xv = *reinterpret_cast<const vec_t *>(sx + i0);
        real *xx = reinterpret_cast<real *>(&xv);
#pragma unroll
        for (int e = 0; e < EPT; ++e) xx[e] = (pix0 + e < len) ? xx[e] - acc[e] : (real)0;
        *reinterpret_cast<vec_t *>(sx + i0) = xv;
        real *ob = x + b * 2 * ns + (i0 < PX ? 0 : ns) + p0 + pix0;
        if (pix0 + EPT <= len) {
            *reinterpret_cast<vec_t *>(ob) = xv;
        } else {
#pragma unroll
            for (int e = 0; e < EPT; ++e)
                if (pix0 + e < len) ob[e] = xx[e];
        }
    }
    __syncthreads();
    // y = Ups^T Ups x' and the four scalars
    double s4[4] = {0.0, 0.0, 0.0, 0.0};
    {
        real a4[4] = {0, 0, 0, 0};
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const int i = i0 + e, p = i % PX;
            real yv = 0;
            if (p < len) {
                const real w = sfx[p] * sx[p] + sfy[p] * sx[PX + p];
                yv = (i < PX ? sfx[p] : sfy[p]) * w;
            }
            sy[i] = yv;
            if (p < len) {  // the tile beyond len holds no copied data
                const real xi = sx[i];
                a4[0] += xi * xi;
                a4[1] += xi * yv;
                a4[2] += xi * sq[i];
                a4[3] += xi * sa[i];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if constexpr (sizeof(real) == 4) s4[k] = (double)warp_sumf(a4[k]);
            else s4[k] = warp_sum(a4[k]);
        }
    }
    const int w = tid >> 5, l = tid & 31;
    if (l == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) s_red[w][k] = s4[k];
    __syncthreads();
    // partials stored output-major, [b][output][chunk], so that the reduction reads each
    // output's chunks contiguously
    double *out = partial + (long long)b * (3 * Kmax + 4) * nchunk + chunk;
    if (tid < 4) {
        double t = 0.0;
        for (int ww = 0; ww < OP_T / 32; ++ww) t += s_red[ww][tid];
        out[(long long)(3 * Kmax + tid) * nchunk] = t;
    }
    // dots of every basis vector with x', y and q: warp w takes j = w, w + 2, ...; lane l holds
    // the elements l + 32 e of x', y, q in registers (consecutive lanes read consecutive words:
    // no bank conflicts); elements beyond the chunk's pixels count as zero
    constexpr int LE = CH / 32;
    real rx[LE], ry[LE], rq[LE];
#pragma unroll
    for (int e = 0; e < LE; ++e) {
        const int i = l + 32 * e;
        const bool in = (i % PX) < len;
        rx[e] = in ? sx[i] : (real)0;
        ry[e] = in ? sy[i] : (real)0;
        rq[e] = in ? sq[i] : (real)0;
    }
    for (int j = w; j < Kb; j += OP_T / 32) {
        const real *vj = sV + (long long)j * CH + l;
        real t1 = 0, t2 = 0, t3 = 0;
#pragma unroll
        for (int e = 0; e < LE; ++e) {
            if (((l + 32 * e) % PX) < len) {
                const real v = vj[32 * e];
                t1 += v * rx[e];
                t2 += v * ry[e];
                t3 += v * rq[e];
            }
        }
        // the warp's partial sums in the storage precision (FP64 work is slow on this GPU), then
        // FP64 across the chunks
        double o1, o2, o3;
        if constexpr (sizeof(real) == 4) {
            o1 = (double)warp_sumf(t1);
            o2 = (double)warp_sumf(t2);
            o3 = (double)warp_sumf(t3);
        } else {
            o1 = warp_sum(t1);
            o2 = warp_sum(t2);
            o3 = warp_sum(t3);
        }
        if (l == 0) {
            out[(long long)j * nchunk] = o1;
            out[(long long)(Kmax + j) * nchunk] = o2;
            out[(long long)(2 * Kmax + j) * nchunk] = o3;
        }
    }
}

// sums of the chunk partials of k_of_proj_gram_pass in FP64 (one warp per output, lanes over
// its contiguous chunks, fixed order): res[b][0..3 Kmax + 4)
__global__ void k_of_pass_reduce(const double *__restrict__ partial, int nchunk, int Kmax, const int *__restrict__ K,
                                 const int *__restrict__ act, double *__restrict__ res) {
    const int b = blockIdx.y;
    if (act && !act[b]) return;
    const int stride = 3 * Kmax + 4, Kb = min(K[b], Kmax);
    const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (o >= stride) return;
    const int j = o < 3 * Kmax ? o % Kmax : 0;
    if (o < 3 * Kmax && j >= Kb) return;
    const double *src = partial + ((long long)b * stride + o) * nchunk;
    double sum = 0.0;
#pragma unroll 8
    for (int c = lane; c < nchunk; c += 32) sum += src[c];
    sum = warp_sum(sum);
    if (lane == 0) res[(long long)b * stride + o] = sum;
}

// ||x[b]||^2 per chunk
template <typename real, bool EXACT = false>
__global__ void __launch_bounds__(KT) k_norm2(const real *__restrict__ x, long long N, long long xstride,
                                              double *__restrict__ partial, int nchunk) {
    __shared__ double sh[KT / 32];
    const int b = blockIdx.y, chunk = blockIdx.x;
    const long long i0 = (long long)chunk * CHUNK + threadIdx.x;
    if constexpr (EXACT && sizeof(real) == 4) {
        DFAcc a;
#pragma unroll
        for (int e = 0; e < KE; ++e) {
            const long long i = i0 + (long long)e * KT;
            if (i < N) {
                const float v = x[b * xstride + i];
                a.add_prod(v, v);
            }
        }
        const double s = block_sum_to_double(a.value(), sh);
        if (threadIdx.x == 0) partial[(long long)b * nchunk + chunk] = s;
        return;
    }
    real n2 = 0;
#pragma unroll
    for (int e = 0; e < KE; ++e) {
        const long long i = i0 + (long long)e * KT;
        if (i < N) {
            const real v = x[b * xstride + i];
            n2 += v * v;
        }
    }
    const double s = block_sum_to_double(n2, sh);
    if (threadIdx.x == 0) partial[(long long)b * nchunk + chunk] = s;
}

// out[b] = sum_chunk partial[b][chunk], one warp per problem
__global__ void k_sum_scalar_chunks(const double *__restrict__ partial, int nchunk, double *__restrict__ out, int B) {
    const int b = blockIdx.x, lane = threadIdx.x;
    if (b >= B) return;
    double s = 0.0;
#pragma unroll 8
    for (int c = lane; c < nchunk; c += 32) s += partial[(long long)b * nchunk + c];
    s = warp_sum(s);
    if (lane == 0) out[b] = s;
}

// Append x[b] / ||x[b]|| as vector K[b] when ||x[b]|| > tol * scale[b] and the
// problem is still growing (scale == null: only ||x|| > 0 is required); the
// new vector is also written to stage[b] when stage != null.
__device__ __forceinline__ bool append_ok(int grow, int Kb, int Kmax, double nrm2, const double *scale, int b, double tol) {
    const double nr = sqrt(nrm2);
    const double sc = scale ? scale[b] : 0.0;
    return grow && Kb < Kmax && (nr > tol * sc) && (nr > 0.0) && isfinite(nr);
}

// The per-problem decision and scale of an append, once per problem (FP64):
// slot[b] = K[b] and inv[b] = 1/||x[b]|| when the vector is appended (then
// K[b] += 1), slot[b] = -1 and grow[b] = 0 otherwise; appended[b] (may be
// null) records which. k_append's threads then do no FP64 arithmetic.
template <typename real>
__global__ void k_append_prep(int *__restrict__ K, int Kmax, const double *__restrict__ nrm2, const double *__restrict__ scale,
                              double tol, int *__restrict__ grow, int B, int *__restrict__ slot, real *__restrict__ inv,
                              int *__restrict__ appended) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int Kb = K[b];
    const bool ok = append_ok(grow[b], Kb, Kmax, nrm2[b], scale, b, tol);
    slot[b] = ok ? Kb : -1;
    inv[b] = ok ? (real)(1.0 / sqrt(nrm2[b])) : (real)0;
    if (ok) K[b] = Kb + 1;
    else grow[b] = 0;
    if (appended) appended[b] = ok;
}

// The same with ||x[b]||^2 summed here from the per-block partials of the update
// that formed x (one warp per problem, lanes over the partials, then a fixed tree:
// the order of k_sum_scalar_chunks), written to nrm2_out, and sqrt(||x[b]||^2)
// written to sq1[b] and sq2[b] (each may be null) for problems still growing
// (grow[b] as it was on entry).
template <typename real>
__global__ void k_append_prep_sum(int *__restrict__ K, int Kmax, const double *__restrict__ parts, int nparts,
                                  double *__restrict__ nrm2_out, const double *__restrict__ scale, double tol,
                                  int *__restrict__ grow, int B, int *__restrict__ slot, real *__restrict__ inv,
                                  int *__restrict__ appended, double *__restrict__ sq1, double *__restrict__ sq2) {
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (b >= B) return;
    double s = 0.0;
#pragma unroll 8
    for (int c = lane; c < nparts; c += 32) s += parts[(long long)b * nparts + c];
    s = warp_sum(s);
    if (lane != 0) return;
    nrm2_out[b] = s;
    const int g = grow[b];
    if (g) {
        const double r = sqrt(s);
        if (sq1) sq1[b] = r;
        if (sq2) sq2[b] = r;
    }
    const int Kb = K[b];
    const bool ok = append_ok(g, Kb, Kmax, s, scale, b, tol);
    slot[b] = ok ? Kb : -1;
    inv[b] = ok ? (real)(1.0 / sqrt(s)) : (real)0;
    if (ok) K[b] = Kb + 1;
    else grow[b] = 0;
    if (appended) appended[b] = ok;
}

template <typename real>
__global__ void __launch_bounds__(KT) k_append(real *__restrict__ V, long long N, int Kmax, const int *__restrict__ slot,
                                               const real *__restrict__ inv, const real *__restrict__ x, long long xstride,
                                               real *__restrict__ stage) {
    const int b = blockIdx.y;
    const int sl = slot[b];
    if (sl < 0) return;
    const real iv = inv[b];
    real *vd = V + ((long long)b * Kmax + sl) * N;
    for (long long i = blockIdx.x * (long long)KT + threadIdx.x; i < N; i += (long long)gridDim.x * KT) {
        const real v = x[b * xstride + i] * iv;
        vd[i] = v;
        if (stage) stage[b * N + i] = v;
    }
}

mof_status set_wait_polls(long long polls) {
    const long long v = polls < 0 ? MBAR_MAX_POLLS : (polls > MBAR_MAX_POLLS ? MBAR_MAX_POLLS : polls);
    MOF_CUDA(cudaMemcpyToSymbol(g_wait_polls, &v, sizeof(v)));
    MOF_CUDA(cudaDeviceSynchronize());
    return MOF_OK;
}

// ------------------------------------------------------------ host launchers
template <typename real>
void Krylov<real>::dots(const BasisRef<real> &B, const real *x, long long xstride, double *out, long long ostride, double sign,
                        cudaStream_t st) const {
    DotVecs<real> xs{};
    xs.x[0] = x;
    xs.stride[0] = xstride;
    DotOuts o{};
    o.o[0] = DotOut{out, ostride, 1, 0, 0, sign};
    multidot(B, 1, xs, o, st);
}

template <typename real>
static bool vec_ok(const void *base, long long N, long long stride) {
    return sizeof(real) == 4 && (N % 4) == 0 && (stride % 4) == 0 && (reinterpret_cast<uintptr_t>(base) % 16) == 0;
}

template <typename real>
void Krylov<real>::multidot(const BasisRef<real> &B, int nv, const DotVecs<real> &xs, const DotOuts &outs,
                            cudaStream_t st, bool exact) const {
    const int nc = (int)mdot_chunks<real>(B.N);
    const dim3 grid(nc, B.B);
    const bool vec = vec_ok<real>(B.V, B.N, (long long)B.Kmax * B.N);
#define MDOT(NVv)                                                                                                       \
    if (exact) ::mof::count_launch(), k_mdot<real, NVv, false, true><<<grid, KT, 0, st>>>(B.V, B.N, B.Kmax, B.K, B.act, xs, partial, nc); \
    else if (vec) ::mof::count_launch(), k_mdot<real, NVv, true><<<grid, KT, 0, st>>>(B.V, B.N, B.Kmax, B.K, B.act, xs, partial, nc); \
    else ::mof::count_launch(), k_mdot<real, NVv, false><<<grid, KT, 0, st>>>(B.V, B.N, B.Kmax, B.K, B.act, xs, partial, nc);
    if (nv == 1) {
        MDOT(1)
    } else if (nv == 2) {
        MDOT(2)
    } else {
        MDOT(3)
    }
#undef MDOT
    ::mof::count_launch(), k_sum_chunks<<<dim3((nv * B.Kmax + SUMT / 32 - 1) / (SUMT / 32), B.B), SUMT, 0, st>>>(partial, nc, nv, B.Kmax, B.K, B.act, outs);
}

template <typename real>
void Krylov<real>::combine(const BasisRef<real> &B, const double *c, long long cstride, real *out, long long ostride,
                           cudaStream_t st) const {
    const int nb = (int)((B.N + 4LL * CT - 1) / (4LL * CT));
    const bool vec = vec_ok<real>(B.V, B.N, (long long)B.Kmax * B.N) && (ostride % 4 == 0);
    if (vec)
        ::mof::count_launch(), k_combine<real, 0, true><<<dim3(nb, B.B), CT, 0, st>>>(B.V, B.N, B.Kmax, B.K, B.act, c, cstride,
                                                                                   nullptr, 0, out, ostride, nullptr, nb);
    else
        ::mof::count_launch(), k_combine<real, 0, false><<<dim3(nb, B.B), CT, 0, st>>>(B.V, B.N, B.Kmax, B.K, B.act, c, cstride,
                                                                                    nullptr, 0, out, ostride, nullptr, nb);
}

template <typename real>
void Krylov<real>::combine_minus(const BasisRef<real> &B, const double *c, long long cstride, const real *x, long long xstride,
                                 real *out, long long ostride, double *nrm2_out, cudaStream_t st) const {
    const int nb = (int)((B.N + 4LL * CT - 1) / (4LL * CT));
    const bool vec = vec_ok<real>(B.V, B.N, (long long)B.Kmax * B.N) && (ostride % 4 == 0);
    double *np = nrm2_out ? partial : nullptr;
    if (vec)
        ::mof::count_launch(), k_combine<real, 2, true><<<dim3(nb, B.B), CT, 0, st>>>(B.V, B.N, B.Kmax, B.K, B.act, c, cstride, x,
                                                                                   xstride, out, ostride, np, nb);
    else
        ::mof::count_launch(), k_combine<real, 2, false><<<dim3(nb, B.B), CT, 0, st>>>(B.V, B.N, B.Kmax, B.K, B.act, c, cstride, x,
                                                                                    xstride, out, ostride, np, nb);
    if (nrm2_out) ::mof::count_launch(), k_sum_scalar_chunks<<<B.B, 32, 0, st>>>(partial, nb, nrm2_out, B.B);
}

template <typename real>
void Krylov<real>::subtract(const BasisRef<real> &B, const double *c, long long cstride, const real *x, long long xstride,
                            real *out, long long ostride, double *nrm2_out, cudaStream_t st) const {
    const int nb = (int)((B.N + 4LL * CT - 1) / (4LL * CT));
    const bool vec = vec_ok<real>(B.V, B.N, (long long)B.Kmax * B.N) && (ostride % 4 == 0);
    double *np = nrm2_out ? partial : nullptr;
    if (vec)
        ::mof::count_launch(), k_combine<real, 1, true><<<dim3(nb, B.B), CT, 0, st>>>(B.V, B.N, B.Kmax, B.K, B.act, c, cstride, x,
                                                                                   xstride, out, ostride, np, nb);
    else
        ::mof::count_launch(), k_combine<real, 1, false><<<dim3(nb, B.B), CT, 0, st>>>(B.V, B.N, B.Kmax, B.K, B.act, c, cstride, x,
                                                                                    xstride, out, ostride, np, nb);
    if (nrm2_out) ::mof::count_launch(), k_sum_scalar_chunks<<<B.B, 32, 0, st>>>(partial, nb, nrm2_out, B.B);
}

template <typename real>
int Krylov<real>::subtract_parts(const BasisRef<real> &B, const double *c, long long cstride, const real *x, long long xstride,
                                 real *out, long long ostride, cudaStream_t st) const {
    const int nb = (int)((B.N + 4LL * CT - 1) / (4LL * CT));
    const bool vec = vec_ok<real>(B.V, B.N, (long long)B.Kmax * B.N) && (ostride % 4 == 0);
    if (vec)
        ::mof::count_launch(), k_combine<real, 1, true><<<dim3(nb, B.B), CT, 0, st>>>(B.V, B.N, B.Kmax, B.K, B.act, c, cstride, x,
                                                                                   xstride, out, ostride, partial, nb);
    else
        ::mof::count_launch(), k_combine<real, 1, false><<<dim3(nb, B.B), CT, 0, st>>>(B.V, B.N, B.Kmax, B.K, B.act, c, cstride, x,
                                                                                    xstride, out, ostride, partial, nb);
    return nb;
}

template <typename real>
void Krylov<real>::norm2(const real *x, long long N, long long xstride, int nb, double *out, cudaStream_t st,
                         bool exact) const {
    const int nc = (int)krylov_chunks(N);
    if (exact) ::mof::count_launch(), k_norm2<real, true><<<dim3(nc, nb), KT, 0, st>>>(x, N, xstride, partial, nc);
    else ::mof::count_launch(), k_norm2<real><<<dim3(nc, nb), KT, 0, st>>>(x, N, xstride, partial, nc);
    ::mof::count_launch(), k_sum_scalar_chunks<<<nb, 32, 0, st>>>(partial, nc, out, nb);
}

template <typename real>
bool Krylov<real>::sub_dot(const BasisRef<real> &B, const double *c, long long cstride, real *x, long long xstride,
                           double *out, cudaStream_t st, int kcap, int *nparts) const {
    const long long es = sizeof(real);
    const bool ok = B.Kmax <= 64 && (B.N * es) % 16 == 0 && (xstride * es) % 16 == 0 &&
                    (reinterpret_cast<uintptr_t>(B.V) % 16) == 0 && (reinterpret_cast<uintptr_t>(x) % 16) == 0;
    if (!ok) return false;
    static std::atomic<bool> configured{false};
    if (!configured.load()) {  // the largest tile this instantiation can need (65 chunks)
        if (cudaFuncSetAttribute(k_sub_dot<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65 * SD_BYTES) != cudaSuccess)
            return false;
        configured.store(true);
    }
    const int nc = (int)subdot_chunks(B.N, (int)es);
    const int kc = kcap > 0 ? std::min(kcap, B.Kmax) : B.Kmax;  // vectors the tile holds
    const size_t smem = (size_t)(kc + 1) * SD_BYTES;
    ::mof::count_launch(), k_sub_dot<real><<<dim3(nc, B.B), SDT, smem, st>>>(B.V, B.N, B.Kmax, B.K, B.act, c, cstride, x, xstride,
                                                                         x, xstride, partial, nc, err, kc,
                                                                         nparts ? partial + (long long)B.B * nc * B.Kmax : nullptr);
    DotOuts o{};
    o.o[0] = DotOut{out, B.Kmax, 1, 0, 0, 1.0};
    ::mof::count_launch(), k_sum_chunks<<<dim3((B.Kmax + SUMT / 32 - 1) / (SUMT / 32), B.B), SUMT, 0, st>>>(partial, nc, 1, B.Kmax,
                                                                                                          B.K, B.act, o);
    if (nparts) *nparts = nc;
    return true;
}

template <typename real>
void Krylov<real>::reorth(const BasisRef<real> &B, real *x, long long xstride, double *coef, double *nrm2_out,
                          cudaStream_t st) const {
    // classical Gram-Schmidt against V, twice (CGS2); coef is [B][Kmax] scratch
    dots(B, x, xstride, coef, B.Kmax, 1.0, st);
    reorth_second(B, x, xstride, coef, coef, nrm2_out, st);
}

template <typename real>
void Krylov<real>::reorth_second(const BasisRef<real> &B, real *x, long long xstride, const double *c1, double *coef,
                                 double *nrm2_out, cudaStream_t st, int kcap) const {
    // the first projection's coefficients are given (c1; null: zero), the second are
    // taken by dot products, fused with the first update where the layout allows
    if (c1) {
        if (!sub_dot(B, c1, B.Kmax, x, xstride, coef, st, kcap)) {
            subtract(B, c1, B.Kmax, x, xstride, x, xstride, nullptr, st);
            dots(B, x, xstride, coef, B.Kmax, 1.0, st);
        }
    } else {
        dots(B, x, xstride, coef, B.Kmax, 1.0, st);
    }
    subtract(B, coef, B.Kmax, x, xstride, x, xstride, nrm2_out, st);
}

template <typename real>
int Krylov<real>::reorth_second_parts(const BasisRef<real> &B, real *x, long long xstride, const double *c1, double *coef,
                                      cudaStream_t st, int kcap) const {
    if (c1) {
        if (!sub_dot(B, c1, B.Kmax, x, xstride, coef, st, kcap)) {
            subtract(B, c1, B.Kmax, x, xstride, x, xstride, nullptr, st);
            dots(B, x, xstride, coef, B.Kmax, 1.0, st);
        }
    } else {
        dots(B, x, xstride, coef, B.Kmax, 1.0, st);
    }
    return subtract_parts(B, coef, B.Kmax, x, xstride, x, xstride, st);
}

template <typename real>
void Krylov<real>::append_parts(const BasisRef<real> &B, int *Kmut, const real *x, long long xstride, int nparts,
                                double *nrm2_out, const double *scale, double tol, int *grow, int *appended, real *stage,
                                double *sq1, double *sq2, cudaStream_t st, const double *parts) const {
    int *slot = reinterpret_cast<int *>(aux);
    real *inv = reinterpret_cast<real *>(aux + B.B);
    ::mof::count_launch(), k_append_prep_sum<real><<<(B.B + 1) / 2, 64, 0, st>>>(Kmut, B.Kmax, parts ? parts : partial, nparts,
                                                                                nrm2_out, scale, tol, grow, B.B, slot, inv,
                                                                                appended, sq1, sq2);
    const int blocks = (int)std::min<long long>(1024, (B.N + KT - 1) / KT);
    ::mof::count_launch(), k_append<real><<<dim3(blocks, B.B), KT, 0, st>>>(B.V, B.N, B.Kmax, slot, inv, x, xstride, stage);
}

template <typename real>
void Krylov<real>::append(const BasisRef<real> &B, int *Kmut, const real *x, long long xstride, const double *nrm2,
                          const double *scale, double tol, int *grow, int *appended, real *stage, cudaStream_t st) const {
    int *slot = reinterpret_cast<int *>(aux);
    real *inv = reinterpret_cast<real *>(aux + B.B);
    ::mof::count_launch(), k_append_prep<real><<<(B.B + 63) / 64, 64, 0, st>>>(Kmut, B.Kmax, nrm2, scale, tol, grow, B.B, slot, inv,
                                                                              appended);
    const int blocks = (int)std::min<long long>(1024, (B.N + KT - 1) / KT);
    ::mof::count_launch(), k_append<real><<<dim3(blocks, B.B), KT, 0, st>>>(B.V, B.N, B.Kmax, slot, inv, x, xstride, stage);
}

// Per pair (one warp): the append decision on ||x'|| (as k_append_prep), and for an appended
// vector v = x' / ||x'||, its Gram columns G_A, G_L, g, its Euclidean overlaps Mg and the slot
// and scale of k_append (see k_of_proj_gram_pass for the formulas).
template <typename real>
__global__ void k_of_pass_finish(const double *__restrict__ res, const double *__restrict__ d, int Kmax, int *__restrict__ K,
                                 const int *__restrict__ act, const double *__restrict__ scale, double tol,
                                 int *__restrict__ grow, double *__restrict__ GA, double *__restrict__ GL,
                                 double *__restrict__ g, double *__restrict__ Mg, double *__restrict__ nrm2_out,
                                 int *__restrict__ appended, int *__restrict__ slot, real *__restrict__ inv) {
    const int b = blockIdx.x, lane = threadIdx.x;
    if (act && !act[b]) {
        if (lane == 0) {
            slot[b] = -1;
            if (appended) appended[b] = 0;
        }
        return;
    }
    const int stride = 3 * Kmax + 4, Kb = min(K[b], Kmax);
    const double *rs = res + (long long)b * stride;
    const double *c2 = rs, *ay = rs + Kmax, *aq = rs + 2 * Kmax, *sc = rs + 3 * Kmax;
    const double *db = d + (long long)b * Kmax;
    const long long KK = (long long)Kmax * Kmax;
    double *A = GA + b * KK, *L = GL + b * KK, *M = Mg + b * KK;
    const double nr2 = sc[0];
    const bool ok = append_ok(grow[b], Kb, Kmax, nr2, scale, b, tol);
    // (G_L d)_i and d^T (V^T q) - d^T G_L d for the new column of G_L
    double dq = 0.0, dGd = 0.0;
    for (int i = lane; i < Kb; i += 32) {
        double gd = 0.0;
        for (int k = 0; k < Kb; ++k) gd += L[(long long)i * Kmax + k] * db[k];
        dq += db[i] * aq[i];
        dGd += db[i] * gd;
    }
    dq = warp_sum(dq);
    dGd = warp_sum(dGd);
    if (ok) {
        const double ib = 1.0 / sqrt(nr2), ib2 = 1.0 / nr2;
        for (int i = lane; i < Kb; i += 32) {
            double gd = 0.0;
            for (int k = 0; k < Kb; ++k) gd += L[(long long)i * Kmax + k] * db[k];
            const double va = ay[i] * ib, vl = (aq[i] - gd) * ib, vm = c2[i] * ib;
            A[(long long)i * Kmax + Kb] = va;
            A[(long long)Kb * Kmax + i] = va;
            L[(long long)i * Kmax + Kb] = vl;
            L[(long long)Kb * Kmax + i] = vl;
            M[(long long)i * Kmax + Kb] = vm;
            M[(long long)Kb * Kmax + i] = vm;
        }
        __syncwarp();
        if (lane == 0) {
            A[(long long)Kb * Kmax + Kb] = sc[1] * ib2;
            L[(long long)Kb * Kmax + Kb] = (sc[2] - dq + dGd) * ib2;
            M[(long long)Kb * Kmax + Kb] = 1.0;
            g[(long long)b * Kmax + Kb] = sc[3] * ib;
        }
    }
    if (lane == 0) {
        nrm2_out[b] = nr2;
        slot[b] = ok ? Kb : -1;
        inv[b] = ok ? (real)(1.0 / sqrt(nr2)) : (real)0;
        if (ok) K[b] = Kb + 1;
        else grow[b] = 0;
        if (appended) appended[b] = ok;
    }
}

// q[b] = L^T L r[b] on both components (the graph Laplacian with free boundary, one thread
// per pixel and component)
template <typename real>
__global__ void k_of_lap(const real *__restrict__ r, real *__restrict__ q, int nx, int ny, const int *__restrict__ act) {
    const int b = blockIdx.z >> 1, c = blockIdx.z & 1;
    if (act && !act[b]) return;
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const long long ns = (long long)nx * ny, i = (long long)y * nx + x;
    const real *f = r + (2LL * b + c) * ns;
    const real v0 = f[i];
    real v = 0;
    if (x > 0) v += v0 - f[i - 1];
    if (x < nx - 1) v += v0 - f[i + 1];
    if (y > 0) v += v0 - f[i - nx];
    if (y < ny - 1) v += v0 - f[i + nx];
    q[(2LL * b + c) * ns + i] = v;
}

template <typename real>
bool of_pass_applicable(long long ns, const void *V, const void *x) {
    const long long es = sizeof(real);
    return (ns * es) % 16 == 0 && (reinterpret_cast<uintptr_t>(V) % 16) == 0 && (reinterpret_cast<uintptr_t>(x) % 16) == 0;
}

template <typename real>
mof_status launch_of_proj_gram_pass(const BasisRef<real> &B, int *Kmut, long long ns, int nx, int ny, const double *d, real *x,
                                    real *q, const real *AtB, const real *ux, const real *uy, double *partial,
                                    double *res, int *err, int kcap, const double *scale, double tol, int *grow,
                                    double *GA, double *GL, double *g, double *Mg, double *nrm2_out, int *appended,
                                    double *aux, cudaStream_t st) {
    static std::atomic<bool> configured{false};
    if (!configured.load()) {
        if (cudaFuncSetAttribute(k_of_proj_gram_pass<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, 140 * 1024) !=
            cudaSuccess)
            return fail(MOF_ECUDA, "shared-memory attribute of the Solve-OF pass");
        configured.store(true);
    }
    const int nc = (int)of_pass_chunks(ns, (int)sizeof(real));
    const int kc = kcap > 0 ? std::min(kcap, B.Kmax) : B.Kmax;
    const size_t smem = (size_t)(kc + 5) * 2048;
    const dim3 lg((nx + 31) / 32, (ny + 7) / 8, 2 * B.B);
    ::mof::count_launch(), k_of_lap<real><<<lg, dim3(32, 8), 0, st>>>(x, q, nx, ny, B.act);
    ::mof::count_launch(), k_of_proj_gram_pass<real><<<dim3(nc, B.B), OP_T, smem, st>>>(B.V, ns, B.Kmax, B.K, B.act, d, x, q, AtB,
                                                                                     ux, uy, partial, nc, err, kc);
    const int stride = of_pass_stride(B.Kmax);
    ::mof::count_launch(), k_of_pass_reduce<<<dim3((stride + 7) / 8, B.B), 256, 0, st>>>(partial, nc, B.Kmax, B.K, B.act, res);
    int *slot = reinterpret_cast<int *>(aux);
    real *inv = reinterpret_cast<real *>(aux + B.B);
    ::mof::count_launch(), k_of_pass_finish<real><<<B.B, 32, 0, st>>>(res, d, B.Kmax, Kmut, B.act, scale, tol, grow, GA, GL, g,
                                                                     Mg, nrm2_out, appended, slot, inv);
    const int blocks = (int)std::min<long long>(1024, (B.N + KT - 1) / KT);
    ::mof::count_launch(), k_append<real><<<dim3(blocks, B.B), KT, 0, st>>>(B.V, B.N, B.Kmax, slot, inv, x, B.N, nullptr);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

template bool of_pass_applicable<float>(long long, const void *, const void *);
template bool of_pass_applicable<double>(long long, const void *, const void *);
template mof_status launch_of_proj_gram_pass<float>(const BasisRef<float> &, int *, long long, int, int, const double *, float *,
                                                    float *, const float *, const float *, const float *, double *, double *,
                                                    int *, int, const double *, double, int *, double *, double *, double *,
                                                    double *, double *, int *, double *, cudaStream_t);
template mof_status launch_of_proj_gram_pass<double>(const BasisRef<double> &, int *, long long, int, int, const double *, double *,
                                                     double *, const double *, const double *, const double *, double *,
                                                     double *, int *, int, const double *, double, int *, double *, double *,
                                                     double *, double *, double *, int *, double *, cudaStream_t);

template struct Krylov<float>;
template struct Krylov<double>;

}  // namespace mof
