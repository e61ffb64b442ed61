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
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

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
        real a[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) a[v] = 0;
        if constexpr (VEC) {
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
                    a[v] += q0.x * y0.x + q0.y * y0.y + q0.z * y0.z + q0.w * y0.w;
                    a[v] += q1.x * y1.x + q1.y * y1.y + q1.z * y1.z + q1.w * y1.w;
                    a[v] += q2.x * y2.x + q2.y * y2.y + q2.z * y2.z + q2.w * y2.w;
                    a[v] += q3.x * y3.x + q3.y * y3.y + q3.z * y3.z + q3.w * y3.w;
                }
            }
            for (; i < n4; i += 32) {
                const float4 q = __ldcs(v4 + i);
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const float4 y = reinterpret_cast<const float4 *>(sx[v])[i];
                    a[v] += q.x * y.x + q.y * y.y + q.z * y.z + q.w * y.w;
                }
            }
        } else {
            for (int i = l; i < len; i += 32) {
                const real q = vj[i];
#pragma unroll
                for (int v = 0; v < NV; ++v) a[v] += q * sx[v][i];
            }
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
    const long long a = krylov_chunks(N) * 3 * Kmax, b = subdot_chunks(N, 8) * Kmax;
    return a > b ? a : b;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// poll the mbarrier phase with a bound; false when the bound ran out
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned phase) {
    for (long long it = 0; it < MBAR_MAX_POLLS; ++it) {
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
                                                 double *__restrict__ partial, int nchunk, int *__restrict__ err, int kcap) {
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
    if (!mbar_wait(bar_a, 0)) {
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
                           double *out, cudaStream_t st, int kcap) const {
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
                                                                         x, xstride, partial, nc, err, kc);
    DotOuts o{};
    o.o[0] = DotOut{out, B.Kmax, 1, 0, 0, 1.0};
    ::mof::count_launch(), k_sum_chunks<<<dim3((B.Kmax + SUMT / 32 - 1) / (SUMT / 32), B.B), SUMT, 0, st>>>(partial, nc, 1, B.Kmax,
                                                                                                          B.K, B.act, o);
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
                                double *sq1, double *sq2, cudaStream_t st) const {
    int *slot = reinterpret_cast<int *>(aux);
    real *inv = reinterpret_cast<real *>(aux + B.B);
    ::mof::count_launch(), k_append_prep_sum<real><<<(B.B + 1) / 2, 64, 0, st>>>(Kmut, B.Kmax, partial, nparts, nrm2_out, scale, tol,
                                                                                grow, B.B, slot, inv, appended, sq1, sq2);
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

template struct Krylov<float>;
template struct Krylov<double>;

}  // namespace mof
