// Solver layer of libmof: Solve-OF (Alg. 2) batched over all frame pairs,
// MMGKS-OF (Alg. 1), their workspace, and per-kernel-class timing.
//
// Every quantity that steers the iteration (basis sizes, growth flags,
// lambda, z, norms) lives in device memory, and every kernel reads it there:
// the host enqueues a fixed sequence of launches per outer iteration and
// synchronises only at the end of mof_solve.
#include "solver.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <string>
#include <vector>

namespace mof {

// ============================================================ kernel timing
struct Timer {
    std::vector<std::string> names;
    std::vector<double> ms;
    std::vector<long long> count;
    struct Pending {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    // While a graph is being captured, scopes record external event nodes into
    // the graph, with events owned by that graph (never reused elsewhere).
    std::vector<Pending> *sink = nullptr;
    std::vector<cudaEvent_t> *owned = nullptr;

    int cls(const char *name) {
        for (size_t i = 0; i < names.size(); ++i)
            if (names[i] == name) return (int)i;
        names.push_back(name);
        ms.push_back(0.0);
        count.push_back(0);
        return (int)names.size() - 1;
    }
    cudaEvent_t ev() {
        if (owned) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            owned->push_back(e);
            return e;
        }
        if (used == pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        return pool[used++];
    }
    void reset() {
        for (auto &v : ms) v = 0.0;
        for (auto &c : count) c = 0;
        pending.clear();
        used = 0;
    }
    void collect_list(const std::vector<Pending> &lst) {
        for (auto &p : lst) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
                ms[p.cls] += t;
                count[p.cls] += 1;
            }
        }
    }
    void collect() {
        collect_list(pending);
        pending.clear();
        used = 0;
    }
    ~Timer() {
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// Scoped timing of one launch group on `st` when timing is enabled.
struct Scope {
    Timer *t;
    int c;
    cudaEvent_t b;
    cudaStream_t st;
    Scope(Timer *tm, const char *name, cudaStream_t s) : t(tm), c(-1), b(nullptr), st(s) {
        if (!t) return;
        c = t->cls(name);
        cudaEvent_t a = t->ev();
        b = t->ev();
        if (t->sink) {
            cudaEventRecordWithFlags(a, st, cudaEventRecordExternal);
            t->sink->push_back({c, a, b});
        } else {
            cudaEventRecord(a, st);
            t->pending.push_back({c, a, b});
        }
    }
    ~Scope() {
        if (!t) return;
        if (t->sink) cudaEventRecordWithFlags(b, st, cudaEventRecordExternal);
        else cudaEventRecord(b, st);
    }
};

// ============================================================ workspace
struct Arena {
    char *base = nullptr;
    size_t off = 0, cap = 0;
    template <typename T>
    T *take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T *p = reinterpret_cast<T *>(base + off);
        off += sizeof(T) * count;
        return p;
    }
};

constexpr int MAX_OF_STREAMS = 64;
constexpr int AUTO_OF_STREAMS = 64;

template <typename real>
struct WS {
    int Kmax = 0, Kof = 0, of_ell = 0, ell = 0, max_outer = 0;
    char *mem = nullptr;
    size_t bytes = 0;
    // ---- image step (one problem)
    real *V, *HV, *U, *u, *un, *r, *tm, *tn, *b, *q, *uT, *s, *sr, *vnew, *hvnew;
    int *rad_s, *rad_sr, *rad_rev, *dest;
    double *GH, *GT, *gH, *z, *lam, *coef, *c1, *nrm2, *nrm2b, *scaleR, *alpha, *beta, *beta1, *alpha1, *bb, *gpart;
    int *K, *KU, *grow, *gkb, *flag, *err, *appended;
    double *report;  // [max_outer][8]
    // ---- Solve-OF (P pairs)
    real *ux, *uy, *ut, *bof, *Vof, *Uof, *AtB, *wv, *wu, *y1, *y2, *sof, *vnew_of, *q_of;
    double *GA, *GL, *gof, *zof, *gam, *nrm_of, *coef_of, *coefU_of, *scale_of, *alpha_of, *alpha1_of, *beta_of,
        *beta1_of, *bb_of, *Mg_of, *pres_of;
    int *Kv_of, *Ku_of, *grow_of, *gkb_of, *act_of, *app_of, *flag_of;
    real *wf_of = nullptr, *wl_of = nullptr;  // IRLS weights of Solve-OF with p = q = 1 (P ns, 4 P ns)
    double *rn_of = nullptr;                  // norm^2 of its residual before orthogonalisation (P)
    int pq1 = 0;                              // workspace holds the p = q = 1 arrays
    double *partial;
    double *kaux;  // Krylov append scratch, 2 per problem
    int *iter;  // device index of the outer iteration (report slot)
    int gram_ctas = 0;
    // one captured graph per outer-iteration variant: bit 0 Solve-OF, bit 1 expansion,
    // bit 2 timing scopes present
    struct IterGraph {
        cudaGraphExec_t exec = nullptr;
        long long kernels = 0;  // kernel nodes per replay
        std::vector<Timer::Pending> ev;
        std::vector<cudaEvent_t> owned;
    };
    IterGraph graphs[8];
    mof_solver_params gkey{};
    int gkey_n = -1;
    int gkey_wm = 0;                   // M(s) mode the graphs were captured with
    // the stand-alone Solve-OF (mof_solve_of), captured once per parameter set
    IterGraph ofgraph;
    mof_solver_params ofkey{};
    cudaStream_t ss = nullptr;  // internal stream (graphs cannot be captured on the legacy stream)
    cudaEvent_t join = nullptr;
    // Solve-OF pair groups: one stream each, forked from and joined to ss
    cudaStream_t gs[MAX_OF_STREAMS] = {};
    cudaEvent_t gfork = nullptr, gdone[MAX_OF_STREAMS] = {};
    // side stream of the image step (the Psi rows of the weighted Gram beside Solve-OF)
    cudaStream_t side = nullptr;
    cudaEvent_t side_fork = nullptr, side_done = nullptr;
    void drop_graphs() {
        for (auto &g : graphs) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            for (auto e : g.owned) cudaEventDestroy(e);
            g = IterGraph();
        }
        drop_of_graph();
    }
    void drop_of_graph() {
        if (ofgraph.exec) cudaGraphExecDestroy(ofgraph.exec);
        ofgraph = IterGraph();
    }
};

struct Holder {
    void *scr[SCR_COUNT] = {};
    WS<float> *w32 = nullptr;
    WS<double> *w64 = nullptr;
    void *host_stage = nullptr;  // device staging of mof_solve_host: b | u | s | sr
    Timer timer;
    // Solve-OF on downsampled frames (of_scale > 1): an internal problem of the coarse size,
    // with its own workspace
    mof_problem *coarse = nullptr;
    int coarse_scale = 0;
};

template <typename real>
static WS<real> *&ws_slot(Holder *h) {
    if constexpr (sizeof(real) == 8) return h->w64;
    else return h->w32;
}

static Holder *holder(mof_problem *p) {
    if (!p->ws) p->ws = new Holder();
    return static_cast<Holder *>(p->ws);
}

template <typename real>
static void free_ws(WS<real> *w) {
    if (!w) return;
    w->drop_graphs();
    if (w->ss) cudaStreamDestroy(w->ss);
    if (w->join) cudaEventDestroy(w->join);
    for (int g = 0; g < MAX_OF_STREAMS; ++g) {
        if (w->gs[g]) cudaStreamDestroy(w->gs[g]);
        if (w->gdone[g]) cudaEventDestroy(w->gdone[g]);
    }
    if (w->gfork) cudaEventDestroy(w->gfork);
    if (w->side) cudaStreamDestroy(w->side);
    if (w->side_fork) cudaEventDestroy(w->side_fork);
    if (w->side_done) cudaEventDestroy(w->side_done);
    if (w->mem) cudaFree(w->mem);
    delete w;
}

void free_workspace(mof_problem *p) {
    if (!p->ws) return;
    Holder *h = static_cast<Holder *>(p->ws);
    for (auto &s : h->scr)
        if (s) cudaFree(s);
    if (h->host_stage) cudaFree(h->host_stage);
    free_ws(h->w32);
    free_ws(h->w64);
    if (h->coarse) mof_problem_destroy(h->coarse);
    delete h;
    p->ws = nullptr;
}

mof_status apply_scratch(mof_problem *p, ScratchKind kind, void **out) {
    Holder *h = holder(p);
    if (!h->scr[kind]) {
        const size_t es = p->precision == MOF_FP64 ? 8 : 4;
        size_t bytes = 0;
        switch (kind) {
            case SCR_IMAGE: bytes = es * p->n; break;
            case SCR_RADIUS: bytes = sizeof(int) * (2 * (size_t)(p->nt - 1) * tile_bound_ints(p) + 16); break;
            case SCR_DEST: bytes = sizeof(int) * (p->nt - 1) * p->ns; break;
            case SCR_FLOWROWS: bytes = es * 2 * (p->nt - 1) * p->ns; break;
            default: return fail(MOF_EINVAL, "bad scratch kind");
        }
        MOF_CUDA(cudaMalloc(&h->scr[kind], bytes));
    }
    *out = h->scr[kind];
    return MOF_OK;
}

constexpr int TG_T = 256;      // theta-gram block
constexpr int TG_PIX = 64;     // pixels per theta-gram tile
constexpr int TG_ROWS = 4 * TG_PIX;
// theta-gram CTAs per SM of the persistent grid: three in FP32 (registers bounded so that
// three are resident), two in FP64 (unbounded registers)
template <typename real>
constexpr int tg_ctas_per_sm() { return sizeof(real) == 4 ? 4 : 2; }
template <typename real>
constexpr int tg_min_blocks() { return sizeof(real) == 4 ? 4 : 1; }

template <typename real>
static size_t theta_gram_smem(int Kmax) {
    // the row tile, reused at the end for the FP64 group sums ([groups][blocks][16] <= [256][16])
    const size_t tile = sizeof(real) * ((size_t)(((Kmax + 3) / 4) * 4) * (TG_ROWS + 4) + 4 * (size_t)((Kmax + 3) / 4));
    const size_t red = sizeof(double) * 256 * 16;
    return tile > red ? tile : red;
}

// Sizes of the weighted Gram of Solve-OF with p = q = 1 (k_of_wgram): threads, pixels
// per tile, CTAs per pair, quads of columns, 4x4 blocks, partial doubles per CTA.
constexpr int WG_T = 256, WG_P = 64, WG_CTAS = 64;
__host__ __device__ constexpr int wg_k4f(int K) { return (K + 4) / 4; }  // quads of K + 1 columns
__host__ __device__ constexpr int wg_k4l(int K) { return (K + 3) / 4; }
__host__ __device__ constexpr int wg_nblk(int K) {
    return wg_k4f(K) * (wg_k4f(K) + 1) / 2 + wg_k4l(K) * (wg_k4l(K) + 1) / 2;
}
__host__ __device__ constexpr int wg_pstride(int Kmax) { return wg_nblk(Kmax) * 16; }
// shared memory: the staged rows, later reused for the per-slot FP64 sums
template <typename real>
constexpr size_t wg_smem(int Kmax) {
    const size_t rows = ((size_t)wg_k4f(Kmax) * (WG_P + 1) + (size_t)wg_k4l(Kmax) * (4 * WG_P + 1)) * 4 * sizeof(real);
    const size_t nsl = (size_t)(wg_nblk(Kmax) > WG_T ? wg_nblk(Kmax) : WG_T);
    const size_t slots = nsl * 16 * sizeof(double);
    return rows > slots ? rows : slots;
}

template <typename real>
__global__ void __launch_bounds__(WG_T) k_of_wgram(const real *__restrict__ V, int Kmax, const int *__restrict__ K,
                                                   const int *__restrict__ act, const real *__restrict__ ux,
                                                   const real *__restrict__ uy, const real *__restrict__ bof,
                                                   const real *__restrict__ wf, const real *__restrict__ wl, int nx, int ny,
                                                   double *__restrict__ partial);

// doubles of Krylov scratch per frame pair of Solve-OF: the Krylov kernels' chunk
// partials, and the per-CTA partials of the Gram columns (of_ell columns at once)
static long long of_partial_per_pair(const mof_problem *p, int Kof, int of_ell) {
    const long long ns = p->ns;
    const long long gram_chunks = (ns + 511) / 512;  // chunks of the FP64 Gram kernel (the smaller)
    const long long gram = (long long)std::min(of_ell, Kof) * gram_chunks * (2LL * Kof + 1);
    const long long wgram = (long long)WG_CTAS * wg_pstride(Kof);
    const long long pass = of_pass_chunks(ns, 8) * of_pass_stride(Kof);  // k_of_proj_gram_pass (FP64 chunks)
    return std::max(std::max(std::max(krylov_partial_doubles(2 * ns, Kof), gram), wgram), pass);
}

template <typename real>
static mof_status ensure_ws(mof_problem *p, const mof_solver_params &prm, int n_outer, WS<real> *&w) {
    const int Kmax = prm.ell + n_outer;
    const int Kof = prm.of_ell + prm.of_iters;
    if (w && w->Kmax >= Kmax && w->Kof >= Kof && w->of_ell >= prm.of_ell && w->ell >= prm.ell && w->max_outer >= n_outer &&
        (prm.of_pq != 1 || w->pq1))
        return MOF_OK;
    free_ws(w);
    w = new WS<real>();
    w->Kmax = Kmax;
    w->Kof = Kof;
    w->of_ell = prm.of_ell;
    w->ell = prm.ell;
    w->max_outer = n_outer;
    w->pq1 = prm.of_pq == 1;
    const long long n = p->n, m = p->m, ns = p->ns, P = p->nt - 1, N2 = 2 * ns;
    int dev_sms = 152;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, p->device);
    w->gram_ctas = tg_ctas_per_sm<real>() * dev_sms;
    const long long partial = std::max(krylov_partial_doubles(std::max(n, m), Kmax), P * of_partial_per_pair(p, Kof, prm.of_ell));
    for (int pass = 0; pass < 2; ++pass) {
        Arena a;
        a.base = w->mem;
        // image step
        w->V = a.take<real>((size_t)Kmax * n);
        w->HV = a.take<real>((size_t)Kmax * m);
        w->U = a.take<real>((size_t)(prm.ell + 1) * m);
        w->u = a.take<real>(n);
        w->un = a.take<real>(n);
        w->r = a.take<real>(n);
        w->tm = a.take<real>(m);
        w->tn = a.take<real>(n);
        w->b = a.take<real>(m);
        w->q = a.take<real>(2 * P * ns);
        w->uT = a.take<real>(n);
        w->s = a.take<real>(P * N2);
        w->sr = a.take<real>(P * N2);
        w->vnew = a.take<real>(n);
        w->hvnew = a.take<real>(m);
        const long long bints = tile_bound_ints(p) * P;
        w->rad_s = a.take<int>(bints);
        w->rad_sr = a.take<int>(bints);
        w->rad_rev = a.take<int>(bints);
        w->dest = a.take<int>(P * ns);
        w->GH = a.take<double>((size_t)Kmax * Kmax);
        w->GT = a.take<double>((size_t)Kmax * Kmax);
        w->gH = a.take<double>(Kmax);
        w->z = a.take<double>(Kmax);
        w->lam = a.take<double>(1);
        w->coef = a.take<double>(Kmax + 8);
        w->c1 = a.take<double>(Kmax + 8);
        w->nrm2 = a.take<double>(1);
        w->nrm2b = a.take<double>(1);
        w->scaleR = a.take<double>(1);
        w->alpha = a.take<double>(prm.ell + 2);
        w->beta = a.take<double>(prm.ell + 2);
        w->beta1 = a.take<double>(1);
        w->alpha1 = a.take<double>(1);
        w->bb = a.take<double>(1);
        w->gpart = a.take<double>((size_t)3 * w->gram_ctas * Kmax * Kmax);  // Psi, Mhat, L_t partial sets
        w->K = a.take<int>(1);
        w->KU = a.take<int>(1);
        w->grow = a.take<int>(1);
        w->gkb = a.take<int>(1);
        w->flag = a.take<int>(1);
        w->err = a.take<int>(1);
        w->appended = a.take<int>(1);
        w->report = a.take<double>((size_t)n_outer * 8);
        // Solve-OF
        w->ux = a.take<real>(P * ns);
        w->uy = a.take<real>(P * ns);
        w->ut = a.take<real>(P * ns);
        w->bof = a.take<real>(P * ns);
        w->Vof = a.take<real>((size_t)P * Kof * N2);
        w->Uof = a.take<real>((size_t)P * (prm.of_ell + 1) * ns);
        w->AtB = a.take<real>(P * N2);
        w->wv = a.take<real>(P * N2);
        w->wu = a.take<real>(P * ns);
        w->y1 = a.take<real>(P * N2);
        w->y2 = a.take<real>(P * N2);
        w->sof = a.take<real>(P * N2);
        w->vnew_of = a.take<real>(P * N2);
        w->GA = a.take<double>((size_t)P * Kof * Kof);
        w->GL = a.take<double>((size_t)P * Kof * Kof);
        w->gof = a.take<double>((size_t)P * Kof);
        w->zof = a.take<double>((size_t)P * Kof);
        w->gam = a.take<double>(P);
        w->nrm_of = a.take<double>(P);
        w->coef_of = a.take<double>((size_t)P * Kof);
        w->Mg_of = a.take<double>((size_t)P * Kof * Kof);
        w->pres_of = a.take<double>((size_t)P * of_pass_stride(Kof));
        w->q_of = a.take<real>((size_t)P * N2);
        w->coefU_of = a.take<double>((size_t)P * (prm.of_ell + 1));
        w->scale_of = a.take<double>(P);
        w->alpha_of = a.take<double>(P);
        w->alpha1_of = a.take<double>(P);
        w->beta_of = a.take<double>(P);
        w->beta1_of = a.take<double>(P);
        w->bb_of = a.take<double>(P);
        w->Kv_of = a.take<int>(P);
        w->Ku_of = a.take<int>(P);
        w->grow_of = a.take<int>(P);
        w->gkb_of = a.take<int>(P);
        w->act_of = a.take<int>(P);
        w->app_of = a.take<int>(P);
        w->flag_of = a.take<int>(P);
        w->wf_of = a.take<real>(w->pq1 ? P * ns : 0);
        w->wl_of = a.take<real>(w->pq1 ? 4 * P * ns : 0);
        w->rn_of = a.take<double>(w->pq1 ? P : 0);
        w->partial = a.take<double>((size_t)partial);
        w->kaux = a.take<double>(2 * (size_t)std::max<long long>(P, 1) + 8);
        w->iter = a.take<int>(1);
        if (pass == 0) {
            w->bytes = a.off + 256;
            cudaError_t e = cudaMalloc(&w->mem, w->bytes);
            if (e != cudaSuccess) {
                delete w;
                w = nullptr;
                return cuda_fail(e, "workspace allocation", __FILE__, __LINE__);
            }
            MOF_CUDA(cudaMemset(w->mem, 0, w->bytes));
            MOF_CUDA(cudaStreamCreateWithFlags(&w->ss, cudaStreamNonBlocking));
            MOF_CUDA(cudaEventCreateWithFlags(&w->join, cudaEventDisableTiming));
            MOF_CUDA(cudaEventCreateWithFlags(&w->gfork, cudaEventDisableTiming));
            MOF_CUDA(cudaStreamCreateWithFlags(&w->side, cudaStreamNonBlocking));
            MOF_CUDA(cudaEventCreateWithFlags(&w->side_fork, cudaEventDisableTiming));
            MOF_CUDA(cudaEventCreateWithFlags(&w->side_done, cudaEventDisableTiming));
            for (int g = 0; g < MAX_OF_STREAMS; ++g) {
                MOF_CUDA(cudaStreamCreateWithFlags(&w->gs[g], cudaStreamNonBlocking));
                MOF_CUDA(cudaEventCreateWithFlags(&w->gdone[g], cudaEventDisableTiming));
            }
        }
    }
    const size_t sm = theta_gram_smem<real>(Kmax);
    (void)sm;
    if (w->pq1)
        MOF_CUDA(cudaFuncSetAttribute(k_of_wgram<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wg_smem<real>(Kof)));
    return MOF_OK;
}

// ============================================================ small kernels
// Per-problem FP64 scalar converted to the storage type once per block and
// shared: GB300 issues FP64 (conversions included) at a small fraction of
// the FP32 rate, so bandwidth-bound kernels keep FP64 out of their threads.
// Call once per kernel, before any thread-dependent return.
template <typename real>
__device__ __forceinline__ real block_scalar(const double *p) {
    __shared__ real v;
    if (threadIdx.x == 0 && threadIdx.y == 0) v = (real)*p;
    __syncthreads();
    return v;
}

template <typename real>
__global__ void k_fill(real *x, long long n, real v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) x[i] = v;
}
__global__ void k_fill_int(int *x, int n, int v) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = v;
}
template <typename real>
__global__ void k_copy(const real *__restrict__ a, real *__restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) b[i] = a[i];
}
template <typename real>
__global__ void k_neg(const real *__restrict__ a, real *__restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) b[i] = -a[i];
}
// x[b] -= coef[b] * y[b]  (coef device, per problem)
template <typename real>
__global__ void k_axpy_dev(real *__restrict__ x, long long xstride, const real *__restrict__ y, long long ystride,
                           const double *__restrict__ coef, long long N, const int *__restrict__ act) {
    const int b = blockIdx.y;
    if (act && !act[b]) return;
    const real c = block_scalar<real>(coef + b);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        x[b * xstride + i] -= c * y[b * ystride + i];
}
// err |= 16 when the data's squared norm is not finite (a NaN or an infinity in b)
__global__ void k_flag_nonfinite(const double *__restrict__ v, int *__restrict__ err) {
    if (threadIdx.x == 0 && !isfinite(v[0])) atomicOr(err, 16);
}
__global__ void k_sqrt_into(const double *__restrict__ a, double *__restrict__ b, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = sqrt(a[i]);
}
__global__ void k_sqrt_into_if(const double *__restrict__ a, double *__restrict__ b, int n, const int *__restrict__ act) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && (!act || act[i])) b[i] = sqrt(a[i]);
}
__global__ void k_mul_into(const double *__restrict__ a, const double *__restrict__ c, double *__restrict__ out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] * c[i];
}
__global__ void k_of_activate(const double *__restrict__ bb, int *__restrict__ act, int *__restrict__ gkb,
                              int *__restrict__ grow, int *__restrict__ Kv, int *__restrict__ Ku, double *__restrict__ beta1,
                              int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int a = bb[i] > 0.0 && isfinite(bb[i]);
    act[i] = a;
    gkb[i] = a;
    grow[i] = a;
    Kv[i] = 0;
    Ku[i] = 0;
    beta1[i] = sqrt(bb[i]);
}
// copy column K-1 of a [B][ld][ld] matrix into row K-1
__global__ void k_sym_last(double *__restrict__ G, int ld, const int *__restrict__ K, const int *__restrict__ act) {
    const int b = blockIdx.x;
    if (act && !act[b]) return;
    const int j = K[b] - 1;
    if (j < 0) return;
    double *Gb = G + (long long)b * ld * ld;
    for (int i = threadIdx.x; i < j; i += blockDim.x) Gb[j * ld + i] = Gb[i * ld + j];
}
// copy a staged vector into slot K-1 of a basis of one problem
template <typename real>
__global__ void k_store_slot(real *__restrict__ base, long long N, const int *__restrict__ K, const int *__restrict__ app,
                             const real *__restrict__ v) {
    if (!app[0]) return;
    real *d = base + (long long)(K[0] - 1) * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) d[i] = v[i];
}

// ------------------------------------------------------------ Upsilon kernels
// GKB steps of Solve-OF, one problem per frame pair (blockIdx.y):
//   out = Upsilon^T u_j - beta_j v_{j-1}     (V side, length 2 ns)
template <typename real>
__global__ void k_of_upsT(const real *__restrict__ ux, const real *__restrict__ uy, const real *__restrict__ U, int ldU,
                          int j, const real *__restrict__ V, int ldV, const double *__restrict__ beta,
                          real *__restrict__ out, long long ns, const int *__restrict__ act) {
    const int b = blockIdx.y;
    if (!act[b]) return;
    const real *uj = U + ((long long)b * ldU + j) * ns;
    const real *vp = j > 0 ? V + ((long long)b * ldV + j - 1) * 2 * ns : nullptr;
    const real bj = j > 0 ? block_scalar<real>(beta + b) : (real)0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ns; i += (long long)gridDim.x * blockDim.x) {
        const real r = uj[i];
        real o0 = ux[b * ns + i] * r, o1 = uy[b * ns + i] * r;
        if (vp) {
            o0 -= bj * vp[i];
            o1 -= bj * vp[ns + i];
        }
        out[b * 2 * ns + i] = o0;
        out[b * 2 * ns + ns + i] = o1;
    }
}
//   out = Upsilon v_j - alpha_j u_j           (U side, length ns)
template <typename real>
__global__ void k_of_ups(const real *__restrict__ ux, const real *__restrict__ uy, const real *__restrict__ V, int ldV, int j,
                         const real *__restrict__ U, int ldU, const double *__restrict__ alpha, real *__restrict__ out,
                         long long ns, const int *__restrict__ act) {
    const int b = blockIdx.y;
    if (!act[b]) return;
    const real *vj = V + ((long long)b * ldV + j) * 2 * ns;
    const real *uj = U + ((long long)b * ldU + j) * ns;
    const real aj = block_scalar<real>(alpha + b);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ns; i += (long long)gridDim.x * blockDim.x)
        out[b * ns + i] = ux[b * ns + i] * vj[i] + uy[b * ns + i] * vj[ns + i] - aj * uj[i];
}

// Graph Laplacian of one component with free boundary: (Psi^T Psi f)(x,y).
template <typename real>
__device__ __forceinline__ real lap_at(const real *__restrict__ f, int nx, int ny, int x, int y) {
    const long long i = (long long)y * nx + x;
    const real c = f[i];
    real v = 0;
    if (x > 0) v += c - f[i - 1];
    if (x < nx - 1) v += c - f[i + 1];
    if (y > 0) v += c - f[i - nx];
    if (y < ny - 1) v += c - f[i + nx];
    return v;
}

// r = Ups^T Ups s - Ups^T b + gamma (L(+)L)^T (L(+)L) s  (normal-equation residual of Alg. 2)
template <typename real>
__global__ void k_of_resid(const real *__restrict__ ux, const real *__restrict__ uy, const real *__restrict__ AtB,
                           const real *__restrict__ s, const double *__restrict__ gam, real *__restrict__ r, int nx, int ny,
                           const int *__restrict__ act) {
    const int b = blockIdx.z;
    if (!act[b]) return;
    const real g = block_scalar<real>(gam + b);
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const long long ns = (long long)nx * ny, i = (long long)y * nx + x;
    const real *v = s + b * 2 * ns;
    const real ax = ux[b * ns + i], ay = uy[b * ns + i];
    const real a = ax * v[i] + ay * v[ns + i];
    r[b * 2 * ns + i] = ax * a - AtB[b * 2 * ns + i] + g * lap_at(v, nx, ny, x, y);
    r[b * 2 * ns + ns + i] = ay * a - AtB[b * 2 * ns + ns + i] + g * lap_at(v + ns, nx, ny, x, y);
}

// ---- Euclidean Gram Mg = V^T V of a pair's stored Solve-OF basis. The Golub-Kahan start
// leaves orthonormal vectors (Mg = I there); each GKS append stores x'/||x'|| where x' is the
// residual after ONE projection pass, and records its inner products with the earlier vectors
// (the second pass's coefficients c2 = V^T x', which the fused pass computes anyway) in Mg.
// The projection of the next residual then uses d = Mg^-1 (V^T r), the orthogonal projection
// onto the stored basis's span; so the second update pass over the basis (x' - V c2) is never
// applied to the vectors. The span, the Grams of the stored vectors and everything the small
// solver computes from them (z, the parameter, s = V z) are those of the basis CGS twice
// would store, up to rounding.
__global__ void k_of_mg_init(double *__restrict__ Mg, int ld, const int *__restrict__ act, int B) {
    const int b = blockIdx.x;
    if (b >= B || (act && !act[b])) return;
    double *M = Mg + (long long)b * ld * ld;
    for (int e = threadIdx.x; e < ld * ld; e += blockDim.x) M[e] = (e / ld == e % ld) ? 1.0 : 0.0;
}

// c[b] <- Mg[b]^-1 c[b] over the first K[b] entries: Cholesky in shared memory by one warp
// (lanes over rows), then the two triangular solves. Mg is near I (unit diagonal, off
// diagonal the stored vectors' residual overlaps), so the factorisation is well conditioned.
__global__ void __launch_bounds__(32) k_of_mg_solve(const double *__restrict__ Mg, double *__restrict__ c, int ld,
                                                    const int *__restrict__ K, const int *__restrict__ act) {
    extern __shared__ double mg_sm[];  // [ld][ld + 1] Cholesky factor (lower), then [ld] the right side
    const int b = blockIdx.x, lane = threadIdx.x;
    if (act && !act[b]) return;
    const int Kb = min(K[b], ld), L = ld + 1;
    double *Lm = mg_sm, *y = mg_sm + (long long)ld * L;
    const double *M = Mg + (long long)b * ld * ld;
    double *cb = c + (long long)b * ld;
    for (int e = lane; e < Kb * Kb; e += 32) Lm[(e / Kb) * L + e % Kb] = M[(e / Kb) * ld + e % Kb];
    for (int i = lane; i < Kb; i += 32) y[i] = cb[i];
    __syncwarp();
    for (int j = 0; j < Kb; ++j) {
        // column j: rows i >= j, s_i = M[i][j] - sum_{k<j} L[i][k] L[j][k]
        for (int i = j + lane; i < Kb; i += 32) {
            double sum = Lm[i * L + j];
            for (int k = 0; k < j; ++k) sum -= Lm[i * L + k] * Lm[j * L + k];
            Lm[i * L + j] = sum;
        }
        __syncwarp();
        const double d = sqrt(fmax(Lm[j * L + j], 1e-300));
        for (int i = j + 1 + lane; i < Kb; i += 32) Lm[i * L + j] /= d;
        __syncwarp();
        if (lane == 0) Lm[j * L + j] = d;
        __syncwarp();
    }
    if (lane == 0) {  // L y = c, then L^T d = y (K <= 64 sequential steps)
        for (int i = 0; i < Kb; ++i) {
            double t = y[i];
            for (int k = 0; k < i; ++k) t -= Lm[i * L + k] * y[k];
            y[i] = t / Lm[i * L + i];
        }
        for (int i = Kb - 1; i >= 0; --i) {
            double t = y[i];
            for (int k = i + 1; k < Kb; ++k) t -= Lm[k * L + i] * y[k];
            y[i] = t / Lm[i * L + i];
        }
    }
    __syncwarp();
    for (int i = lane; i < Kb; i += 32) cb[i] = y[i];
}

// After an append (appended[b]; K[b] already counts the new vector): the new column of Mg,
// Mg[i][new] = Mg[new][i] = c2[b][i] / ||x'|| for the earlier vectors, 1 on the diagonal.
__global__ void k_of_mg_update(double *__restrict__ Mg, const double *__restrict__ c2, const double *__restrict__ nrm2,
                               int ld, const int *__restrict__ K, const int *__restrict__ appended,
                               const int *__restrict__ act) {
    const int b = blockIdx.x;
    if ((act && !act[b]) || !appended[b]) return;
    const int knew = min(K[b], ld) - 1;
    const double inv = 1.0 / sqrt(nrm2[b]);
    double *M = Mg + (long long)b * ld * ld;
    for (int i = threadIdx.x; i < knew; i += blockDim.x) {
        const double v = c2[(long long)b * ld + i] * inv;
        M[(long long)i * ld + knew] = v;
        M[(long long)knew * ld + i] = v;
    }
    if (threadIdx.x == 0) M[(long long)knew * ld + knew] = 1.0;
}

// First CGS projection of the GKS residual from the Gram matrices: with
// r = (Ups^T Ups + gamma (L(+)L)^T (L(+)L)) V z - Ups^T b, V^T r = (G_A + gamma G_L) z - g
// exactly, so the coefficients need no pass over V. One warp per pair.
__global__ void k_of_proj_gram(const double *__restrict__ GA, const double *__restrict__ GL, const double *__restrict__ g,
                               const double *__restrict__ z, const double *__restrict__ gam, const int *__restrict__ K,
                               const int *__restrict__ act, int ld, double *__restrict__ c) {
    const int b = blockIdx.x, lane = threadIdx.x;
    if (act && !act[b]) return;
    const int Kb = min(K[b], ld);
    const double *A = GA + (long long)b * ld * ld, *L = GL + (long long)b * ld * ld, *zb = z + (long long)b * ld;
    const double gm = gam[b];
    // the Grams are stored symmetric: row i is read as column i, lanes over i (coalesced)
    for (int i = lane; i < Kb; i += 32) {
        double sa = 0.0, sl = 0.0;
#pragma unroll 4
        for (int k = 0; k < Kb; ++k) {
            const double zk = zb[k];
            sa += A[k * ld + i] * zk;
            sl += L[k * ld + i] * zk;
        }
        c[(long long)b * ld + i] = sa + gm * sl - g[(long long)b * ld + i];
    }
}

// Gram columns of Solve-OF: for column j and every i <= j,
//   G_A[i][j] = (Ups v_i)^T (Ups v_j) = v_i^T (Ups^T Ups v_j),
//   G_L[i][j] = (L v_i)^T (L v_j) = v_i^T (L^T L v_j),   g[j] = (Ups v_j)^T b,
// with Ups v = u_x v_x + u_y v_y pointwise and L the forward differences in x
// and y of both velocity components (no boundary row), so L^T L is the graph
// Laplacian of each component with free boundary. Column j is blockIdx.z (mode
// 0: the first columns, j < K) or K - 1 (mode 1: the vector appended last,
// where appended). A CTA owns a chunk of OFC pixels of one pair: it stages
// Ups^T Ups v_j and L^T L v_j (both components) in shared memory, and its warps
// stream the basis vectors i = w, w + 8, ... over the chunk with plain
// coalesced loads, taking two dot products per vector, with sums per chunk in
// the storage precision; k_of_gram_reduce adds the chunks in FP64.
constexpr int OFG_T = 256;
template <typename real>
constexpr int ofc() { return 4096 / (int)sizeof(real); }  // pixels per chunk: 1024 (FP32), 512 (FP64)

template <typename real>
__device__ __forceinline__ real warp_sum_r(real v) {
    if constexpr (sizeof(real) == 4) return warp_sumf(v);
    else return warp_sum(v);
}

template <typename real>
__global__ void __launch_bounds__(OFG_T) k_of_gram_cols(const real *__restrict__ V, int Kmax, const int *__restrict__ K,
                                                        const int *__restrict__ act, int mode, const real *__restrict__ ux,
                                                        const real *__restrict__ uy, const real *__restrict__ bof, int nx,
                                                        int ny, double *__restrict__ partial) {
    constexpr int OFC = ofc<real>();
    __shared__ __align__(16) real s_y[4][OFC];  // (Ups^T Ups v_j)_x, _y, (L^T L v_j)_x, _y
    __shared__ real s_red[OFG_T / 32];
    const int b = blockIdx.y, chunk = blockIdx.x, nchunk = gridDim.x;
    if (!act[b]) return;
    const int Kb = min(K[b], Kmax);
    const int j = mode == 0 ? (int)blockIdx.z : Kb - 1;
    if (j < 0 || j >= Kb) return;
    const long long ns = (long long)nx * ny, N2 = 2 * ns;
    const int c0 = chunk * OFC;
    const int len = (int)min((long long)OFC, ns - c0);
    const real *Vb = V + (long long)b * Kmax * N2;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    double *out = partial + (((long long)b * gridDim.z + blockIdx.z) * nchunk + chunk) * (2 * Kmax + 1);
    // stage the normal-equation parts of column j; g_j on the way
    const real *vj = Vb + (long long)j * N2;
    real gs = 0;
    for (int q = tid; q < OFC; q += OFG_T) {
        real y0 = 0, y1 = 0, l0 = 0, l1 = 0;
        if (q < len) {
            const int p = c0 + q;
            const int y = p / nx, x = p - y * nx;
            const real fx = ux[b * ns + p], fy = uy[b * ns + p];
            const real a = fx * vj[p] + fy * vj[ns + p];
            y0 = fx * a;
            y1 = fy * a;
            l0 = lap_at(vj, nx, ny, x, y);
            l1 = lap_at(vj + ns, nx, ny, x, y);
            gs += a * bof[b * ns + p];
        }
        s_y[0][q] = y0;
        s_y[1][q] = y1;
        s_y[2][q] = l0;
        s_y[3][q] = l1;
    }
    gs = warp_sum_r(gs);
    if (lane == 0) s_red[wid] = gs;
    __syncthreads();
    if (tid == 0) {
        double dg = 0.0;
        for (int w = 0; w < OFG_T / 32; ++w) dg += (double)s_red[w];
        out[2 * Kmax] = dg;
    }
    // 4 pixels per lane with 16-byte loads where the layout allows it (FP32, a full
    // chunk, both components 16-byte aligned)
    const bool quad = sizeof(real) == 4 && (ns % 4) == 0 && len == OFC;
    for (int i = wid; i <= j; i += OFG_T / 32) {
        const real *vi = Vb + (long long)i * N2 + c0;
        real ga = 0, gl = 0;
        if (quad) {
            // each step's eight products summed in FP32, the steps' partials accumulated
            // with their rounding errors (DFAcc::add), the lanes in FP64
            const float4 *X4 = reinterpret_cast<const float4 *>(vi);
            const float4 *Y4 = reinterpret_cast<const float4 *>(vi + ns);
            const float4 *A0 = reinterpret_cast<const float4 *>(s_y[0]), *A1 = reinterpret_cast<const float4 *>(s_y[1]);
            const float4 *L0 = reinterpret_cast<const float4 *>(s_y[2]), *L1 = reinterpret_cast<const float4 *>(s_y[3]);
            DFAcc da, dl;
            // two quads of both components per step (16 products per partial); OFC / 4 is a
            // multiple of 64, so every lane takes the same number of steps
            for (int q = lane; q < OFC / 4; q += 64) {
                const float4 X = __ldcs(X4 + q), Y = __ldcs(Y4 + q), X2 = __ldcs(X4 + q + 32), Y2 = __ldcs(Y4 + q + 32);
                const float4 a0 = A0[q], a1 = A1[q], l0 = L0[q], l1 = L1[q];
                const float4 b0 = A0[q + 32], b1 = A1[q + 32], m0 = L0[q + 32], m1 = L1[q + 32];
                float pa = X.x * a0.x + X.y * a0.y + X.z * a0.z + X.w * a0.w + Y.x * a1.x + Y.y * a1.y + Y.z * a1.z + Y.w * a1.w;
                pa += X2.x * b0.x + X2.y * b0.y + X2.z * b0.z + X2.w * b0.w + Y2.x * b1.x + Y2.y * b1.y + Y2.z * b1.z + Y2.w * b1.w;
                float pl = X.x * l0.x + X.y * l0.y + X.z * l0.z + X.w * l0.w + Y.x * l1.x + Y.y * l1.y + Y.z * l1.z + Y.w * l1.w;
                pl += X2.x * m0.x + X2.y * m0.y + X2.z * m0.z + X2.w * m0.w + Y2.x * m1.x + Y2.y * m1.y + Y2.z * m1.z + Y2.w * m1.w;
                da.add(pa);
                dl.add(pl);
            }
            const double sa = warp_sum(da.value()), sl = warp_sum(dl.value());
            if (lane == 0) {
                out[2 * i] = sa;
                out[2 * i + 1] = sl;
            }
            continue;
        } else {
            for (int q = lane; q < len; q += 32) {
                const real vx = vi[q], vy = vi[ns + q];
                ga += vx * s_y[0][q] + vy * s_y[1][q];
                gl += vx * s_y[2][q] + vy * s_y[3][q];
            }
        }
        ga = warp_sum_r(ga);
        gl = warp_sum_r(gl);
        if (lane == 0) {
            out[2 * i] = (double)ga;
            out[2 * i + 1] = (double)gl;
        }
    }
}

// Sum the CTA partials of k_of_gram_cols in FP64 (one warp per output) and write
// G_A[b][i][j] = G_A[b][j][i], G_L likewise, g[b][j].
__global__ void k_of_gram_reduce(const double *__restrict__ partial, int nctas, int Kmax, const int *__restrict__ K,
                                 const int *__restrict__ act, int mode, double *__restrict__ GA, double *__restrict__ GL,
                                 double *__restrict__ g) {
    const int b = blockIdx.y;
    if (!act[b]) return;
    const int Kb = min(K[b], Kmax);
    const int j = mode == 0 ? (int)blockIdx.z : Kb - 1;
    if (j < 0 || j >= Kb) return;
    const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    const int nout = 2 * (j + 1) + 1;
    if (o >= nout) return;
    const int slot = o == nout - 1 ? 2 * Kmax : o;
    const double *src = partial + ((long long)b * gridDim.z + blockIdx.z) * nctas * (2 * Kmax + 1) + slot;
    double sum = 0.0;
#pragma unroll 8
    for (int c = lane; c < nctas; c += 32) sum += src[(long long)c * (2 * Kmax + 1)];
    sum = warp_sum(sum);
    if (lane != 0) return;
    const long long KK = (long long)Kmax * Kmax;
    if (o == nout - 1) {
        g[(long long)b * Kmax + j] = sum;
        return;
    }
    const int i = o >> 1;
    double *G = (o & 1) ? GL : GA;
    G[b * KK + (long long)i * Kmax + j] = sum;
    G[b * KK + (long long)j * Kmax + i] = sum;
}

// four consecutive values from 16-byte aligned shared memory
template <typename real>
struct Quad {
    real x, y, z, w;
};
__device__ __forceinline__ Quad<float> load_quad(const float *p) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Quad<double> load_quad(const double *p) {
    const double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
    return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void store_quad(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store_quad(double *p, const double (&v)[4]) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2 *>(p + 2) = make_double2(v[2], v[3]);
}

// ------------------------------------------------ Solve-OF with p = q = 1 (MM-GKS)
// App. A applied to the flow problem of a pair: at every iteration the IRLS
// weights of the current velocity s, wf = ((Ups s - b)^2 + eps^2)^(-1/2) per pixel
// and wl = ((L s)^2 + eps^2)^(-1/2) per difference row (rows of L: the x and y
// forward differences of each component; a row past the frame's last column or
// row is zero and gets no weight). s = nullptr stands for s = 0 (first iteration).
// The arrays hold the square roots of the weights (the Gram scales its rows by them).
template <typename real>
__global__ void k_of_irls_weights(const real *__restrict__ ux, const real *__restrict__ uy, const real *__restrict__ bof,
                                  const real *__restrict__ s, real eps2, real *__restrict__ wf, real *__restrict__ wl,
                                  int nx, int ny, const int *__restrict__ act) {
    const int b = blockIdx.z;
    if (!act[b]) return;
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const long long ns = (long long)nx * ny, i = (long long)y * nx + x;
    const real *v = s ? s + b * 2 * ns : nullptr;
    const real res = (v ? ux[b * ns + i] * v[i] + uy[b * ns + i] * v[ns + i] : (real)0) - bof[b * ns + i];
    wf[b * ns + i] = (real)1 / sqrt(sqrt(res * res + eps2));
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const real *vc = v ? v + c * ns : nullptr;
        const real dx = (vc && x < nx - 1) ? vc[i + 1] - vc[i] : (real)0;
        const real dy = (vc && y < ny - 1) ? vc[i + nx] - vc[i] : (real)0;
        wl[(b * 4 + 2 * c) * ns + i] = (real)1 / sqrt(sqrt(dx * dx + eps2));
        wl[(b * 4 + 2 * c + 1) * ns + i] = (real)1 / sqrt(sqrt(dy * dy + eps2));
    }
}

// r = Ups^T W_f (Ups s - b) + gamma L^T W_L L s: the residual of the majorant's normal
// equations at the new s (weights of the iteration's start).
template <typename real>
__global__ void k_of_resid_w(const real *__restrict__ ux, const real *__restrict__ uy, const real *__restrict__ bof,
                             const real *__restrict__ s, const real *__restrict__ wf, const real *__restrict__ wl,
                             const double *__restrict__ gam, real *__restrict__ r, int nx, int ny,
                             const int *__restrict__ act) {
    const int b = blockIdx.z;
    if (!act[b]) return;
    const real g = block_scalar<real>(gam + b);
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const long long ns = (long long)nx * ny, i = (long long)y * nx + x;
    const real *v = s + b * 2 * ns;
    const real ax = ux[b * ns + i], ay = uy[b * ns + i];
    const real sf = wf[b * ns + i];
    const real e = sf * sf * (ax * v[i] + ay * v[ns + i] - bof[b * ns + i]);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const real *vc = v + c * ns;
        const real *wx = wl + (b * 4 + 2 * c) * ns, *wy = wx + ns;
        const real vi = vc[i];
        real lap = 0;  // (L^T W_L L v_c)(i): weighted edge differences into and out of i
        if (x > 0) lap += wx[i - 1] * wx[i - 1] * (vi - vc[i - 1]);
        if (x < nx - 1) lap -= wx[i] * wx[i] * (vc[i + 1] - vi);
        if (y > 0) lap += wy[i - nx] * wy[i - nx] * (vi - vc[i - nx]);
        if (y < ny - 1) lap -= wy[i] * wy[i] * (vc[i + nx] - vi);
        r[b * 2 * ns + c * ns + i] = (c == 0 ? ax : ay) * e + g * lap;
    }
}

// The weighted Grams of the majorant over the first K basis vectors of a pair:
//   [G_A g; g^T bb] = sum_pixels wf (a; b)(a; b)^T,  a_j = ux v_j + uy v_j' at the pixel,
//   G_L = sum over the difference rows of wl d d^T,  d_j = the row applied to v_j.
// A CTA owns a strided set of tiles of WG_P pixels of one pair. Per tile the
// pixel factors (sqrt(wf) ux, sqrt(wf) uy, sqrt(wf) b, sqrt(wl) of the four
// difference rows, zero where a row leaves the frame) are staged once, then the
// rows times the square-root weights are staged as quads of columns (fidelity:
// WG_P rows of K + 1 columns, the last one b; regulariser: 4 WG_P rows of K
// columns), and each thread accumulates 4x4 blocks of the upper triangle over
// its row group in the storage precision (a CTA adds ns / (WG_P gridDim.x)
// tiles, about 1000 rows per sum at the bench size). The row groups of a
// block meet in shared memory; the CTA writes one FP64 partial per block and
// k_of_wgram_reduce adds the CTAs in FP64.
template <typename real>
__device__ __forceinline__ void wg_block(int idx, int nbf, int k4f, int k4l, bool &fid, int &I, int &J) {
    fid = idx < nbf;
    int rem = fid ? idx : idx - nbf;
    const int k4 = fid ? k4f : k4l;
    I = 0;
    while (rem >= k4 - I) {
        rem -= k4 - I;
        ++I;
    }
    J = I + rem;
}

template <typename real>
__global__ void __launch_bounds__(WG_T) k_of_wgram(const real *__restrict__ V, int Kmax, const int *__restrict__ K,
                                                   const int *__restrict__ act, const real *__restrict__ ux,
                                                   const real *__restrict__ uy, const real *__restrict__ bof,
                                                   const real *__restrict__ wf, const real *__restrict__ wl, int nx, int ny,
                                                   double *__restrict__ partial) {
    static_assert(WG_P == 64 && WG_T == 256, "index arithmetic below uses shifts for WG_P = 64");
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ real s_ax[WG_P], s_ay[WG_P], s_b[WG_P], s_l[4 * WG_P];
    const int b = blockIdx.y;
    if (!act[b]) return;
    const int Kb = min(K[b], Kmax);
    const int k4f = wg_k4f(Kb), k4l = wg_k4l(Kb);
    const int nbf = k4f * (k4f + 1) / 2, nbl = k4l * (k4l + 1) / 2, nbt = nbf + nbl;
    const long long ns = (long long)nx * ny, N2 = 2 * ns;
    const int ntiles = (int)((ns + WG_P - 1) / WG_P);
    constexpr int RSF = WG_P + 1, RSL = 4 * WG_P + 1;  // padded row counts (bank spread per quad)
    real *F = reinterpret_cast<real *>(smraw);          // [k4f][RSF][4]
    real *Lr = F + (size_t)k4f * RSF * 4;               // [k4l][RSL][4]
    const real *Vb = V + (long long)b * Kmax * N2;
    const int tid = threadIdx.x;
    // (block, row group) slots: a fidelity block has WG_P rows, a regulariser block
    // 4 WG_P, so regulariser blocks get four times the groups; with more blocks than
    // threads every thread takes two blocks over all rows
    int RGf = 1, RGl = 1;
    for (int rg = 32; rg >= 1; rg >>= 1) {
        const int f = rg >= 4 ? rg / 4 : 1;
        if (nbf * f + nbl * rg <= WG_T) {
            RGf = f;
            RGl = rg;
            break;
        }
    }
    const int nslot = nbf * RGf + nbl * RGl;
    const int per = nslot <= WG_T ? 1 : 2;
    const int nsl = per == 1 ? nslot : nbt;  // with two per thread: one slot per block, all rows
    int bI[2], bJ[2], r0[2], r1[2];
    bool bfid[2], on[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int slot = tid + q * WG_T;
        on[q] = q < per && slot < nsl;
        bI[q] = bJ[q] = r0[q] = r1[q] = 0;
        bfid[q] = true;
        if (!on[q]) continue;
        int blk, g, rg;
        if (per == 2) {
            blk = slot;
            g = 0;
            rg = 1;
        } else if (slot < nbf * RGf) {
            blk = slot / RGf;
            g = slot - blk * RGf;
            rg = RGf;
        } else {
            blk = nbf + (slot - nbf * RGf) / RGl;
            g = (slot - nbf * RGf) % RGl;
            rg = RGl;
        }
        wg_block<real>(blk, nbf, k4f, k4l, bfid[q], bI[q], bJ[q]);
        const int nrows = bfid[q] ? WG_P : 4 * WG_P;
        r0[q] = g * nrows / rg;
        r1[q] = (g + 1) * nrows / rg;
    }
    real sum[2][16];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int e = 0; e < 16; ++e) sum[q][e] = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long p0 = (long long)tile * WG_P;
        __syncthreads();
        {  // pixel factors: thread = (row d, pixel pl) with d = tid >> 6
            const int d = tid >> 6, pl = tid & (WG_P - 1);
            const long long pix = p0 + pl;
            real sl = 0;
            if (pix < ns) {
                const int y = (int)(pix / nx), x = (int)(pix - (long long)y * nx);
                const bool inside = (d & 1) ? (y < ny - 1) : (x < nx - 1);
                if (inside) sl = wl[(b * 4 + d) * ns + pix];
                if (d == 0) {
                    const real sw = wf[b * ns + pix];
                    s_ax[pl] = sw * ux[b * ns + pix];
                    s_ay[pl] = sw * uy[b * ns + pix];
                    s_b[pl] = sw * bof[b * ns + pix];
                }
            } else if (d == 0) {
                s_ax[pl] = s_ay[pl] = s_b[pl] = 0;
            }
            s_l[tid] = sl;
        }
        __syncthreads();
        // fidelity rows: column j < K: v_j ax + v_j' ay, column K: b (factors hold sqrt(wf)).
        // Thread (pl, quad group): whole quads of columns, the eight loads of a quad in flight.
        {
            const int pl = tid & (WG_P - 1);
            const long long pix = p0 + pl;
            const bool ok = pix < ns;
            const real ax = s_ax[pl], ay = s_ay[pl], bs = s_b[pl];
            for (int q4 = tid >> 6; q4 < k4f; q4 += WG_T / WG_P) {
                real vx[4], vy[4], out[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int j = 4 * q4 + c;
                    const real *vj = Vb + (long long)j * N2;
                    vx[c] = (ok && j < Kb) ? vj[pix] : (real)0;
                    vy[c] = (ok && j < Kb) ? vj[ns + pix] : (real)0;
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int j = 4 * q4 + c;
                    out[c] = j < Kb ? vx[c] * ax + vy[c] * ay : (j == Kb ? bs : (real)0);
                }
                store_quad(F + ((size_t)q4 * RSF + pl) * 4, out);
            }
        }
        // regulariser rows: row rr = d * WG_P + pl = tid, d = 2 c + dir (component c, dir
        // 0: x, 1: y); two quads of columns per step, sixteen loads in flight
        {
            const int rr = tid, d = rr >> 6, pl = rr & (WG_P - 1);
            const real sl = s_l[rr];
            const bool ok = sl != (real)0;  // a nonzero factor: the pixel and its neighbour exist
            const long long pix = p0 + pl, cb = (long long)(d >> 1) * ns + pix;
            const int off = (d & 1) ? nx : 1;
            for (int q4 = 0; q4 < k4l; q4 += 2) {
                real a[8], c2[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int j = 4 * q4 + c;
                    const bool on_ = ok && j < Kb;
                    const real *vc = Vb + (long long)j * N2 + cb;
                    a[c] = on_ ? vc[0] : (real)0;
                    c2[c] = on_ ? vc[off] : (real)0;
                }
                real o0[4], o1[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    o0[c] = sl * (c2[c] - a[c]);
                    o1[c] = sl * (c2[c + 4] - a[c + 4]);
                }
                store_quad(Lr + ((size_t)q4 * RSL + rr) * 4, o0);
                if (q4 + 1 < k4l) store_quad(Lr + ((size_t)(q4 + 1) * RSL + rr) * 4, o1);
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (!on[q]) continue;
            const real *base = bfid[q] ? F : Lr;
            const int rs = bfid[q] ? RSF : RSL;
            const real *pa = base + (size_t)bI[q] * rs * 4, *pb = base + (size_t)bJ[q] * rs * 4;
            for (int r = r0[q]; r < r1[q]; ++r) {
                const Quad<real> A = load_quad(pa + (size_t)r * 4), B = load_quad(pb + (size_t)r * 4);
                const real av[4] = {A.x, A.y, A.z, A.w}, bv[4] = {B.x, B.y, B.z, B.w};
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) sum[q][a * 4 + c] = fma(av[a], bv[c], sum[q][a * 4 + c]);
            }
        }
    }
    // the row groups of each block meet in shared memory (slot-major, FP64)
    __syncthreads();
    double *S = reinterpret_cast<double *>(smraw);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int slot = tid + q * WG_T;
        if (!on[q]) continue;
#pragma unroll
        for (int e = 0; e < 16; ++e) S[(size_t)slot * 16 + e] = (double)sum[q][e];
    }
    __syncthreads();
    double *out = partial + ((long long)b * gridDim.x + blockIdx.x) * wg_pstride(Kmax);
    for (int e = tid; e < nbt * 16; e += WG_T) {
        const int blk = e >> 4, el = e & 15;
        double v = 0.0;
        if (per == 2) {
            v = S[(size_t)blk * 16 + el];
        } else if (blk < nbf) {
            for (int g = 0; g < RGf; ++g) v += S[(size_t)(blk * RGf + g) * 16 + el];
        } else {
            const int s0 = nbf * RGf + (blk - nbf) * RGl;
            for (int g = 0; g < RGl; ++g) v += S[(size_t)(s0 + g) * 16 + el];
        }
        out[e] = v;
    }
}

// Sum the CTA partials of k_of_wgram in FP64 (one warp per block element) and write
// G_A, G_L (symmetric, leading dimension Kmax), g and bb of each pair.
__global__ void k_of_wgram_reduce(const double *__restrict__ partial, int nctas, int Kmax, const int *__restrict__ K,
                                  const int *__restrict__ act, double *__restrict__ GA, double *__restrict__ GL,
                                  double *__restrict__ g, double *__restrict__ bb) {
    const int b = blockIdx.y;
    if (!act[b]) return;
    const int Kb = min(K[b], Kmax);
    const int k4f = wg_k4f(Kb), k4l = wg_k4l(Kb);
    const int nbf = k4f * (k4f + 1) / 2, nbt = nbf + k4l * (k4l + 1) / 2;
    const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (o >= nbt * 16) return;
    const int blk = o >> 4, el = o & 15;
    bool fid;
    int I, J;
    wg_block<double>(blk, nbf, k4f, k4l, fid, I, J);
    const int i = 4 * I + (el >> 2), j = 4 * J + (el & 3);
    if (i > j) return;  // the diagonal blocks hold both triangles
    const int lim = fid ? Kb : Kb - 1;  // the fidelity Gram has the extra column Kb (b)
    if (j > lim) return;
    const long long stride = wg_pstride(Kmax);
    const double *src = partial + (long long)b * nctas * stride + o;
    double sum = 0.0;
#pragma unroll 8
    for (int c = lane; c < nctas; c += 32) sum += src[(long long)c * stride];
    sum = warp_sum(sum);
    if (lane != 0) return;
    const long long KK = (long long)Kmax * Kmax;
    if (fid && j == Kb) {
        if (i == Kb) bb[b] = sum;
        else g[(long long)b * Kmax + i] = sum;
        return;
    }
    double *G = (fid ? GA : GL) + b * KK;
    G[(long long)i * Kmax + j] = sum;
    G[(long long)j * Kmax + i] = sum;
}

// AtB = Upsilon^T b with b = -u_t, and bof = -u_t
template <typename real>
__global__ void k_of_rhs(const real *__restrict__ ux, const real *__restrict__ uy, const real *__restrict__ ut,
                         real *__restrict__ bof, real *__restrict__ AtB, long long ns) {
    const int b = blockIdx.y;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ns; i += (long long)gridDim.x * blockDim.x) {
        const real bv = -ut[b * ns + i];
        bof[b * ns + i] = bv;
        AtB[b * 2 * ns + i] = ux[b * ns + i] * bv;
        AtB[b * 2 * ns + ns + i] = uy[b * ns + i] * bv;
    }
}

// ------------------------------------------------------ weighted Theta Gram
// G = (P Theta V)^T (P Theta V), P^2 = diag(((Theta uk)^2 + eps^2)^(-1/2)), over the
// first K columns of V. A tile of TG_PIX consecutive pixels of one frame yields
// 4 rows per pixel (Psi_x, Psi_y of the frame; Mbar and Mbar' rows of the pair
// starting at the frame), one row per thread: the thread's offsets and
// bilinear weights are computed once per tile, its rows of the K basis vectors
// are generated four vectors at a time (loads of four vectors in flight) and
// stored scaled by P, column-major in shared memory (conflict-free stores).
// The (4x4 block of the upper triangle, row group) pairs are spread over all
// threads; each accumulates outer products of four rows at a time from
// 128-bit shared loads in FP32 registers and carries the running sums across
// tiles with Kahan compensation. At the end the row groups are combined in
// FP64 in shared memory, and the per-CTA partials by k_gram_reduce.
constexpr int TG_S = TG_ROWS + 4;  // column stride of the shared row tile
// column j starts at j * TG_S + 4 * (j / 4): the skew of four floats per group of
// four columns puts the 128-bit reads of the eight column groups a warp's 4x4
// blocks touch on eight different bank quads
__host__ __device__ constexpr int tg_col(int j) { return j * TG_S + 4 * (j / 4); }
constexpr int TG_MAXG = 8;         // row groups per 4x4 block at most
constexpr int TG_VEC = 8;          // basis vectors per step of the difference rows (16 loads in flight)

template <typename real>
__device__ __forceinline__ void warp_axis_s(int x, real v, int n, int &i0, int &i1, real &w, int wm) {
    const real vc = v > (real)16777216 ? (real)16777216 : (v < (real)-16777216 ? (real)-16777216 : v);
    const real fv = floor(vc);
    const int I = x + (int)fv;
    if (wm) { i0 = min(max(x + (int)round(vc), 0), n - 1); w = 0; }  // rounding and clipping
    else if (I < 0) { i0 = 0; w = 0; }
    else if (I >= n - 1) { i0 = n - 1; w = 0; }
    else { i0 = I; w = vc - fv; }
    if (!(v == v)) { i0 = x; w = 0; }
    i1 = min(i0 + 1, n - 1);
}


template <typename real>
__global__ void __launch_bounds__(TG_T, tg_min_blocks<real>()) k_theta_gram(const real *__restrict__ V, long long n, int Kmax, const int *__restrict__ Kp,
                                                     const real *__restrict__ uk, const real *__restrict__ s,
                                                     const real *__restrict__ sr, real eps2, int nx, int ny, int nt,
                                                     int rows, int wm, double *__restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smraw[];
    real *As = reinterpret_cast<real *>(smraw);  // [K4 * 4][TG_S], column j = basis vector j
    const int K = min(Kp[0], Kmax);
    const int K4 = (K + 3) / 4;
    const int nblk = K4 * (K4 + 1) / 2;
    const int nb1 = max(nblk, 1);
    const int RG = max(1, min(TG_MAXG, TG_T / nb1));
    const int tid = threadIdx.x;
    const int g = tid / nb1, blk = tid - g * nb1;
    const bool acc_on = g < RG && blk < nblk;
    // rows of group g: [r0, r1), r0 a multiple of 4; the RG groups cover all TG_ROWS rows
    const int rpg = (((TG_ROWS + RG - 1) / RG + 3) / 4) * 4;
    const int r0 = min(g * rpg, TG_ROWS), r1 = min(r0 + rpg, TG_ROWS);
    int I = 0, J = 0;
    if (acc_on) {
        int rem = blk;
        while (rem >= K4 - I) {
            rem -= K4 - I;
            ++I;
        }
        J = I + rem;
    }
    real sum[4][4], comp[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) sum[a][c] = comp[a][c] = 0;
    // rows: 0 = all four rows per pixel (64 pixels per tile), 1 = the Psi rows only,
    // 2 = the Mhat rows only (128 pixels per tile), 3 = the temporal differences L_t of
    // D1-OF only (one row per pixel, 256 pixels per tile; q = 4)
    const int ns = nx * ny;
    const int ppt = rows == 0 ? TG_PIX : (rows == 3 ? 4 * TG_PIX : 2 * TG_PIX);
    const int tpf = (ns + ppt - 1) / ppt;
    const int np = nt - 1;
    const int ntiles = tpf * (rows >= 2 ? np : nt);
    const int q = rows == 0 ? (tid & 3) : (rows == 3 ? 4 : (tid & 1) + (rows == 2 ? 2 : 0));
    const int pid = rows == 0 ? (tid >> 2) : (rows == 3 ? tid : (tid >> 1));
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int t = tile / tpf;
        const int pix = (tile - t * tpf) * ppt + pid;
        const bool inpix = pix < ns;
        const int y = inpix ? pix / nx : 0, x = inpix ? pix - y * nx : 0;
        bool valid = inpix && (q < 2 || t < np);
        if (q == 0 && x >= nx - 1) valid = false;
        if (q == 1 && y >= ny - 1) valid = false;
        // row value = f[oc] - (w00 f[o00] + w01 f[o01] + w10 f[o10] + w11 f[o11]) within one basis vector
        int oc = 0, o00 = 0, o01 = 0, o10 = 0, o11 = 0;
        real w00 = 0, w01 = 0, w10 = 0, w11 = 0;
        if (valid) {
            const int base = t * ns + pix;
            if (q == 0) {
                oc = base + 1;
                o00 = o01 = o10 = o11 = base;
                w00 = 1;
            } else if (q == 1) {
                oc = base + nx;
                o00 = o01 = o10 = o11 = base;
                w00 = 1;
            } else if (q == 4) {  // u(t+1) - u(t) at the pixel (t < nt - 1)
                oc = base + ns;
                o00 = o01 = o10 = o11 = base;
                w00 = 1;
            } else {
                const real *sv = (q == 2 ? s : sr) + 2LL * t * ns;
                int x0, x1, y0, y1;
                real wx, wy;
                warp_axis_s(x, sv[pix], nx, x0, x1, wx, wm);
                warp_axis_s(y, sv[ns + pix], ny, y0, y1, wy, wm);
                const int fa = (q == 2 ? t : t + 1) * ns, fb = (q == 2 ? t + 1 : t) * ns;
                oc = fa + pix;
                o00 = fb + y0 * nx + x0;
                o01 = fb + y0 * nx + x1;
                o10 = fb + y1 * nx + x0;
                o11 = fb + y1 * nx + x1;
                w00 = (1 - wx) * (1 - wy);
                w01 = wx * (1 - wy);
                w10 = (1 - wx) * wy;
                w11 = wx * wy;
            }
        }
        real sw = 0;
        if (valid) {
            const real nu = uk[oc] - (w00 * uk[o00] + w01 * uk[o01] + w10 * uk[o10] + w11 * uk[o11]);
            sw = (real)1 / sqrt(sqrt(nu * nu + eps2));
        }
        const real *f = V;
        if (rows == 1 || rows == 3) {
            // difference rows (Psi, L_t): f[oc] - f[o00], two loads per vector (the general form
            // below gives the same value, its other weights being zero)
            for (int j = 0; j < K4 * 4; j += TG_VEC, f += TG_VEC * n) {
                real val[TG_VEC];
#pragma unroll
                for (int u = 0; u < TG_VEC; ++u) {
                    val[u] = 0;
                    if (valid && j + u < K) {
                        const real *fu = f + (long long)u * n;
                        val[u] = fu[oc] - fu[o00];
                    }
                }
#pragma unroll
                for (int u = 0; u < TG_VEC; ++u)
                    if (j + u < K4 * 4) As[tg_col(j + u) + tid] = sw * val[u];
            }
        } else {
            for (int j = 0; j < K4 * 4; j += 4, f += 4 * n) {
                real val[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    val[u] = 0;
                    if (valid && j + u < K) {
                        const real *fu = f + (long long)u * n;
                        val[u] = fu[oc] - (w00 * fu[o00] + w01 * fu[o01] + w10 * fu[o10] + w11 * fu[o11]);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) As[tg_col(j + u) + tid] = sw * val[u];
            }
        }
        __syncthreads();
        if (acc_on) {
            real acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][c] = 0;
            const real *pa = As + tg_col(4 * I), *pb = As + tg_col(4 * J);
            for (int r = r0; r < r1; r += 4) {
                Quad<real> va[4], vb[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    va[a] = load_quad(pa + a * TG_S + r);
                    vb[a] = load_quad(pb + a * TG_S + r);
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        acc[a][c] += va[a].x * vb[c].x + va[a].y * vb[c].y + va[a].z * vb[c].z + va[a].w * vb[c].w;
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const real yv = acc[a][c] - comp[a][c];
                    const real tv = sum[a][c] + yv;
                    comp[a][c] = (tv - sum[a][c]) - yv;
                    sum[a][c] = tv;
                }
        }
        __syncthreads();
    }
    // combine the row groups in FP64 (the tile buffer is free now), one partial per CTA
    double *red = reinterpret_cast<double *>(smraw);  // [RG][nblk][16]
    if (acc_on) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) red[((long long)g * nblk + blk) * 16 + a * 4 + c] = (double)sum[a][c] - (double)comp[a][c];
    }
    __syncthreads();
    double *out = partial + (long long)blockIdx.x * Kmax * Kmax;
    for (int e = tid; e < nblk * 16; e += TG_T) {
        const int b = e >> 4, el = e & 15;
        int bi = 0, rem = b;
        while (rem >= K4 - bi) {
            rem -= K4 - bi;
            ++bi;
        }
        const int i = 4 * bi + (el >> 2), jj = 4 * (bi + rem) + (el & 3);
        double v = 0.0;
        for (int gg = 0; gg < RG; ++gg) v += red[((long long)gg * nblk + b) * 16 + el];
        if (i < K && jj < K && i <= jj) out[i * Kmax + jj] = v;
    }
}

// G[i][j] = sum over the per-CTA partials (upper triangle), mirrored. One warp per
// entry: lanes stride over the partials, then a fixed tree (deterministic); warps
// stride over the K^2 entries.
__global__ void k_gram_reduce(const double *__restrict__ partial, int nparts, int Kmax, const int *__restrict__ Kp,
                              double *__restrict__ G) {
    const int K = min(Kp[0], Kmax);
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int e = w0; e < K * K; e += nw) {
        const int i = e / K, j = e % K;
        if (i > j) continue;
        double s = 0.0;
#pragma unroll 8
        for (int c = lane; c < nparts; c += 32) s += partial[(long long)c * Kmax * Kmax + i * Kmax + j];
        s = warp_sum(s);
        if (lane == 0) {
            G[i * Kmax + j] = s;
            G[j * Kmax + i] = s;
        }
    }
}

// report[k] = {lam, resid, rnorm, basis, flag, of_min, of_max}
__global__ void k_report(double *__restrict__ rep, int *__restrict__ iter, const double *__restrict__ lam,
                         const double *__restrict__ resid2, const double *__restrict__ rn2, const int *__restrict__ K,
                         const int *__restrict__ flag, const int *__restrict__ Kof, int P, int of_ran, int expanded,
                         const int *__restrict__ appended) {
    const int k = iter[0];
    iter[0] = k + 1;
    double *r = rep + (long long)k * 8;
    r[0] = lam[0];
    r[1] = sqrt(resid2[0]);
    r[2] = expanded ? sqrt(rn2[0]) : 0.0;
    r[3] = (double)(K[0] - (expanded && appended[0] ? 1 : 0));
    r[4] = (double)flag[0];
    int mn = 1 << 30, mx = 0;
    if (of_ran)
        for (int b = 0; b < P; ++b) {
            mn = min(mn, Kof[b]);
            mx = max(mx, Kof[b]);
        }
    r[5] = of_ran ? (double)mn : 0.0;
    r[6] = of_ran ? (double)mx : 0.0;
}

static inline int fb(long long n) { return (int)std::min<long long>(152 * 8, (n + 255) / 256); }
static inline size_t mg_solve_smem(int ld) { return sizeof(double) * ((size_t)ld * (ld + 1) + ld); }

// ============================================================ Solve-OF
template <typename real>
static mof_status solve_of_impl(mof_problem *p, const mof_solver_params &prm, WS<real> &w, const real *u, real *s_out,
                                Timer *tm, cudaStream_t st) {
    const int P = p->nt - 1;
    const long long ns = p->ns, N2 = 2 * ns;
    const int Kof = w.Kof, ldU = w.of_ell + 1;
    const double tol = prm.breakdown_tol > 0 ? prm.breakdown_tol : (sizeof(real) == 8 ? 1e-10 : 1e-6);
    const dim3 blk2(32, 8);
    {
        Scope sc(tm, "of_fields", st);
        MOF_TRY(launch_of_fields<real>(p, u, prm.of_dr, w.ux, w.uy, w.ut, st));
        ::mof::count_launch(), k_of_rhs<real><<<dim3(fb(ns), P), 256, 0, st>>>(w.ux, w.uy, w.ut, w.bof, w.AtB, ns);
    }
    // The pairs are split into groups, each running its whole Solve-OF (GKB start,
    // initial Gram columns, GKS iterations) on its own stream: a group's small
    // FP64 solves occupy one SM per pair and are latency bound, and its GKB steps
    // are short launches, so the groups fill the GPU together. Every kernel works
    // per pair, so the grouping does not change the result.
    // the plain form: one pair per group, all on the solver's stream one after another
    const int G = prm.plain ? P : std::max(1, std::min(prm.of_streams > 0 ? prm.of_streams : AUTO_OF_STREAMS, P));
    const long long part_pair = of_partial_per_pair(p, Kof, w.of_ell);
    if (!prm.plain) MOF_CUDA(cudaEventRecord(w.gfork, st));
    for (int gi = 0; gi < G; ++gi) {
        const int b0 = (int)((long long)gi * P / G), nb = (int)((long long)(gi + 1) * P / G) - b0;
        const cudaStream_t gst = prm.plain ? st : w.gs[gi];
        if (!prm.plain) MOF_CUDA(cudaStreamWaitEvent(gst, w.gfork, 0));
        Krylov<real> kg;
        kg.partial = w.partial + b0 * part_pair;
        kg.err = w.err;
        kg.aux = w.kaux + 2LL * b0;
        const long long KK = (long long)Kof * Kof;
        real *Vg = w.Vof + (long long)b0 * Kof * N2, *sg = s_out + (long long)b0 * N2, *wvg = w.wv + (long long)b0 * N2;
        real *Ug = w.Uof + (long long)b0 * ldU * ns, *wug = w.wu + (long long)b0 * ns;
        const real *uxg = w.ux + (long long)b0 * ns, *uyg = w.uy + (long long)b0 * ns, *AtBg = w.AtB + (long long)b0 * N2;
        const real *bofg = w.bof + (long long)b0 * ns;
        int *Kvg = w.Kv_of + b0, *Kug = w.Ku_of + b0, *actg = w.act_of + b0, *appg = w.app_of + b0, *gkbg = w.gkb_of + b0;
        double *nrmg = w.nrm_of + b0, *bbg = w.bb_of + b0;
        const int pb = (nb + 63) / 64;
        BasisRef<real> BV{Vg, N2, Kof, nb, Kvg, gkbg};
        BasisRef<real> BU{Ug, ns, ldU, nb, Kug, gkbg};
        {
            Scope sc(tm, "of_gkb", gst);
            kg.norm2(bofg, ns, ns, nb, bbg, gst);
            ::mof::count_launch(), k_of_activate<<<pb, 64, 0, gst>>>(bbg, actg, gkbg, w.grow_of + b0, Kvg, Kug, w.beta1_of + b0, nb);
            kg.norm2(AtBg, N2, N2, nb, nrmg, gst);
            ::mof::count_launch(), k_sqrt_into<<<pb, 64, 0, gst>>>(nrmg, w.scale_of + b0, nb);
            // u_1 = b / ||b||
            kg.append(BU, Kug, bofg, ns, bbg, nullptr, 0.0, gkbg, nullptr, nullptr, gst);
            for (int j = 0; j < w.of_ell && j < prm.of_ell; ++j) {
                ::mof::count_launch(), k_of_upsT<real><<<dim3(fb(ns), nb), 256, 0, gst>>>(uxg, uyg, Ug, ldU, j, Vg, Kof, w.beta_of + b0, wvg, ns, gkbg);
                // V^T x = 0 by the recurrence; alpha (and alpha_1) = ||x|| with the append
                const int nv = kg.reorth_second_parts(BV, wvg, N2, nullptr, w.coef_of + (long long)b0 * Kof, gst);
                kg.append_parts(BV, Kvg, wvg, N2, nv, nrmg, j == 0 ? nullptr : w.alpha1_of + b0, tol, gkbg, nullptr, nullptr,
                                w.alpha_of + b0, j == 0 ? w.alpha1_of + b0 : nullptr, gst);
                ::mof::count_launch(), k_of_ups<real><<<dim3(fb(ns), nb), 256, 0, gst>>>(uxg, uyg, Vg, Kof, j, Ug, ldU, w.alpha_of + b0, wug, ns, gkbg);
                const int nu = kg.reorth_second_parts(BU, wug, ns, nullptr, w.coefU_of + (long long)b0 * ldU, gst);
                kg.append_parts(BU, Kug, wug, ns, nu, nrmg, w.beta1_of + b0, tol, gkbg, nullptr, nullptr, w.beta_of + b0, nullptr,
                                gst);
            }
        }
        const dim3 gg((p->nx + 31) / 32, (p->ny + 7) / 8, nb);
        BasisRef<real> BAg{Vg, N2, Kof, nb, Kvg, actg};
        const int gram_ctas = (int)((ns + ofc<real>() - 1) / ofc<real>());
        const int gram_red = (2 * Kof + 1 + 7) / 8;
        const real *bofg2 = w.bof + (long long)b0 * ns;
        const bool pq1 = prm.of_pq == 1;
        real *wfg = pq1 ? w.wf_of + (long long)b0 * ns : nullptr, *wlg = pq1 ? w.wl_of + (long long)b0 * 4 * ns : nullptr;
        if (!pq1) {
            Scope sc(tm, "of_gram", gst);
            const int ncol = std::min(prm.of_ell, Kof);
            ::mof::count_launch(), k_of_gram_cols<real><<<dim3(gram_ctas, nb, ncol), OFG_T, 0, gst>>>(Vg, Kof, Kvg, actg, 0, uxg, uyg, bofg2,
                                                                                                   p->nx, p->ny, kg.partial);
            ::mof::count_launch(), k_of_gram_reduce<<<dim3(gram_red, nb, ncol), 256, 0, gst>>>(kg.partial, gram_ctas, Kof, Kvg, actg, 0,
                                                                                             w.GA + b0 * KK, w.GL + b0 * KK,
                                                                                             w.gof + (long long)b0 * Kof);
        }
        ::mof::count_launch(), k_of_mg_init<<<nb, 256, 0, gst>>>(w.Mg_of + (long long)b0 * KK, Kof, actg, nb);
        // the one-pass projection with the Gram column needs 16-byte aligned component segments
        const bool pass_ok = !pq1 && Kof <= 64 && of_pass_applicable<real>(ns, Vg, wvg);
        SmallArgs sa{};
        sa.GA = w.GA + b0 * KK;
        sa.GL = w.GL + b0 * KK;
        sa.g = w.gof + (long long)b0 * Kof;
        sa.bb = w.bb_of + b0;
        sa.K = Kvg;
        sa.active = actg;
        sa.ld = Kof;
        sa.B = nb;
        sa.rule = MOF_RULE_GCV;
        sa.lam = w.gam + b0;
        sa.z = w.zof + (long long)b0 * Kof;
        sa.flag = w.flag_of + b0;
        sa.err = w.err;
        BasisRef<real> BS{Vg, N2, Kof, nb, Kvg, nullptr};
        const int wg_ctas = (int)std::min<long long>(WG_CTAS, (ns + WG_P - 1) / WG_P);
        for (int it = 0; it < prm.of_iters; ++it) {
            if (pq1) {
                // MM-GKS: IRLS weights of the current velocity (zero at the start), then the
                // weighted Grams of the whole basis
                Scope sc(tm, "of_irls", gst);
                ::mof::count_launch(), k_of_irls_weights<real><<<gg, blk2, 0, gst>>>(uxg, uyg, bofg2, it == 0 ? nullptr : sg,
                                                                                   (real)(prm.eps * prm.eps), wfg, wlg, p->nx,
                                                                                   p->ny, actg);
                ::mof::count_launch(), k_of_wgram<real><<<dim3(wg_ctas, nb), WG_T, wg_smem<real>(Kof), gst>>>(
                    Vg, Kof, Kvg, actg, uxg, uyg, bofg2, wfg, wlg, p->nx, p->ny, kg.partial);
                ::mof::count_launch(), k_of_wgram_reduce<<<dim3((wg_pstride(Kof) + 7) / 8, nb), 256, 0, gst>>>(
                    kg.partial, wg_ctas, Kof, Kvg, actg, w.GA + b0 * KK, w.GL + b0 * KK, w.gof + (long long)b0 * Kof,
                    w.bb_of + b0);
            }
            {
                Scope sc(tm, "of_small", gst);
                MOF_TRY(launch_small_solve(sa, gst));
            }
            {
                Scope sc(tm, "of_combine", gst);
                kg.combine(BS, sa.z, Kof, sg, N2, gst);
            }
            if (it == prm.of_iters - 1) break;
            if (pq1) {
                Scope sc(tm, "of_resid", gst);
                ::mof::count_launch(), k_of_resid_w<real><<<gg, blk2, 0, gst>>>(uxg, uyg, bofg2, sg, wfg, wlg, sa.lam, wvg, p->nx,
                                                                              p->ny, actg);
                // the growth test compares with the residual's own norm (the weights rescale it)
                kg.norm2(wvg, N2, N2, nb, w.rn_of + b0, gst);
                ::mof::count_launch(), k_sqrt_into<<<pb, 64, 0, gst>>>(w.rn_of + b0, w.scale_of + b0, nb);
            } else {
                Scope sc(tm, "of_resid", gst);
                ::mof::count_launch(), k_of_resid<real><<<gg, blk2, 0, gst>>>(uxg, uyg, AtBg, sg, sa.lam, wvg, p->nx, p->ny, actg);
            }
            {
                // Projection of the residual onto the complement of the stored basis's span in
                // one pass over the basis: V^T r from the Grams, d = Mg^-1 V^T r, then the fused
                // pass x' = r - V d with c2 = V^T x' and ||x'||^2; the append stores x'/||x'|| and
                // c2 / ||x'|| becomes the new column of Mg (see k_of_mg_init).
                double *cg = w.coef_of + (long long)b0 * Kof;
                double *Mgg = w.Mg_of + (long long)b0 * KK;
                {
                    Scope sc(tm, "of_reorth", gst);
                    ::mof::count_launch(), k_of_proj_gram<<<nb, 32, 0, gst>>>(sa.GA, sa.GL, sa.g, sa.z, sa.lam, Kvg, actg, Kof, cg);
                    ::mof::count_launch(), k_of_mg_solve<<<nb, 32, mg_solve_smem(Kof), gst>>>(Mgg, cg, Kof, Kvg, actg);
                }
                // at GKS iteration it the basis holds at most of_ell + it vectors (one append per iteration)
                const int kcap = std::min(Kof, prm.of_ell + it);
                if (pass_ok) {
                    // p = q = 2: the projection, the new vector's Gram columns and the append in
                    // one pass over the basis (no separate Gram-column pass after it)
                    Scope sc(tm, "of_subdot", gst);
                    MOF_TRY(launch_of_proj_gram_pass<real>(BAg, Kvg, ns, p->nx, p->ny, cg, wvg, w.q_of + (long long)b0 * N2, AtBg,
                                                           uxg, uyg, kg.partial, w.pres_of + (long long)b0 * of_pass_stride(Kof),
                                                           w.err, kcap, w.scale_of + b0, tol, w.grow_of + b0, w.GA + b0 * KK,
                                                           w.GL + b0 * KK,
                                                           w.gof + (long long)b0 * Kof, Mgg, w.nrm_of + b0, appg, kg.aux, gst));
                    continue;
                }
                bool fused;
                int nparts = 0;
                {
                    Scope sc(tm, "of_subdot", gst);
                    fused = kg.sub_dot(BAg, cg, Kof, wvg, N2, cg, gst, kcap, &nparts);
                }
                Scope sc(tm, "of_reorth", gst);
                if (fused) {
                    kg.append_parts(BAg, Kvg, wvg, N2, nparts, w.nrm_of + b0, w.scale_of + b0, tol, w.grow_of + b0, appg, nullptr,
                                    nullptr, nullptr, gst, kg.partial + (long long)nb * nparts * Kof);
                } else {
                    kg.subtract(BAg, cg, Kof, wvg, N2, wvg, N2, nullptr, gst);
                    kg.dots(BAg, wvg, N2, cg, Kof, 1.0, gst);
                    kg.norm2(wvg, N2, N2, nb, w.nrm_of + b0, gst);
                    kg.append(BAg, Kvg, wvg, N2, w.nrm_of + b0, w.scale_of + b0, tol, w.grow_of + b0, appg, nullptr, gst);
                }
                ::mof::count_launch(), k_of_mg_update<<<nb, 64, 0, gst>>>(Mgg, cg, w.nrm_of + b0, Kof, Kvg, appg, actg);
            }
            if (!pq1) {
                Scope sc(tm, "of_gram", gst);
                ::mof::count_launch(), k_of_gram_cols<real><<<dim3(gram_ctas, nb, 1), OFG_T, 0, gst>>>(Vg, Kof, Kvg, appg, 1, uxg, uyg, bofg2,
                                                                                                    p->nx, p->ny, kg.partial);
                ::mof::count_launch(), k_of_gram_reduce<<<dim3(gram_red, nb, 1), 256, 0, gst>>>(kg.partial, gram_ctas, Kof, Kvg, appg, 1,
                                                                                              w.GA + b0 * KK, w.GL + b0 * KK,
                                                                                              w.gof + (long long)b0 * Kof);
            }
        }
        if (!prm.plain) MOF_CUDA(cudaEventRecord(w.gdone[gi], gst));
    }
    if (!prm.plain)
        for (int gi = 0; gi < G; ++gi) MOF_CUDA(cudaStreamWaitEvent(st, w.gdone[gi], 0));
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

// ------------------------------------------------------------ Solve-OF on rescaled frames
// Sec. 4.1.5 / Sec. 5: with of_scale = a > 1 Solve-OF runs on the frames' a x a block means
// and the velocities are interpolated back to the full grid (times a). The coarse problem
// (geometry of the coarse frames; its projector is never used) and its workspace are
// created on first use, which callers make before any graph capture.
template <typename real>
static mof_status ensure_coarse(mof_problem *p, const mof_solver_params &prm, mof_problem **pc_out, WS<real> **wc_out) {
    const int a = prm.of_scale;
    Holder *h = holder(p);
    if (!h->coarse || h->coarse_scale != a) {
        if (h->coarse) {
            mof_problem_destroy(h->coarse);
            h->coarse = nullptr;
        }
        std::vector<int> na(p->nt, 1);
        std::vector<double> ang(p->nt, 0.0);
        mof_geometry g{p->nx / a, p->ny / a, p->nt, 1, na.data(), ang.data(), 1.0, 1.0};
        MOF_TRY(mof_problem_create(&g, p->precision, &h->coarse));
        h->coarse_scale = a;
    }
    WS<real> *&wc = ws_slot<real>(holder(h->coarse));
    MOF_TRY(ensure_ws<real>(h->coarse, prm, 1, wc));
    *pc_out = h->coarse;
    *wc_out = wc;
    return MOF_OK;
}

// err |= the coarse solve's error word, which is then cleared
__global__ void k_merge_err(int *__restrict__ err, int *__restrict__ cerr) {
    if (threadIdx.x == 0) {
        err[0] |= cerr[0];
        cerr[0] = 0;
    }
}

template <typename real>
static mof_status of_step(mof_problem *p, const mof_solver_params &prm, WS<real> &w, const real *u, real *s_out, Timer *tm,
                          cudaStream_t st) {
    if (prm.of_scale <= 1) return solve_of_impl<real>(p, prm, w, u, s_out, tm, st);
    mof_problem *pc = nullptr;
    WS<real> *wc = nullptr;
    MOF_TRY(ensure_coarse<real>(p, prm, &pc, &wc));  // already in place: nothing is allocated here
    {
        Scope sc(tm, "of_fields", st);
        MOF_TRY(launch_downsample<real>(p, prm.of_scale, u, wc->u, st));
    }
    MOF_TRY(solve_of_impl<real>(pc, prm, *wc, wc->u, wc->s, tm, st));
    Scope sc(tm, "of_fields", st);
    MOF_TRY(launch_upsample_velocity<real>(p, prm.of_scale, wc->s, s_out, st));
    ::mof::count_launch(), k_merge_err<<<1, 32, 0, st>>>(w.err, wc->err);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

// ============================================================ MMGKS-OF
// One MMGKS-OF solve (Alg. 1) as phases, so that several problems can be
// interleaved on their own streams (mof_solve_batch): begin() enqueues the set-up
// and the GKB start, step(k) outer iteration k (captured once per variant into a
// CUDA graph and replayed), end() the copies of the results, result() reads the
// report and the device error word after the stream has finished. Every
// data-dependent decision is taken on the device, so nothing synchronises the
// host before end().
template <typename real>
struct SolveRun {
    mof_problem *p = nullptr;
    mof_solver_params prm{};
    int n_outer = 0;
    const real *b_in = nullptr;
    real *u_out = nullptr, *s_out = nullptr, *sr_out = nullptr;
    mof_report *report = nullptr;
    WS<real> *wp = nullptr;
    Timer *tm = nullptr;
    cudaStream_t st = nullptr;
    long long n = 0, m = 0, ns = 0;
    int P = 0, Kmax = 0;
    double tol = 0;
    Krylov<real> kr;
    size_t tg_smem = 0;
    SmallArgs sa{};
    real eps2 = 0;
    std::vector<double> rep;
    int err = 0;

    mof_status begin(cudaStream_t ust);
    mof_status iteration(bool of_now, bool expand);
    mof_status step(int k);
    mof_status end();
    mof_status result();
};

template <typename real>
mof_status SolveRun<real>::begin(cudaStream_t ust) {
    Holder *h = holder(p);
    WS<real> *&slot = ws_slot<real>(h);
    MOF_TRY(ensure_ws<real>(p, prm, n_outer, slot));
    wp = slot;
    WS<real> &w = *wp;
    // all work runs on the problem's own stream, ordered after the caller's stream
    st = w.ss;
    MOF_CUDA(cudaEventRecord(w.join, ust));
    MOF_CUDA(cudaStreamWaitEvent(st, w.join, 0));
    tm = p->timing ? &h->timer : nullptr;
    if (tm) tm->reset();
    n = p->n;
    m = p->m;
    ns = p->ns;
    P = p->nt - 1;
    Kmax = w.Kmax;
    tol = prm.breakdown_tol > 0 ? prm.breakdown_tol : (sizeof(real) == 8 ? 1e-10 : 1e-6);
    kr.partial = w.partial;
    kr.err = w.err;
    kr.aux = w.kaux;
    tg_smem = theta_gram_smem<real>(Kmax);
    MOF_CUDA(cudaFuncSetAttribute(k_theta_gram<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tg_smem));

    BasisRef<real> BV{w.V, n, Kmax, 1, w.K, nullptr};
    BasisRef<real> BH{w.HV, m, Kmax, 1, w.K, nullptr};
    BasisRef<real> BU{w.U, m, w.ell + 1, 1, w.KU, w.gkb};
    {
        Scope sc(tm, "init", st);
        ::mof::count_launch(), k_fill_int<<<1, 32, 0, st>>>(w.K, 1, 0);
        ::mof::count_launch(), k_fill_int<<<1, 32, 0, st>>>(w.KU, 1, 0);
        ::mof::count_launch(), k_fill_int<<<1, 32, 0, st>>>(w.grow, 1, 1);
        ::mof::count_launch(), k_fill_int<<<1, 32, 0, st>>>(w.gkb, 1, 1);
        ::mof::count_launch(), k_fill_int<<<1, 32, 0, st>>>(w.err, 1, 0);
        ::mof::count_launch(), k_fill_int<<<1, 32, 0, st>>>(w.flag, 1, 0);
        ::mof::count_launch(), k_fill_int<<<1, 32, 0, st>>>(w.iter, 1, 0);
        ::mof::count_launch(), k_fill<real><<<fb(n), 256, 0, st>>>(w.u, n, (real)0);
        ::mof::count_launch(), k_fill<real><<<fb(2 * P * ns), 256, 0, st>>>(w.s, 2 * P * ns, (real)0);
        ::mof::count_launch(), k_fill<real><<<fb(2 * P * ns), 256, 0, st>>>(w.sr, 2 * P * ns, (real)0);
        ::mof::count_launch(), k_copy<real><<<fb(m), 256, 0, st>>>(b_in, w.b, m);
        MOF_TRY(launch_tile_bounds<real>(p, w.s, w.sr, w.rad_s, w.rad_sr, st));
    }
    // ---- GKB on H from b / ||b|| (Sec. 4.1.1), H V_l = U_{l+1} B_l
    {
        Scope sc(tm, "gkb", st);
        kr.norm2(w.b, m, m, 1, w.bb, st, true);  // ||b||^2 enters rho0^2 = ||b||^2 - ||c||^2 of DP
        ::mof::count_launch(), k_flag_nonfinite<<<1, 32, 0, st>>>(w.bb, w.err);
        ::mof::count_launch(), k_sqrt_into<<<1, 1, 0, st>>>(w.bb, w.beta1, 1);
        kr.append(BU, w.KU, w.b, m, w.bb, nullptr, 0.0, w.gkb, nullptr, nullptr, st);
        for (int j = 0; j < prm.ell; ++j) {
            MOF_TRY(launch_backproject<real>(p, w.U + (long long)j * m, w.r, st, prm.plain));
            if (j > 0) ::mof::count_launch(), k_axpy_dev<real><<<dim3(fb(n), 1), 256, 0, st>>>(w.r, n, w.V + (long long)(j - 1) * n, n, w.beta, n, w.gkb);
            kr.reorth_second(BV, w.r, n, nullptr, w.coef, w.nrm2, st);  // V^T x = 0 by the recurrence
            if (j == 0) ::mof::count_launch(), k_sqrt_into_if<<<1, 1, 0, st>>>(w.nrm2, w.alpha1, 1, w.gkb);
            ::mof::count_launch(), k_sqrt_into_if<<<1, 1, 0, st>>>(w.nrm2, w.alpha, 1, w.gkb);
            kr.append(BV, w.K, w.r, n, w.nrm2, j == 0 ? nullptr : w.alpha1, tol, w.gkb, nullptr, nullptr, st);
            MOF_TRY(launch_project<real>(p, w.V + (long long)j * n, w.uT, w.HV + (long long)j * m, st, prm.plain));
            ::mof::count_launch(), k_copy<real><<<fb(m), 256, 0, st>>>(w.HV + (long long)j * m, w.tm, m);
            ::mof::count_launch(), k_axpy_dev<real><<<dim3(fb(m), 1), 256, 0, st>>>(w.tm, m, w.U + (long long)j * m, m, w.alpha, m, w.gkb);
            kr.reorth_second(BU, w.tm, m, nullptr, w.coef, w.nrm2, st);
            ::mof::count_launch(), k_sqrt_into_if<<<1, 1, 0, st>>>(w.nrm2, w.beta, 1, w.gkb);
            kr.append(BU, w.KU, w.tm, m, w.nrm2, w.beta1, tol, w.gkb, nullptr, nullptr, st);
        }
        // breakdown scale of the expansions: ||H^T b|| = alpha_1 beta_1
        ::mof::count_launch(), k_mul_into<<<1, 1, 0, st>>>(w.alpha1, w.beta1, w.scaleR, 1);
        for (int j = 0; j < prm.ell; ++j) {
            DotVecs<real> xs{{w.HV + (long long)j * m, w.b, nullptr}, {m, m, 0}};
            DotOuts o{};
            o.o[0] = DotOut{w.GH + j, 0, Kmax, 0, 0, 1.0};
            o.o[1] = DotOut{w.gH, 0, 1, 0, 0, 1.0};
            kr.multidot(BH, 2, xs, o, st, true);
        }
    }
    sa = SmallArgs{};
    sa.GA = w.GH;
    sa.GL = w.GT;
    sa.g = w.gH;
    sa.bb = w.bb;
    sa.K = w.K;
    sa.active = nullptr;
    sa.ld = Kmax;
    sa.B = 1;
    sa.rule = prm.image_rule;
    sa.target2 = (prm.eta * prm.noise_norm) * (prm.eta * prm.noise_norm);
    sa.lam_fixed = prm.lam_fixed;
    sa.lam = w.lam;
    sa.z = w.z;
    sa.flag = w.flag;
    sa.err = w.err;
    eps2 = (real)(prm.eps * prm.eps);
    if (std::memcmp(&w.gkey, &prm, sizeof(prm)) != 0 || w.gkey_n != n_outer || w.gkey_wm != p->warp_mode) {
        w.drop_graphs();
        w.gkey = prm;
        w.gkey_n = n_outer;
        w.gkey_wm = p->warp_mode;
    }
    MOF_TRY(prepare_small_solve(Kmax));
    MOF_TRY(prepare_small_solve(w.Kof));
    if (prm.of_scale > 1) {
        mof_problem *pc;
        WS<real> *wc;
        MOF_TRY(ensure_coarse<real>(p, prm, &pc, &wc));
    }
    return MOF_OK;
}

// One outer iteration of Alg. 1 (k is tracked on the device).
template <typename real>
mof_status SolveRun<real>::iteration(bool of_now, bool expand) {
    WS<real> &w = *wp;
    BasisRef<real> BV{w.V, n, Kmax, 1, w.K, nullptr};
    BasisRef<real> BH{w.HV, m, Kmax, 1, w.K, nullptr};
        // The weighted Gram of Theta = [Psi; (L_t;) Mhat] in parts: the Psi rows (and the
        // temporal differences of D1-OF) depend on the basis and u_k only, so they are
        // accumulated on a side stream while Solve-OF runs; the Mhat rows follow the new
        // flow. The reduction adds all sets of partials.
        const long long gsz = (long long)w.gram_ctas * Kmax * Kmax;
        double *gpart_psi = w.gpart, *gpart_m = w.gpart + gsz, *gpart_t = w.gpart + 2 * gsz;
        const int nsets = prm.temporal_tv ? 3 : 2;
        const cudaStream_t pst = of_now ? w.side : st;
        if (of_now) {
            MOF_CUDA(cudaEventRecord(w.side_fork, st));
            MOF_CUDA(cudaStreamWaitEvent(w.side, w.side_fork, 0));
        }
        {
            Scope sc(tm, "theta_gram", pst);
            ::mof::count_launch(), k_theta_gram<real><<<w.gram_ctas, TG_T, tg_smem, pst>>>(w.V, n, Kmax, w.K, w.u, w.s, w.sr, eps2, p->nx,
                                                                                      p->ny, p->nt, 1, p->warp_mode, gpart_psi);
            if (prm.temporal_tv)
                ::mof::count_launch(), k_theta_gram<real><<<w.gram_ctas, TG_T, tg_smem, pst>>>(w.V, n, Kmax, w.K, w.u, w.s, w.sr, eps2,
                                                                                          p->nx, p->ny, p->nt, 3, p->warp_mode, gpart_t);
        }
        if (of_now) {
            MOF_CUDA(cudaEventRecord(w.side_done, w.side));
            MOF_TRY(of_step<real>(p, prm, w, w.u, w.s, tm, st));
            Scope sc(tm, "reverse_flow", st);
            MOF_TRY(launch_reverse_flow<real>(p, w.s, w.rad_rev, w.dest, w.sr, st));
            MOF_TRY(launch_tile_bounds<real>(p, w.s, w.sr, w.rad_s, w.rad_sr, st));
        }
        {
            Scope sc(tm, "theta_gram", st);
            ::mof::count_launch(), k_theta_gram<real><<<w.gram_ctas, TG_T, tg_smem, st>>>(w.V, n, Kmax, w.K, w.u, w.s, w.sr, eps2, p->nx,
                                                                                     p->ny, p->nt, 2, p->warp_mode, gpart_m);
            if (of_now) MOF_CUDA(cudaStreamWaitEvent(st, w.side_done, 0));
            ::mof::count_launch(), k_gram_reduce<<<152, 256, 0, st>>>(w.gpart, nsets * w.gram_ctas, Kmax, w.K, w.GT);
        }
        {
            Scope sc(tm, "small_solve", st);
            MOF_TRY(launch_small_solve(sa, st));
        }
        {
            Scope sc(tm, "combine", st);
            kr.combine(BV, w.z, Kmax, w.un, n, st);
            kr.combine_minus(BH, w.z, Kmax, w.b, m, w.tm, m, w.nrm2b, st);  // H V z - b
        }
        if (expand) {
            {
                Scope sc(tm, "backproject", st);
                MOF_TRY(launch_backproject<real>(p, w.tm, w.tn, st, prm.plain));
            }
            {
                Scope sc(tm, "reg_normal", st);
                MOF_TRY(launch_reg_normal<real>(p, prm.temporal_tv, w.un, w.u, w.s, w.sr, w.rad_s, w.rad_sr, prm.eps, 1.0, w.lam, w.tn, w.q, w.r,
                                                st));
            }
            {
                Scope sc(tm, "reorth", st);
                // V^T r = (G_H + lam G_Theta) z - g_H exactly: the first projection from the Grams
                ::mof::count_launch(), k_of_proj_gram<<<1, 32, 0, st>>>(w.GH, w.GT, w.gH, w.z, w.lam, w.K, nullptr, Kmax, w.c1);
                kr.reorth_second(BV, w.r, n, w.c1, w.coef, w.nrm2, st);
                kr.append(BV, w.K, w.r, n, w.nrm2, w.scaleR, tol, w.grow, w.appended, w.vnew, st);
            }
            {
                Scope sc(tm, "project", st);
                MOF_TRY(launch_project<real>(p, w.vnew, w.uT, w.hvnew, st, prm.plain));
                ::mof::count_launch(), k_store_slot<real><<<fb(m), 256, 0, st>>>(w.HV, m, w.K, w.appended, w.hvnew);
            }
            {
                Scope sc(tm, "gram_h", st);
                BasisRef<real> BHn{w.HV, m, Kmax, 1, w.K, w.appended};
                DotVecs<real> xs{{w.hvnew, w.b, nullptr}, {m, m, 0}};
                DotOuts o{};
                o.o[0] = DotOut{w.GH, 0, Kmax, 1, 1, 1.0};
                o.o[1] = DotOut{w.gH, 0, 1, 0, 0, 1.0};
                kr.multidot(BHn, 2, xs, o, st, true);
                ::mof::count_launch(), k_sym_last<<<1, 64, 0, st>>>(w.GH, Kmax, w.K, w.appended);
            }
        }
        {
            Scope sc(tm, "misc", st);
            ::mof::count_launch(), k_copy<real><<<fb(n), 256, 0, st>>>(w.un, w.u, n);
            // the Solve-OF basis sizes live in the coarse workspace when Solve-OF runs downsampled
            const int *kof = w.Kv_of;
            if (prm.of_scale > 1 && holder(p)->coarse) kof = ws_slot<real>(holder(holder(p)->coarse))->Kv_of;
            ::mof::count_launch(), k_report<<<1, 1, 0, st>>>(w.report, w.iter, w.lam, w.nrm2b, w.nrm2, w.K, w.flag, kof, P,
                                                             of_now ? 1 : 0, expand ? 1 : 0, w.appended);
        }
        MOF_LAUNCH_CHECK();
        return MOF_OK;
}

template <typename real>
mof_status SolveRun<real>::step(int k) {
    WS<real> &w = *wp;
    const bool of_now = prm.tau > 0 && (k % prm.tau) == 0;
    const bool expand = k < n_outer - 1;
    if (prm.plain) return iteration(of_now, expand);  // every launch from the host, no graph
    auto &G = w.graphs[(of_now ? 1 : 0) | (expand ? 2 : 0) | (tm ? 4 : 0)];
    if (!G.exec) {
        if (tm) {
            tm->sink = &G.ev;
            tm->owned = &G.owned;
        }
        const long long before = launches_so_far();
        MOF_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        const mof_status cs = iteration(of_now, expand);
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(st, &graph);
        G.kernels = launches_so_far() - before;
        count_launches_add(-G.kernels);  // captured, not executed
        if (tm) {
            tm->sink = nullptr;
            tm->owned = nullptr;
        }
        if (cs != MOF_OK || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            w.drop_graphs();
            if (cs != MOF_OK) return cs;
            return cuda_fail(ce, "graph capture of an outer iteration", __FILE__, __LINE__);
        }
        const cudaError_t ie = cudaGraphInstantiate(&G.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            G.exec = nullptr;
            return cuda_fail(ie, "graph instantiation", __FILE__, __LINE__);
        }
    }
    MOF_CUDA(cudaGraphLaunch(G.exec, st));
    count_launches_add(G.kernels);
    if (tm) {
        MOF_CUDA(cudaStreamSynchronize(st));
        tm->collect_list(G.ev);
    }
    return MOF_OK;
}

template <typename real>
mof_status SolveRun<real>::end() {
    WS<real> &w = *wp;
    MOF_LAUNCH_CHECK();
    if (u_out) MOF_CUDA(cudaMemcpyAsync(u_out, w.u, sizeof(real) * n, cudaMemcpyDeviceToDevice, st));
    if (s_out) MOF_CUDA(cudaMemcpyAsync(s_out, w.s, sizeof(real) * 2 * P * ns, cudaMemcpyDeviceToDevice, st));
    if (sr_out) MOF_CUDA(cudaMemcpyAsync(sr_out, w.sr, sizeof(real) * 2 * P * ns, cudaMemcpyDeviceToDevice, st));
    rep.assign((size_t)n_outer * 8, 0.0);
    err = 0;
    MOF_CUDA(cudaMemcpyAsync(rep.data(), w.report, sizeof(double) * rep.size(), cudaMemcpyDeviceToHost, st));
    MOF_CUDA(cudaMemcpyAsync(&err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    return MOF_OK;
}

template <typename real>
mof_status SolveRun<real>::result() {
    MOF_CUDA(cudaStreamSynchronize(st));
    if (tm) tm->collect();
    if (report)
        for (int k = 0; k < n_outer; ++k) {
            const double *r = &rep[(size_t)k * 8];
            report[k].lambda = r[0];
            report[k].resid = r[1];
            report[k].rnorm = r[2];
            report[k].basis = (int)r[3];
            report[k].flag = (int)r[4];
            report[k].of_basis_min = (int)r[5];
            report[k].of_basis_max = (int)r[6];
        }
    if (err & 4) return fail(MOF_ETIMEOUT, "a bounded device wait ran out (code %d)", err);
    if (err & 16) return fail(MOF_ENUMERIC, "the data b hold a non-finite value (code %d)", err);
    if (err & 8) return fail(MOF_ENUMERIC, "a basis exceeded an internal size bound (code %d)", err);
    if (err) return fail(MOF_ENUMERIC, "device reported a numerical failure (code %d): factorisation or non-finite value", err);
    return MOF_OK;
}

template <typename real>
static mof_status solve_impl(mof_problem *p, const mof_solver_params &prm, int n_outer, const real *b_in, real *u_out,
                             real *s_out, real *sr_out, mof_report *report, cudaStream_t ust) {
    SolveRun<real> run;
    run.p = p;
    run.prm = prm;
    run.n_outer = n_outer;
    run.b_in = b_in;
    run.u_out = u_out;
    run.s_out = s_out;
    run.sr_out = sr_out;
    run.report = report;
    MOF_TRY(run.begin(ust));
    for (int k = 0; k < n_outer; ++k) MOF_TRY(run.step(k));
    MOF_TRY(run.end());
    return run.result();
}

template <typename real>
static mof_status solve_of_entry(mof_problem *p, const mof_solver_params &prm, const real *u, real *s, cudaStream_t ust) {
    Holder *h = holder(p);
    WS<real> *&wp = ws_slot<real>(h);
    MOF_TRY(ensure_ws<real>(p, prm, 1, wp));
    WS<real> &w = *wp;
    Timer *tm = p->timing ? &h->timer : nullptr;
    if (tm) tm->reset();
    MOF_TRY(prepare_small_solve(w.Kof));
    if (prm.of_scale > 1) {
        mof_problem *pc;
        WS<real> *wc;
        MOF_TRY(ensure_coarse<real>(p, prm, &pc, &wc));
    }
    // all work on the problem's own stream, ordered after the caller's stream
    const cudaStream_t st = w.ss;
    MOF_CUDA(cudaEventRecord(w.join, ust));
    MOF_CUDA(cudaStreamWaitEvent(st, w.join, 0));
    const long long nimg = p->n, nvel = (long long)(p->nt - 1) * 2 * p->ns;
    if (tm || prm.plain) {  // timed calls and the plain form run eagerly
        ::mof::count_launch(), k_fill_int<<<1, 32, 0, st>>>(w.err, 1, 0);
        MOF_TRY(of_step<real>(p, prm, w, u, s, tm, st));
    } else {
        // one captured graph per parameter set, over workspace copies of u and s (fixed
        // addresses), replayed: the Solve-OF launches thousands of short kernels
        if (w.ofgraph.exec && std::memcmp(&w.ofkey, &prm, sizeof(prm)) != 0) w.drop_of_graph();
        if (!w.ofgraph.exec) {
            const long long before = launches_so_far();
            MOF_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            ::mof::count_launch(), k_fill_int<<<1, 32, 0, st>>>(w.err, 1, 0);
            const mof_status cs = of_step<real>(p, prm, w, w.u, w.s, nullptr, st);
            cudaGraph_t graph = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(st, &graph);
            w.ofgraph.kernels = launches_so_far() - before;
            count_launches_add(-w.ofgraph.kernels);  // captured, not executed
            if (cs != MOF_OK || ce != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                if (cs != MOF_OK) return cs;
                return cuda_fail(ce, "graph capture of Solve-OF", __FILE__, __LINE__);
            }
            const cudaError_t ie = cudaGraphInstantiate(&w.ofgraph.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) {
                w.ofgraph.exec = nullptr;
                return cuda_fail(ie, "graph instantiation", __FILE__, __LINE__);
            }
            w.ofkey = prm;
        }
        MOF_CUDA(cudaMemcpyAsync(w.u, u, sizeof(real) * nimg, cudaMemcpyDeviceToDevice, st));
        MOF_CUDA(cudaGraphLaunch(w.ofgraph.exec, st));
        count_launches_add(w.ofgraph.kernels);
        MOF_CUDA(cudaMemcpyAsync(s, w.s, sizeof(real) * nvel, cudaMemcpyDeviceToDevice, st));
    }
    int err = 0;
    MOF_CUDA(cudaMemcpyAsync(&err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    MOF_CUDA(cudaStreamSynchronize(st));
    if (tm) tm->collect();
    if (err & 4) return fail(MOF_ETIMEOUT, "a bounded device wait ran out (code %d)", err);
    if (err & 8) return fail(MOF_ENUMERIC, "a basis exceeded an internal size bound (code %d)", err);
    if (err) return fail(MOF_ENUMERIC, "device reported a numerical failure (code %d)", err);
    return MOF_OK;
}

static mof_status check_params(const mof_problem *p, const mof_solver_params *prm, int n_outer, bool image_step = true) {
    if (!p || !prm) return fail(MOF_EINVAL, "null problem or parameters");
    if (n_outer < 1) return fail(MOF_EINVAL, "n_outer must be >= 1");
    if (prm->ell < 1 || prm->of_ell < 1 || prm->of_iters < 1 || prm->tau < 0 || prm->of_dr < 1 || prm->of_dr > 64 ||
        prm->of_streams < 0 || prm->of_streams > MAX_OF_STREAMS)
        return fail(MOF_EINVAL, "invalid solver parameters");
    if (prm->ell + n_outer > 60 || prm->of_ell + prm->of_iters > 64)
        return fail(MOF_EUNSUPPORTED,
                    "Krylov bases larger than 60 (image step) / 64 (Solve-OF) vectors are not supported "
                    "(ell + n_outer = %d, of_ell + of_iters = %d)",
                    prm->ell + n_outer, prm->of_ell + prm->of_iters);
    if (!(prm->eps > 0) || !std::isfinite(prm->eps)) return fail(MOF_EINVAL, "eps must be finite and > 0");
    if (prm->temporal_tv != 0 && prm->temporal_tv != 1) return fail(MOF_EINVAL, "temporal_tv must be 0 or 1");
    if (prm->of_pq != 1 && prm->of_pq != 2) return fail(MOF_EINVAL, "of_pq must be 1 or 2 (got %d)", prm->of_pq);
    if (prm->plain != 0 && prm->plain != 1) return fail(MOF_EINVAL, "plain must be 0 or 1 (got %d)", prm->plain);
    if (prm->of_scale < 1 || p->nx % prm->of_scale || p->ny % prm->of_scale || p->nx / prm->of_scale < 2 ||
        p->ny / prm->of_scale < 2)
        return fail(MOF_EINVAL, "of_scale must be >= 1, divide nx and ny and leave frames of at least 2x2 (got %d for %d x %d)",
                    prm->of_scale, p->nx, p->ny);
    if (!image_step) return MOF_OK;
    if (prm->image_rule == MOF_RULE_DP && !(prm->noise_norm >= 0))
        return fail(MOF_EINVAL, "the discrepancy principle needs noise_norm >= 0");
    if (prm->image_rule == MOF_RULE_FIXED && !(prm->lam_fixed > 0)) return fail(MOF_EINVAL, "fixed rule needs lam_fixed > 0");
    if (prm->image_rule < 0 || prm->image_rule > 2) return fail(MOF_EINVAL, "unknown image rule");
    return MOF_OK;
}

}  // namespace mof

using namespace mof;

extern "C" {

mof_status mof_solve_of(mof_problem *p, const mof_solver_params *prm, const void *u, void *s, void *stream) {
    MOF_TRY(check_params(p, prm, 1, false));
    if (!u || !s) return fail(MOF_EINVAL, "null array");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (p->precision == MOF_FP64) return solve_of_entry<double>(p, *prm, (const double *)u, (double *)s, st);
    return solve_of_entry<float>(p, *prm, (const float *)u, (float *)s, st);
}

mof_status mof_solve(mof_problem *p, const mof_solver_params *prm, int n_outer, const void *b, void *u_out, void *s_out,
                     void *sr_out, mof_report *report, void *stream) {
    MOF_TRY(check_params(p, prm, n_outer));
    if (!b || !u_out) return fail(MOF_EINVAL, "null b or u_out");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (p->precision == MOF_FP64)
        return solve_impl<double>(p, *prm, n_outer, (const double *)b, (double *)u_out, (double *)s_out, (double *)sr_out,
                                  report, st);
    return solve_impl<float>(p, *prm, n_outer, (const float *)b, (float *)u_out, (float *)s_out, (float *)sr_out, report,
                             st);
}

// One problem of a batch in either precision.
struct AnyRun {
    int fp64 = 0;
    SolveRun<float> f;
    SolveRun<double> d;
    mof_status begin(cudaStream_t st) { return fp64 ? d.begin(st) : f.begin(st); }
    mof_status step(int k) { return fp64 ? d.step(k) : f.step(k); }
    mof_status end() { return fp64 ? d.end() : f.end(); }
    mof_status result() { return fp64 ? d.result() : f.result(); }
};

static mof_status check_batch(mof_problem *const *ps, int count, const mof_solver_params *prm, int n_outer,
                              const void *const *b, void *const *u_out) {
    if (!ps || !prm || !b || !u_out) return fail(MOF_EINVAL, "null batch array");
    if (count < 1) return fail(MOF_EINVAL, "batch count must be >= 1");
    for (int i = 0; i < count; ++i) {
        if (!ps[i] || !b[i] || !u_out[i]) return fail(MOF_EINVAL, "null problem, b or u_out at batch index %d", i);
        for (int j = 0; j < i; ++j)
            if (ps[j] == ps[i]) return fail(MOF_EINVAL, "problem at batch index %d repeats index %d", i, j);
        const mof_status st = check_params(ps[i], &prm[i], n_outer);
        if (st != MOF_OK) return st;
    }
    return MOF_OK;
}

// Enqueue every problem's solve, interleaved outer iteration by outer iteration on
// the problems' own streams, then wait for all of them.
static mof_status batch_run(mof_problem *const *ps, int count, const mof_solver_params *prm, int n_outer,
                            const void *const *b, void *const *u_out, void *const *s_out, mof_report *const *reports,
                            cudaStream_t st) {
    std::vector<AnyRun> runs((size_t)count);
    for (int i = 0; i < count; ++i) {
        AnyRun &r = runs[i];
        r.fp64 = ps[i]->precision == MOF_FP64;
        void *so = s_out ? s_out[i] : nullptr;
        mof_report *rep = reports ? reports[i] : nullptr;
        if (r.fp64) {
            r.d.p = ps[i];
            r.d.prm = prm[i];
            r.d.n_outer = n_outer;
            r.d.b_in = (const double *)b[i];
            r.d.u_out = (double *)u_out[i];
            r.d.s_out = (double *)so;
            r.d.report = rep;
        } else {
            r.f.p = ps[i];
            r.f.prm = prm[i];
            r.f.n_outer = n_outer;
            r.f.b_in = (const float *)b[i];
            r.f.u_out = (float *)u_out[i];
            r.f.s_out = (float *)so;
            r.f.report = rep;
        }
        MOF_TRY(r.begin(st));
    }
    for (int k = 0; k < n_outer; ++k)
        for (auto &r : runs) MOF_TRY(r.step(k));
    for (auto &r : runs) MOF_TRY(r.end());
    mof_status first = MOF_OK;
    for (int i = 0; i < count; ++i) {
        const mof_status rs = runs[i].result();
        if (rs != MOF_OK && first == MOF_OK) {
            char msg[512];
            std::snprintf(msg, sizeof(msg), "%s", mof_last_error());
            first = fail(rs, "batch index %d: %s", i, msg);
        }
    }
    return first;
}

mof_status mof_solve_batch(mof_problem *const *problems, int count, const mof_solver_params *params, int n_outer,
                           const void *const *b, void *const *u_out, void *const *s_out, mof_report *const *reports,
                           void *stream) {
    MOF_TRY(check_batch(problems, count, params, n_outer, b, u_out));
    return batch_run(problems, count, params, n_outer, b, u_out, s_out, reports, reinterpret_cast<cudaStream_t>(stream));
}

mof_status mof_autotune(mof_problem *const *problems, int count, mof_solver_params *params, int n_probe,
                        const void *const *b, void *const *u_scratch, double *best_ms, void *stream) {
    if (n_probe < 1) return fail(MOF_EINVAL, "n_probe must be >= 1");
    MOF_TRY(check_batch(problems, count, params, n_probe, b, u_scratch));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int maxp = 1;
    for (int i = 0; i < count; ++i) maxp = std::max(maxp, problems[i]->nt - 1);
    std::vector<mof_solver_params> trial(params, params + count);
    cudaEvent_t e0, e1;
    MOF_CUDA(cudaEventCreate(&e0));
    MOF_CUDA(cudaEventCreate(&e1));
    int best = -1;
    float best_t = 0.0f;
    mof_status out = MOF_OK;
    for (int g : {1, 2, 4, 8, 16, 32, 64}) {
        if (g > maxp && g != 1) continue;
        for (auto &t : trial) t.of_streams = g;
        // the first run captures the graphs of this configuration; the second is timed
        out = batch_run(problems, count, trial.data(), n_probe, b, u_scratch, nullptr, nullptr, st);
        if (out != MOF_OK) break;
        if (cudaEventRecord(e0, st) != cudaSuccess) break;
        out = batch_run(problems, count, trial.data(), n_probe, b, u_scratch, nullptr, nullptr, st);
        if (out != MOF_OK) break;
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        if (best < 0 || t < best_t) {
            best = g;
            best_t = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (out != MOF_OK) return out;
    for (int i = 0; i < count; ++i) params[i].of_streams = best;
    if (best_ms) *best_ms = best_t;
    return MOF_OK;
}

mof_status mof_solve_host(mof_problem *p, const mof_solver_params *prm, int n_outer, const void *b_host, void *u_host,
                          void *s_host, void *sr_host, mof_report *report, void *stream) {
    MOF_TRY(check_params(p, prm, n_outer));
    if (!b_host || !u_host) return fail(MOF_EINVAL, "null b or u");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t es = p->precision == MOF_FP64 ? 8 : 4;
    Holder *h = holder(p);
    if (!h->host_stage) MOF_CUDA(cudaMalloc(&h->host_stage, es * (p->m + p->n + 2 * p->nv) + 1024));
    char *base = static_cast<char *>(h->host_stage);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    void *db = base, *du = base + al(es * p->m), *ds = (char *)du + al(es * p->n), *dsr = (char *)ds + es * p->nv;
    MOF_CUDA(cudaMemcpyAsync(db, b_host, es * p->m, cudaMemcpyHostToDevice, st));
    MOF_TRY(mof_solve(p, prm, n_outer, db, du, s_host ? ds : nullptr, sr_host ? dsr : nullptr, report, stream));
    MOF_CUDA(cudaMemcpyAsync(u_host, du, es * p->n, cudaMemcpyDeviceToHost, st));
    if (s_host) MOF_CUDA(cudaMemcpyAsync(s_host, ds, es * p->nv, cudaMemcpyDeviceToHost, st));
    if (sr_host) MOF_CUDA(cudaMemcpyAsync(sr_host, dsr, es * p->nv, cudaMemcpyDeviceToHost, st));
    MOF_CUDA(cudaStreamSynchronize(st));
    return MOF_OK;
}

mof_status mof_get_timing(const mof_problem *p, int cap, const char **names, double *ms, long long *launches, int *count) {
    if (!p) return fail(MOF_EINVAL, "null problem");
    const Holder *h = static_cast<const Holder *>(p->ws);
    const int nc = h ? (int)h->timer.names.size() : 0;
    if (count) *count = nc;
    for (int i = 0; i < nc && i < cap; ++i) {
        if (names) names[i] = h->timer.names[i].c_str();
        if (ms) ms[i] = h->timer.ms[i];
        if (launches) launches[i] = h->timer.count[i];
    }
    return MOF_OK;
}

}  // extern "C"
