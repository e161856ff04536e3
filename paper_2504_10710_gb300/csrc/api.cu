// C ABI of the GLL p-multigrid solver (include/glls.h): problem set-up and
// upload, the gamma-cycle driver (Algorithm 2) and the outer flexible CG.
#include "../../include/glls.h"
#include "device.cuh"
#include "setup.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

using namespace glls;

namespace {

thread_local std::string g_last_error;

// Device-wide operations of the library are serialised: stream capture (of
// the solve graphs) on one side, and on the other the calls that synchronise
// the whole device (cudaDeviceSynchronize, cudaFree) or change kernel
// attributes, which are not allowed while any stream of the context is
// capturing, whichever thread issues them.  Taken around each capture, the
// device phase of problem_create / problem_clone, and glls_problem_destroy.
std::recursive_mutex g_device_mutex;

// Failure injection for tests (glls_debug_fail_alloc_after): when >= 0, the
// number of device allocations that may still succeed; later ones fail with
// cudaErrorMemoryAllocation as if cudaMalloc had run out of memory.
std::atomic<long long> g_alloc_countdown{-1};

cudaError_t dev_malloc(void** p, size_t bytes) {
    if (g_alloc_countdown.load() >= 0 && g_alloc_countdown.fetch_sub(1) <= 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

glls_status fail(glls_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

// Makes the problem's device current for the duration of an entry point and
// restores the caller's current device when it returns.
struct DeviceScope {
    int prev = -1;
    bool restore = false;
    cudaError_t err = cudaSuccess;
    explicit DeviceScope(int dev) {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) {
            err = cudaSetDevice(dev);
            restore = err == cudaSuccess;
        }
    }
    ~DeviceScope() {
        if (restore) cudaSetDevice(prev);
    }
};

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(e_ == cudaErrorMemoryAllocation ? GLLS_ERR_OOM : GLLS_ERR_CUDA,            \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                       \
    } while (0)

template <typename T>
struct LevelStore {
    DevLevel<T> dev;
    T* r = nullptr;    // level right-hand side (coarse levels)
    T* x = nullptr;    // level iterate
    T* y = nullptr;    // A x scratch
    T* t1 = nullptr;   // transfer temporaries
    T* t2 = nullptr;
};

}  // namespace

// Read-only mesh data (geometry factors, line bands, transfers, coarse
// inverse, mass), shared by a problem and its clones; freed with the last one.
struct SharedData {
    int device = 0;
    std::vector<void*> allocs;
    size_t bytes = 0;
    ~SharedData() {
        DeviceScope scope(device);
        for (void* a : allocs) cudaFree(a);
    }
};

struct glls_problem {
    int device = 0;
    std::shared_ptr<SharedData> shared;
    int dim = 2;
    int nelem[3] = {1, 1, 1};
    int p = 1;
    int smoother = 0, restriction = 0;
    int nrhs = 1;          // right-hand sides solved together (vectors hold nrhs copies of their grid)
    std::vector<int> orders;
    std::vector<LevelStore<double>> L64;
    std::vector<LevelStore<float>> L32;
    DevCoarse<double> C64;
    DevCoarse<float> C32;
    long long N = 0;       // fine nodes
    long long N0 = 0;      // coarsest nodes
    // fine-level FP64 solve state
    double *f = nullptr, *g = nullptr, *v = nullptr, *f0 = nullptr;
    const double* mass = nullptr;
    double *xk = nullptr, *rk = nullptr, *pk = nullptr, *qk = nullptr, *zk = nullptr, *yk = nullptr;
    double *S = nullptr, *part = nullptr, *hostS = nullptr;
    unsigned* ticket = nullptr;
    float *r32 = nullptr, *z32 = nullptr;
    std::vector<void*> allocs;
    size_t bytes = 0;
    double setup_ms = 0.0;
    double setup_phase_ms[6] = {0, 0, 0, 0, 0, 0};   // see glls_info
    cudaStream_t capture_stream = nullptr, capture_stream2 = nullptr;
    // cached graph of one outer iteration (host-driven loop) and of the whole
    // solve (device-driven loop)
    cudaGraphExec_t iter_exec = nullptr;
    int g_gamma = -1, g_m = -1, g_prec = -1, g_krylov = -1;
    double g_alpha = 0.0;
    cudaGraphExec_t solve_exec = nullptr;
    glls_solve_opts solve_key{};
    long long kern_fixed = 0, kern_iter = 0;   // kernel nodes of the solve graph (outside / inside the loop)
    // GMRES workspace (allocated on first use): Krylov basis V, preconditioned
    // basis Z, Hessenberg column halves, partial sums
    double *gV = nullptr, *gZ = nullptr, *gh = nullptr, *gpart = nullptr;
    int gm = 0;
    bool has_rhs = false, has_dirichlet = false;

    template <typename T>
    cudaError_t alloc(T** ptr, size_t count) {
        void* p_ = nullptr;
        cudaError_t e = dev_malloc(&p_, sizeof(T) * (count ? count : 1));
        if (e != cudaSuccess) return e;
        allocs.push_back(p_);
        bytes += sizeof(T) * (count ? count : 1);
        *ptr = static_cast<T*>(p_);
        return cudaSuccess;
    }
    // read-only data: allocated into the shared block
    template <typename T, typename S>
    cudaError_t upload(const T** dst, const std::vector<S>& src) {
        T* d = nullptr;
        void* p_ = nullptr;
        const size_t count = src.size() ? src.size() : 1;
        cudaError_t e = dev_malloc(&p_, sizeof(T) * count);
        if (e != cudaSuccess) return e;
        shared->allocs.push_back(p_);
        shared->bytes += sizeof(T) * count;
        d = static_cast<T*>(p_);
        std::vector<T> tmp(src.begin(), src.end());
        e = cudaMemcpy(d, tmp.data(), sizeof(T) * tmp.size(), cudaMemcpyHostToDevice);
        *dst = d;
        return e;
    }
};

namespace {

// Per-instance work vectors of every level (zeroed: boundary entries stay zero).
// Owns a problem under construction: a failed create or clone releases
// everything allocated so far through glls_problem_destroy.
struct ProblemDeleter {
    void operator()(glls_problem* P) const { glls_problem_destroy(P); }
};
using ProblemPtr = std::unique_ptr<glls_problem, ProblemDeleter>;

template <typename T>
glls_status alloc_level_vectors(glls_problem* P, std::vector<LevelStore<T>>& Ls) {
    for (auto& s : Ls) {
        const long long n = s.dev.N * P->nrhs;
        CK(P->alloc(&s.r, n));
        CK(P->alloc(&s.x, n));
        CK(P->alloc(&s.y, n));
        CK(P->alloc(&s.t1, n));
        CK(P->alloc(&s.t2, n));
        CK(cudaMemset(s.r, 0, sizeof(T) * n));
        CK(cudaMemset(s.x, 0, sizeof(T) * n));
        CK(cudaMemset(s.y, 0, sizeof(T) * n));
    }
    return GLLS_OK;
}

// Per-instance Krylov state, scalars, streams.
// Per right-hand side: f, f0 and the Krylov vectors; g and the lifting v
// are shared.  Scalars, partial sums and tickets per right-hand side.
glls_status alloc_instance(glls_problem* P) {
    const long long N = P->N, k = P->nrhs;
    double** vecs[] = {&P->f, &P->f0, &P->xk, &P->rk, &P->pk, &P->qk, &P->zk, &P->yk};
    for (double** vp : vecs) {
        CK(P->alloc(vp, N * k));
        CK(cudaMemset(*vp, 0, sizeof(double) * N * k));
    }
    double** shared_vecs[] = {&P->g, &P->v};
    for (double** vp : shared_vecs) {
        CK(P->alloc(vp, N));
        CK(cudaMemset(*vp, 0, sizeof(double) * N));
    }
    CK(P->alloc(&P->S, S_COUNT * k));
    CK(P->alloc(&P->part, k * std::max<long long>(2 * kMaxReduceBlocks, 3 * kDotBlocks + P->L64.back().dev.E + 1)));
    CK(P->alloc(&P->ticket, k));
    CK(cudaMemset(P->ticket, 0, sizeof(unsigned) * k));
    CK(P->alloc(&P->r32, N * k));
    CK(P->alloc(&P->z32, N * k));
    CK(cudaMemset(P->r32, 0, sizeof(float) * N * k));
    CK(cudaMemset(P->z32, 0, sizeof(float) * N * k));
    CK(cudaMallocHost(&P->hostS, sizeof(double) * S_COUNT * k));
    CK(cudaStreamCreateWithFlags(&P->capture_stream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&P->capture_stream2, cudaStreamNonBlocking));
    return GLLS_OK;
}

// Largest input window (max(start) + width - min(start)) of `tile`
// consecutive rows starting at multiples of `tile`.
int band_span(const Band1D& b, int tile) {
    int best = 0;
    for (int r0 = 0; r0 < b.rows; r0 += tile) {
        int lo = b.start[r0], hi = b.start[r0] + b.width;
        for (int r = r0; r < std::min(b.rows, r0 + tile); ++r) {
            lo = std::min(lo, b.start[r]);
            hi = std::max(hi, b.start[r] + b.width);
        }
        best = std::max(best, hi - lo);
    }
    return best;
}

template <typename T>
glls_status upload_levels(glls_problem* P, const std::vector<LevelHost>& H, std::vector<LevelStore<T>>& out) {
    out.assign(H.size(), LevelStore<T>());
    for (size_t l = 0; l < H.size(); ++l) {
        const LevelHost& h = H[l];
        LevelStore<T>& s = out[l];
        DevLevel<T>& d = s.dev;
        d.dim = h.dim;
        d.p = h.p;
        d.n1 = h.p + 1;
        d.nloc = h.nloc;
        d.ncomp = h.ncomp;
        for (int a = 0; a < 3; ++a) { d.ne[a] = h.ne[a]; d.n[a] = h.n[a]; }
        d.N = h.N;
        d.E = h.E;
        CK(P->upload(&d.G, h.G));
        CK(P->upload(&d.D, h.D));
        CK(P->upload(&d.diag, h.diag));
        for (int a = 0; a < h.dim; ++a) CK(P->upload(&d.off[a], h.off[a]));
        for (int a = 0; a < h.dim; ++a) {
            using V2 = typename Vec2Of<T>::type;
            std::vector<V2> packed(h.N);
            for (long long i = 0; i < h.N; ++i) {
                packed[i].x = (T)h.diag[i];
                packed[i].y = (T)h.off[a][i];
            }
            V2* dptr = nullptr;
            void* p_ = nullptr;
            CK(dev_malloc(&p_, sizeof(V2) * packed.size()));
            P->shared->allocs.push_back(p_);
            P->shared->bytes += sizeof(V2) * packed.size();
            dptr = static_cast<V2*>(p_);
            CK(cudaMemcpy(dptr, packed.data(), sizeof(V2) * packed.size(), cudaMemcpyHostToDevice));
            d.band[a] = dptr;
        }
        if (h.lblock) {
            using V2 = typename Vec2Of<T>::type;
            for (int a = 0; a < h.dim; ++a) {
                CK(P->upload(&d.blk[a], h.blk[a]));
                const size_t nv = h.vband[a].size() / 2;
                std::vector<V2> packed(nv ? nv : 1);
                for (size_t i = 0; i < nv; ++i) {
                    packed[i].x = (T)h.vband[a][2 * i];
                    packed[i].y = (T)h.vband[a][2 * i + 1];
                }
                void* p_ = nullptr;
                CK(dev_malloc(&p_, sizeof(V2) * packed.size()));
                P->shared->allocs.push_back(p_);
                P->shared->bytes += sizeof(V2) * packed.size();
                CK(cudaMemcpy(p_, packed.data(), sizeof(V2) * packed.size(), cudaMemcpyHostToDevice));
                d.vband[a] = static_cast<const V2*>(p_);
            }
        }
        if (l > 0) {
            for (int a = 0; a < h.dim; ++a) {
                const Band1D* bs[2] = {&h.P[a], &h.R[a]};
                DevBand<T>* ds[2] = {&d.P[a], &d.R[a]};
                for (int k = 0; k < 2; ++k) {
                    ds[k]->rows = bs[k]->rows;
                    ds[k]->cols = bs[k]->cols;
                    ds[k]->width = bs[k]->width;
                    ds[k]->span32 = band_span(*bs[k], 32);
                    ds[k]->span8 = band_span(*bs[k], 8);
                    CK(P->upload(&ds[k]->start, bs[k]->start));
                    CK(P->upload(&ds[k]->coef, bs[k]->coef));
                }
            }
        }
    }
    return alloc_level_vectors<T>(P, out);
}

// Coarsest-level solver data in precision T: node index (FP64 copy only),
// block-CR operators padded to 16-byte rows, the dense inverse of the system
// left after block CR (16-byte rows for vector loads).
template <typename T>
glls_status upload_coarse(glls_problem* P, const CoarseHost& C, DevCoarse<T>& D) {
    constexpr int V = 16 / sizeof(T);
    D.n = C.n;
    D.nr = C.nr;
    D.ld = (C.nr + V - 1) / V * V;
    D.nb = C.nb;
    D.m = C.m;
    D.ldm = (C.m + V - 1) / V * V;
    D.cr_levels = C.cr_levels;
    if ((size_t)D.ld * sizeof(T) > kMaxDynSmemBytes)
        return fail(GLLS_ERR_INVALID, "coarsest level too large for the dense coarse solver "
                                      "(use GLLS_COARSE_BLOCK_CR with more levels)");
    if (sizeof(T) == sizeof(double)) CK(P->upload(&D.index, C.index));
    auto pad = [&](const std::vector<double>& src, long long rows, long long cols, long long ld) {
        std::vector<T> out((size_t)rows * ld, T(0));
        for (long long i = 0; i < rows; ++i)
            for (long long j = 0; j < cols; ++j) out[(size_t)i * ld + j] = (T)src[(size_t)i * cols + j];
        return out;
    };
    const size_t mm = (size_t)C.m * C.m;
    for (int l = 0; l < C.cr_levels; ++l) {
        const long long nfh = (long long)(C.fh[l].size() / mm), nagk = (long long)(C.agk[l].size() / mm);
        CK(P->upload(&D.fh[l], pad(C.fh[l], nfh * C.m, C.m, D.ldm)));
        CK(P->upload(&D.agk[l], pad(C.agk[l], nagk * C.m, C.m, D.ldm)));
    }
    CK(P->upload(&D.inv, pad(C.inv, C.nr, C.nr, D.ld)));
    return GLLS_OK;
}

template <typename T>
std::vector<LevelStore<T>>& levels_of(glls_problem* P);
template <>
std::vector<LevelStore<double>>& levels_of<double>(glls_problem* P) { return P->L64; }
template <>
std::vector<LevelStore<float>>& levels_of<float>(glls_problem* P) { return P->L32; }
template <typename T>
const DevCoarse<T>& coarse_of(glls_problem* P);
template <>
const DevCoarse<double>& coarse_of<double>(glls_problem* P) { return P->C64; }
template <>
const DevCoarse<float>& coarse_of<float>(glls_problem* P) { return P->C32; }

// rc = R_l (r - y) on level l-1
template <typename T>
void restrict_residual(glls_problem* P, int l, const T* r, const T* y, T* rc, cudaStream_t st, int nrhs = 1) {
    auto& Ls = levels_of<T>(P);
    const DevLevel<T>& F = Ls[l].dev;
    const DevLevel<T>& C = Ls[l - 1].dev;
    // axes 0 and 1 in one fused launch (then axis 2 in 3-D)
    const int mid[3] = {C.n[0], C.n[1], F.n[2]};
    const bool only2 = F.dim == 2;
    if (launch_transfer2<T>(F.R[0], F.R[1], F.n, mid, r, y, only2 ? rc : Ls[l].t1, false, only2, st, nullptr,
                            nrhs)) {
        if (!only2) launch_transfer<T>(F.R[2], 2, mid, C.n, Ls[l].t1, nullptr, rc, false, true, st, nullptr, nrhs);
        return;
    }
    int cur[3] = {F.n[0], F.n[1], F.n[2]};
    const T* in = r;
    const T* in2 = y;
    for (int a = 0; a < F.dim; ++a) {
        int nxt[3] = {cur[0], cur[1], cur[2]};
        nxt[a] = C.n[a];
        const bool last = a == F.dim - 1;
        T* out = last ? rc : (a % 2 == 0 ? Ls[l].t1 : Ls[l].t2);
        launch_transfer<T>(F.R[a], a, cur, nxt, in, in2, out, false, last, st, nullptr, nrhs);
        in = out;
        in2 = nullptr;
        for (int k = 0; k < 3; ++k) cur[k] = nxt[k];
    }
}

// x += P_l e; clear (optional, level-l sized) is reset to 0 by the last pass
template <typename T>
void prolong_add(glls_problem* P, int l, const T* e, T* x, cudaStream_t st, T* clear = nullptr, int nrhs = 1) {
    auto& Ls = levels_of<T>(P);
    const DevLevel<T>& F = Ls[l].dev;
    const DevLevel<T>& C = Ls[l - 1].dev;
    const int mid[3] = {F.n[0], F.n[1], C.n[2]};
    const bool only2 = F.dim == 2;
    if (launch_transfer2<T>(F.P[0], F.P[1], C.n, mid, e, nullptr, only2 ? x : Ls[l].t1, only2, false, st,
                            only2 ? clear : nullptr, nrhs)) {
        if (!only2) launch_transfer<T>(F.P[2], 2, mid, F.n, Ls[l].t1, nullptr, x, true, false, st, clear, nrhs);
        return;
    }
    int cur[3] = {C.n[0], C.n[1], C.n[2]};
    const T* in = e;
    for (int a = 0; a < F.dim; ++a) {
        int nxt[3] = {cur[0], cur[1], cur[2]};
        nxt[a] = F.n[a];
        const bool last = a == F.dim - 1;
        T* out = last ? x : (a % 2 == 0 ? Ls[l].t1 : Ls[l].t2);
        launch_transfer<T>(F.P[a], a, cur, nxt, in, nullptr, out, last, false, st, last ? clear : nullptr, nrhs);
        in = out;
        for (int k = 0; k < 3; ++k) cur[k] = nxt[k];
    }
}

// x <- x + alpha B_s^-1 (r - A x).  x_is_zero: x = alpha B_s^-1 r without
// the apply.  The level scratch y is zero on entry and on exit: the apply
// accumulates into it and the line solve resets what it reads.
template <typename T>
void smooth(glls_problem* P, int l, int s, T alpha, const T* r, T* x, bool x_is_zero, cudaStream_t st,
            int nrhs = 1) {
    auto& Ls = levels_of<T>(P);
    if (x_is_zero) {
        launch_line_solve<T>(Ls[l].dev, s, 3, nullptr, r, nullptr, x, alpha, st, nrhs);
    } else {
        launch_apply<T>(Ls[l].dev, x, Ls[l].y, true, st, true, nullptr, nullptr, nullptr, nrhs);
        launch_line_solve<T>(Ls[l].dev, s, 1, nullptr, r, Ls[l].y, x, alpha, st, nrhs);
    }
}

// Algorithm 2: x = M_l^-1 r from x0 = 0
template <typename T>
void cycle(glls_problem* P, int l, const T* r, T* x, int gamma, int m, T alpha, cudaStream_t st, int nrhs = 1) {
    auto& Ls = levels_of<T>(P);
    // x: boundary entries are zero and stay zero (only interior entries are written)
    if (l == 0) {
        launch_coarse<T>(coarse_of<T>(P), Ls[0].dev.N, r, x, Ls[0].t1, st, true, nrhs);
        return;
    }
    const int d = Ls[l].dev.dim;
    bool zero = true;
    for (int s = 0; s < d; ++s)
        for (int k = 0; k < m; ++k) {
            smooth<T>(P, l, s, alpha, r, x, zero, st, nrhs);
            zero = false;
        }
    for (int g = 0; g < gamma; ++g) {
        launch_apply<T>(Ls[l].dev, x, Ls[l].y, true, st, true, nullptr, nullptr, nullptr, nrhs);
        restrict_residual<T>(P, l, r, Ls[l].y, Ls[l - 1].r, st, nrhs);
        cycle<T>(P, l - 1, Ls[l - 1].r, Ls[l - 1].x, gamma, m, alpha, st, nrhs);
        prolong_add<T>(P, l, Ls[l - 1].x, x, st, Ls[l].y, nrhs);
        for (int s = d - 1; s >= 0; --s)
            for (int k = 0; k < m; ++k) smooth<T>(P, l, s, alpha, r, x, false, st, nrhs);
    }
}

glls_status check_level(glls_problem* P, int level, bool need_coarser) {
    if (!P) return fail(GLLS_ERR_INVALID, "null problem");
    if (level < 0 || level >= (int)P->L64.size()) return fail(GLLS_ERR_INVALID, "level out of range");
    if (need_coarser && level < 1) return fail(GLLS_ERR_INVALID, "level must be >= 1");
    return GLLS_OK;
}

glls_status check_opts(const glls_solve_opts* o) {
    if (!o) return fail(GLLS_ERR_INVALID, "null options");
    if (o->gamma < 1 || o->gamma > 16) return fail(GLLS_ERR_INVALID, "gamma must be in 1..16");
    if (o->m < 1 || o->m > 16) return fail(GLLS_ERR_INVALID, "m must be in 1..16");
    if (!(o->alpha > 0.0)) return fail(GLLS_ERR_INVALID, "alpha must be > 0");
    if (o->precision != GLLS_PREC_FP64 && o->precision != GLLS_PREC_MIXED)
        return fail(GLLS_ERR_INVALID, "bad precision");
    if (o->krylov != GLLS_KRYLOV_FCG && o->krylov != GLLS_KRYLOV_PCG && o->krylov != GLLS_KRYLOV_GMRES)
        return fail(GLLS_ERR_INVALID, "bad krylov");
    if (o->max_iter < 1) return fail(GLLS_ERR_INVALID, "max_iter must be >= 1");
    if (!(o->tol > 0.0)) return fail(GLLS_ERR_INVALID, "tol must be > 0");
    return GLLS_OK;
}

// Dot partials written by launch_apply for L (coloured summation runs the
// node-per-thread kernel and a separate dot over kDotBlocks CTAs).
static int dot_partials_of(const DevLevel<double>& L) {
    return L.colored ? kDotBlocks : apply_dot_partials<double>(L);
}

// Body of one outer iteration (4 launches besides the gamma-cycle):
//   z = M r                      (FP32 cycle on r32 = float(r) in mixed precision)
//   partials of r.z and z.q      (z = double(z32); q reset to 0 after reading)
//   p = z + beta p               (every block sums the r.z, z.q partials)
//   q = A p, partials of p.q     (accumulated per element in the apply)
//   alpha = r.z / p.q; x += alpha p; r -= alpha q; r32 = float(r);
//   S_RR = r.r, S_RZ = r.z, S_ALPHA, S_PQ published by the last block
// Producers write per-block partials and consumers sum them (the same fixed
// order in every block): only the update ends with a grid-wide ticket.
void outer_iteration(glls_problem* P, const glls_solve_opts* o, cudaStream_t st) {
    const int L = (int)P->L64.size() - 1;
    const long long N = P->N;
    const int k = P->nrhs;
    const bool mixed = o->precision == GLLS_PREC_MIXED;
    if (mixed) cycle<float>(P, L, P->r32, P->z32, o->gamma, o->m, (float)o->alpha, st, k);
    else cycle<double>(P, L, P->rk, P->zk, o->gamma, o->m, o->alpha, st, k);
    // partial sums per right-hand side: r.z and z.q (kDotBlocks each), r.r
    // (kDotBlocks), p.q (one per apply CTA)
    double* prz = P->part;
    double* pzq = prz + (long long)k * kDotBlocks;
    double* prr = pzq + (long long)k * kDotBlocks;
    double* ppq = prr + (long long)k * kDotBlocks;
    // mixed precision: q = A p in float-float arithmetic where the level allows
    // it (apply_ff.cu), else in FP64
    const bool ff = mixed && o->tol >= kFfMinTol && apply_ff_supported(P->L64[L].dev);
    const int npq = ff ? apply_ff_partials(P->L64[L].dev) : dot_partials_of(P->L64[L].dev);
    launch_dots_rz_zq(P->rk, P->zk, mixed ? P->z32 : nullptr, P->qk, N, prz, pzq, st, k);
    const int nb = fcg_blocks(N);            // the dots' CTAs: partials of r.z, z.q, r.r per right-hand side
    launch_fcg_direction(P->pk, P->zk, N, prz, pzq, nb, P->S, o->krylov == GLLS_KRYLOV_FCG ? 1 : 0, st, k);
    if (ff) launch_apply_ff(P->L64[L].dev, P->pk, P->qk, true, ppq, st, k);
    else launch_apply<double>(P->L64[L].dev, P->pk, P->qk, true, st, true, P->S + S_PQ, ppq, nullptr, k);
    launch_fcg_update(P->xk, P->rk, P->pk, P->qk, N, ppq, npq, prz, nb, prr, P->S, P->ticket,
                      mixed ? P->r32 : nullptr, st, k);
}

// Lifting and Krylov initialisation (x = p = q = 0, r = f0, S_RR0 = r.r).
// The lifting v of the (shared) Dirichlet data and A v are computed once;
// f0 = M f - A v for every right-hand side.
void solve_prologue(glls_problem* P, const glls_solve_opts* o, cudaStream_t st) {
    const long long N = P->N, NK = P->N * P->nrhs;
    const int L = (int)P->L64.size() - 1;
    const DevLevel<double>& F = P->L64[L].dev;
    launch_boundary_only(P->g, P->v, F.n, F.dim, st);
    launch_apply<double>(F, P->v, P->yk, false, st);
    launch_lift_rhs(P->mass, P->f, P->yk, P->f0, F.n, F.dim, st, P->nrhs);
    cudaMemsetAsync(P->xk, 0, sizeof(double) * NK, st);
    cudaMemsetAsync(P->pk, 0, sizeof(double) * NK, st);
    cudaMemsetAsync(P->qk, 0, sizeof(double) * NK, st);
    cudaMemcpyAsync(P->rk, P->f0, sizeof(double) * NK, cudaMemcpyDeviceToDevice, st);
    launch_dots(P->rk, P->rk, nullptr, nullptr, 1, N, P->part, P->S, S_RR0, S_RR0, P->ticket, st, P->nrhs);
    if (o->precision == GLLS_PREC_MIXED) launch_cast<double, float>(P->rk, P->r32, NK, st);
}

bool same_solve_key(const glls_solve_opts& a, const glls_solve_opts& b) {
    return a.tol == b.tol && a.max_iter == b.max_iter && a.gamma == b.gamma && a.m == b.m && a.alpha == b.alpha &&
           a.precision == b.precision && a.krylov == b.krylov;
}

long long count_kernel_nodes(cudaGraph_t g) {
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return 0;
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
    long long k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

// Adds the whole solve of P to the graph being captured on cs: prologue, a
// conditional WHILE node whose body (captured on cs2) is one outer iteration
// followed by the loop-control kernel, then y = x + v.  Returns the first
// CUDA error; the caller ends the capture.
cudaError_t capture_solve(glls_problem* P, const glls_solve_opts* o, cudaStream_t cs, cudaStream_t cs2) {
    cudaStreamCaptureStatus stt;
    cudaGraph_t capg = nullptr;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &stt, nullptr, &capg, nullptr, nullptr, nullptr);
    cudaGraphConditionalHandle handle = 0;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&handle, capg, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
    solve_prologue(P, o, cs);
    launch_solve_init(P->S, handle, o->tol, o->max_iter, cs, P->nrhs);
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    e = cudaStreamGetCaptureInfo(cs, &stt, nullptr, &capg, &deps, nullptr, &ndeps);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, capg, deps, nullptr, ndeps, &cp);
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(cs2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            outer_iteration(P, o, cs2);
            launch_solve_cond(P->S, handle, o->max_iter, cs2, P->nrhs);
            e = cudaStreamEndCapture(cs2, &body);
            if (e == cudaSuccess) P->kern_iter = count_kernel_nodes(body);
        }
    }
    if (e == cudaSuccess) {   // u = w + v for every right-hand side
        cudaMemcpyAsync(P->yk, P->xk, sizeof(double) * P->N * P->nrhs, cudaMemcpyDeviceToDevice, cs);
        launch_axpy(P->yk, P->v, 1.0, P->N, cs, P->nrhs, true);
    }
    return e;
}

// The whole solve as one cached graph (device-side loop).
glls_status get_solve_graph(glls_problem* P, const glls_solve_opts* o) {
    if (P->solve_exec && same_solve_key(P->solve_key, *o)) return GLLS_OK;
    std::lock_guard<std::recursive_mutex> dev_lock(g_device_mutex);
    if (P->solve_exec) {
        cudaGraphExecDestroy(P->solve_exec);
        P->solve_exec = nullptr;
    }
    cudaStream_t cs = P->capture_stream, cs2 = P->capture_stream2;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = capture_solve(P, o, cs, cs2);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) P->kern_fixed = count_kernel_nodes(graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&P->solve_exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    CK(e);
    P->solve_key = *o;
    return GLLS_OK;
}

// Fills stats / status of a finished device-loop solve from the host copy of S.
// Fills stats[j] for every right-hand side j (stats: nrhs entries) and
// returns the worst status (breakdown, then not converged, then OK).
glls_status solve_result(glls_problem* P, const double* h, glls_stats* stats, double t_ms) {
    glls_status worst = GLLS_OK;
    for (int j = 0; j < P->nrhs; ++j) {
        const double* hj = h + (long long)j * S_COUNT;
        glls_status result = GLLS_OK;
        double rel = 0.0;
        if (hj[S_FLAG] != 0.0) {
            result = GLLS_ERR_BREAKDOWN;
        } else if (hj[S_RR0] > 0.0) {
            rel = std::sqrt(hj[S_RR] / hj[S_RR0]);
            result = hj[S_RR] <= hj[S_TOL2] ? GLLS_OK : GLLS_ERR_NOT_CONVERGED;
        }
        if (result == GLLS_ERR_BREAKDOWN || (result == GLLS_ERR_NOT_CONVERGED && worst == GLLS_OK)) worst = result;
        if (stats) {
            glls_stats& sj = stats[j];
            sj.iterations = (int)(hj[S_DONE] != 0.0 ? hj[S_ITS] : hj[S_ITER]);
            sj.rel_residual = rel;
            sj.setup_ms = P->setup_ms;
            sj.solve_ms = t_ms;
            sj.status = result;
            sj.kernels = P->kern_fixed + P->kern_iter * (long long)h[S_ITER];
        }
    }
    return worst;
}

// Batched solves: one graph whose parallel branches are the whole solves of
// several problems (each with its own device-side loop), cached per
// (problem list, options).
struct BatchEntry {
    std::vector<glls_problem*> probs;
    glls_solve_opts key;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t master = nullptr;
};
std::mutex g_batch_mutex;
std::vector<BatchEntry> g_batches;   // small LRU, newest last

struct WlPlan;
void destroy_plan(WlPlan* W);
bool plan_uses(const WlPlan* W, const glls_problem* P);
extern std::vector<WlPlan*> g_wplans;

void forget_batches_of(glls_problem* P) {
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    for (size_t i = 0; i < g_wplans.size();) {
        if (plan_uses(g_wplans[i], P)) {
            destroy_plan(g_wplans[i]);
            g_wplans.erase(g_wplans.begin() + i);
        } else {
            ++i;
        }
    }
    for (size_t i = 0; i < g_batches.size();) {
        bool hit = false;
        for (auto* q : g_batches[i].probs) hit = hit || q == P;
        if (hit) {
            cudaGraphExecDestroy(g_batches[i].exec);
            cudaStreamDestroy(g_batches[i].master);
            g_batches.erase(g_batches.begin() + i);
        } else {
            ++i;
        }
    }
}

glls_status get_iteration_graph(glls_problem* P, const glls_solve_opts* o) {
    if (P->iter_exec && P->g_gamma == o->gamma && P->g_m == o->m && P->g_prec == o->precision &&
        P->g_krylov == o->krylov && P->g_alpha == o->alpha)
        return GLLS_OK;
    std::lock_guard<std::recursive_mutex> dev_lock(g_device_mutex);
    if (P->iter_exec) {
        cudaGraphExecDestroy(P->iter_exec);
        P->iter_exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(P->capture_stream, cudaStreamCaptureModeThreadLocal));
    outer_iteration(P, o, P->capture_stream);
    CK(cudaStreamEndCapture(P->capture_stream, &graph));
    cudaError_t e = cudaGraphInstantiate(&P->iter_exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    P->g_gamma = o->gamma;
    P->g_m = o->m;
    P->g_prec = o->precision;
    P->g_krylov = o->krylov;
    P->g_alpha = o->alpha;
    return GLLS_OK;
}

}  // namespace

namespace {
template <typename T>
glls_status tune_levels(glls_problem* P, std::vector<LevelStore<T>>& Ls, int prec, int* chosen, float* best_us) {
    cudaStream_t st = P->capture_stream;
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    // band-1 lines per CTA: 16 only in FP32 (launch_line_warp falls back to 8
    // otherwise); line blocks: the launch heuristic (0) or 1..16 lines, at
    // most 256 segment tasks per CTA
    const int cand[4] = {2, 4, 8, 16};
    const int ncand = sizeof(T) == 4 ? 4 : 3;
    const int bcand[6] = {0, 1, 2, 4, 8, 16};
    for (size_t l = 1; l < Ls.size(); ++l)
        for (int s = 0; s < Ls[l].dev.dim; ++s) {
            float best = 1e30f;
            const bool blocks = Ls[l].dev.blk[s] != nullptr;
            int pick = blocks ? 0 : 4;
            for (int ci = 0; ci < (blocks ? 6 : ncand); ++ci) {
                const int c = blocks ? bcand[ci] : cand[ci];
                if (blocks && c * Ls[l].dev.ne[s] > 256) continue;
                if (blocks) Ls[l].dev.lbc[s] = c;
                else Ls[l].dev.lpb[s] = c;
                for (int w = 0; w < 3; ++w)
                    launch_line_solve<T>(Ls[l].dev, s, 0, Ls[l].r, nullptr, nullptr, Ls[l].t2, T(1), st);
                CK(cudaEventRecord(a, st));
                for (int w = 0; w < 10; ++w)
                    launch_line_solve<T>(Ls[l].dev, s, 0, Ls[l].r, nullptr, nullptr, Ls[l].t2, T(1), st);
                CK(cudaEventRecord(b, st));
                CK(cudaEventSynchronize(b));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, a, b));
                if (ms < best) { best = ms; pick = c; }
            }
            if (blocks) Ls[l].dev.lbc[s] = pick;
            else Ls[l].dev.lpb[s] = pick;
            const size_t k = (l * 2 + prec) * 3 + s;
            if (chosen) chosen[k] = pick;
            if (best_us) best_us[k] = best * 100.f;   // 10 launches: ms * 1000 / 10
        }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    CK(cudaGetLastError());
    return GLLS_OK;
}
}  // namespace

// Right-preconditioned flexible GMRES without restart (the paper's outer
// solver, Sec. 3): Arnoldi with classical Gram-Schmidt applied twice, the
// preconditioned directions z_j kept (the FP32 cycle is not exactly linear),
// Givens rotations on the host, x = sum_j y_j z_j.  Host-driven loop.
glls_status gmres_solve(glls_problem* P, const glls_solve_opts* o, cudaStream_t st, int* it_out, double* rel_out) {
    const long long N = P->N;
    const int L = (int)P->L64.size() - 1;
    const DevLevel<double>& F = P->L64[L].dev;
    const int m = std::min(o->max_iter, 400);
    if (P->gm < m) {
        for (double* q : {P->gV, P->gZ, P->gh, P->gpart})
            if (q) {
                cudaFree(q);
                P->allocs.erase(std::remove(P->allocs.begin(), P->allocs.end(), (void*)q), P->allocs.end());
            }
        CK(P->alloc(&P->gV, (size_t)(m + 1) * N));
        CK(P->alloc(&P->gZ, (size_t)m * N));
        CK(P->alloc(&P->gh, 2 * (size_t)(m + 1)));
        CK(P->alloc(&P->gpart, 64 * (size_t)(m + 1)));
        CK(cudaMemset(P->gZ, 0, sizeof(double) * (size_t)m * N));   // boundary entries stay zero
        P->gm = m;
    }
    const bool mixed = o->precision == GLLS_PREC_MIXED;
    solve_prologue(P, o, st);
    std::vector<double> hS(S_COUNT);
    CK(cudaMemcpyAsync(hS.data(), P->S, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const double rr0 = hS[S_RR0];
    *it_out = 0;
    *rel_out = 0.0;
    if (!std::isfinite(rr0)) return fail(GLLS_ERR_BREAKDOWN, "non-finite right-hand side");
    if (rr0 == 0.0) return GLLS_OK;
    const double beta = std::sqrt(rr0);
    launch_scale_by_norm(P->gV, P->rk, P->S + S_RR0, N, st);
    std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m, 0.0), sn(m, 0.0), g(m + 1, 0.0), hv(2 * (m + 1));
    auto Hat = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
    g[0] = beta;
    int kdone = m;
    double rel = 1.0;
    glls_status result = GLLS_ERR_NOT_CONVERGED;
    for (int k = 0; k < m; ++k) {
        double* vk = P->gV + (size_t)k * N;
        double* zk = P->gZ + (size_t)k * N;
        double* w = P->gV + (size_t)(k + 1) * N;
        if (mixed) {
            launch_cast<double, float>(vk, P->r32, N, st);
            cycle<float>(P, L, P->r32, P->z32, o->gamma, o->m, (float)o->alpha, st);
            launch_cast<float, double>(P->z32, zk, N, st);
        } else {
            cycle<double>(P, L, vk, zk, o->gamma, o->m, o->alpha, st);
        }
        launch_apply<double>(F, zk, w, true, st);
        for (int pass = 0; pass < 2; ++pass) {
            launch_multidot(P->gV, N, k + 1, w, N, P->gpart, P->gh + pass * (m + 1), P->ticket, st);
            launch_gs_update(w, P->gV, N, k + 1, P->gh + pass * (m + 1), N, -1.0, st);
        }
        launch_dots(w, w, nullptr, nullptr, 1, N, P->part, P->S, S_RR, S_RR, P->ticket, st);
        CK(cudaMemcpyAsync(hv.data(), P->gh, sizeof(double) * 2 * (m + 1), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(hS.data(), P->S, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int i = 0; i <= k; ++i) Hat(i, k) = hv[i] + hv[(m + 1) + i];
        const double hk1 = std::sqrt(hS[S_RR]);
        if (!std::isfinite(hk1)) return fail(GLLS_ERR_BREAKDOWN, "non-finite Arnoldi vector");
        Hat(k + 1, k) = hk1;
        if (hk1 > 0.0) launch_scale_by_norm(w, w, P->S + S_RR, N, st);
        for (int i = 0; i < k; ++i) {   // previous rotations
            const double t = cs[i] * Hat(i, k) + sn[i] * Hat(i + 1, k);
            Hat(i + 1, k) = -sn[i] * Hat(i, k) + cs[i] * Hat(i + 1, k);
            Hat(i, k) = t;
        }
        const double rr = std::hypot(Hat(k, k), Hat(k + 1, k));
        cs[k] = Hat(k, k) / rr;
        sn[k] = Hat(k + 1, k) / rr;
        Hat(k, k) = rr;
        Hat(k + 1, k) = 0.0;
        g[k + 1] = -sn[k] * g[k];
        g[k] = cs[k] * g[k];
        rel = std::fabs(g[k + 1]) / beta;
        if (rel <= o->tol || hk1 == 0.0) {
            kdone = k + 1;
            result = GLLS_OK;
            break;
        }
    }
    // y = H^-1 g (upper triangular), x = sum_j y_j z_j
    std::vector<double> y(kdone, 0.0);
    for (int i = kdone - 1; i >= 0; --i) {
        double t = g[i];
        for (int j = i + 1; j < kdone; ++j) t -= Hat(i, j) * y[j];
        y[i] = t / Hat(i, i);
    }
    CK(cudaMemcpyAsync(P->gh, y.data(), sizeof(double) * kdone, cudaMemcpyHostToDevice, st));
    launch_gs_update(P->xk, P->gZ, N, kdone, P->gh, N, +1.0, st);
    CK(cudaStreamSynchronize(st));
    *it_out = kdone;
    *rel_out = rel;
    if (result == GLLS_ERR_NOT_CONVERGED) fail(result, "max_iter reached");
    return result;
}

// ===========================================================================
// C ABI
// ===========================================================================
// ---------------------------------------------------------------------------
// Work-list batched solve.  The problems are grouped by their order chain;
// inside a group every step of the solve loop (each apply, line solve,
// transfer, coarsest-solve step and outer-Krylov kernel of Algorithm 2 and
// the flexible CG iteration) is ONE launch over the work list of all the
// group's problems: item j of a launch carries problem j's level data and
// vectors and owns a contiguous range of the launch's CTAs.  Each group is
// one branch of one graph, with its own device-side loop that runs while any
// of its problems is active (stopped problems are frozen as stopped
// right-hand sides are).
// ---------------------------------------------------------------------------
namespace {

enum WlKind { WL_APPLY = 0, WL_LINE, WL_T2, WL_BCR_F, WL_COARSE, WL_BCR_B, WL_FCG };

struct WlRecord {
    int kind = 0;
    bool dbl = false;                  // FP64 items
    int p = 0, cv = 1, wb = 0, ty = 0, l = 0, step = 0;
    bool mask = false, dot = false, add = false;
    bool ff = false;                   // the float-float form of the FP64 outer apply
    int blocks = 0, threads = 256, nitems = 0;
    size_t smem = 0;
    std::vector<unsigned char> items;  // host copy of the item array
    std::vector<int> start{0};         // CTA offsets, nitems + 1
    std::vector<int> owner;            // the group position of each item's problem
    size_t item_bytes = 0, done_at = 0;   // item size and offset of its stop-flag pointer
    size_t off_items = 0, off_start = 0;

    template <class Item>
    void put(const Item& it, int nblocks, int who) {
        const unsigned char* b = reinterpret_cast<const unsigned char*>(&it);
        items.insert(items.end(), b, b + sizeof(Item));
        start.push_back(start.back() + nblocks);
        owner.push_back(who);
        item_bytes = sizeof(Item);
        done_at = offsetof(Item, done);
        ++nitems;
        blocks = start.back();
    }
};

struct WlGroup {
    std::vector<glls_problem*> probs;
    std::vector<int> index;            // position of each problem in the batch
    std::vector<WlRecord> body;        // one outer iteration
    size_t off_S = 0;                  // [n][S_COUNT] scalars in the plan's block
    cudaStream_t s1 = nullptr, s2 = nullptr;
    long long kernels_iter = 0;        // kernel nodes of one pass of the group's loop
};

struct WlPlan {
    std::vector<glls_problem*> probs;
    glls_solve_opts key{};
    std::vector<WlGroup> groups;
    void* dev = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t master = nullptr;
    long long kernels_fixed = 0;
};

std::vector<WlPlan*> g_wplans;   // guarded by g_batch_mutex (newest last)

bool plan_uses(const WlPlan* W, const glls_problem* P) {
    for (const glls_problem* q : W->probs)
        if (q == P) return true;
    return false;
}

void destroy_plan(WlPlan* W) {
    if (W->exec) cudaGraphExecDestroy(W->exec);
    for (auto& g : W->groups) {
        if (g.s1) cudaStreamDestroy(g.s1);
        if (g.s2) cudaStreamDestroy(g.s2);
    }
    if (W->master) cudaStreamDestroy(W->master);
    if (W->dev) cudaFree(W->dev);
    delete W;
}

// Builds the records of one outer iteration of a group in precision T (the
// gamma-cycle) around the FP64 outer kernels; returns "" or why the group
// cannot run as a work list.
template <typename T>
struct WlBuilder {
    WlGroup& G;
    const glls_solve_opts& o;
    bool mixed;

    T* rv(glls_problem* P, int l) {
        auto& Ls = levels_of<T>(P);
        if (l == (int)Ls.size() - 1) return mixed ? (T*)(void*)P->r32 : (T*)(void*)P->rk;
        return Ls[l].r;
    }
    T* xv(glls_problem* P, int l) {
        auto& Ls = levels_of<T>(P);
        if (l == (int)Ls.size() - 1) return mixed ? (T*)(void*)P->z32 : (T*)(void*)P->zk;
        return Ls[l].x;
    }

    std::string apply(int l) {
        WlRecord r;
        r.kind = WL_APPLY;
        r.dbl = sizeof(T) == 8;
        r.mask = true;
        for (size_t j = 0; j < G.probs.size(); ++j) {
            glls_problem* P = G.probs[j];
            const DevLevel<T>& L = levels_of<T>(P)[l].dev;
            r.p = L.p;
            ApplyItem<T> it{L, xv(P, l), levels_of<T>(P)[l].y, nullptr, nullptr};
            r.put(it, apply_list_blocks(L.p, L.E), (int)j);
        }
        G.body.push_back(std::move(r));
        return "";
    }

    std::string line(int l, int s, int mode) {
        WlRecord r;
        r.kind = WL_LINE;
        r.dbl = sizeof(T) == 8;
        r.threads = 32;
        std::vector<size_t> sm0, sm1;
        std::vector<unsigned char> buf(line_block_item_bytes<T>());
        r.item_bytes = buf.size();
        r.done_at = line_block_item_done_offset<T>();
        for (size_t j = 0; j < G.probs.size(); ++j) {
            glls_problem* P = G.probs[j];
            auto& Ls = levels_of<T>(P);
            int blocks = 0, threads = 0, cv = 1;
            size_t smem[2] = {0, 0};
            const int k = line_block_list_item<T>(Ls[l].dev, s, mode, nullptr, rv(P, l), mode == 1 ? Ls[l].y : nullptr,
                                                  xv(P, l), (T)o.alpha, buf.data(), &blocks, &threads, smem, &cv);
            if (k < 0) return "a level's grid lines are outside the line-block kernel's range";
            if (k == 0) continue;
            r.p = Ls[l].dev.p;
            r.items.insert(r.items.end(), buf.begin(), buf.end());
            r.start.push_back(r.start.back() + blocks);
            r.owner.push_back((int)j);
            ++r.nitems;
            r.blocks = r.start.back();
            r.threads = std::max(r.threads, threads);
            r.cv = std::max(r.cv, cv);
            sm0.push_back(smem[0]);
            sm1.push_back(smem[1]);
        }
        const bool spec = line_block_list_specialised(r.p, r.cv);
        for (size_t i = 0; i < sm0.size(); ++i) r.smem = std::max(r.smem, spec ? sm0[i] : sm1[i]);
        if (r.nitems) G.body.push_back(std::move(r));
        return "";
    }

    std::string smooth(int l, int s, bool zero) {
        if (zero) return line(l, s, 3);
        std::string e = apply(l);
        return e.empty() ? line(l, s, 1) : e;
    }

    // restriction (prolong = false: rc = R (r - y)) or x += P e, clearing y
    std::string transfer(int l, bool prolong) {
        WlRecord r;
        r.kind = WL_T2;
        r.dbl = sizeof(T) == 8;
        r.add = prolong;
        r.mask = !prolong;
        for (size_t j = 0; j < G.probs.size(); ++j) {
            glls_problem* P = G.probs[j];
            auto& Ls = levels_of<T>(P);
            const DevLevel<T>& F = Ls[l].dev;
            const DevLevel<T>& C = Ls[l - 1].dev;
            Transfer2Item<T> it{};
            int nout[3];
            if (!prolong) {
                it.M0 = F.R[0];
                it.M1 = F.R[1];
                it.nin = make_int3(F.n[0], F.n[1], F.n[2]);
                nout[0] = C.n[0]; nout[1] = C.n[1]; nout[2] = F.n[2];
                it.in = rv(P, l);
                it.in2 = Ls[l].y;
                it.out = rv(P, l - 1);
                it.clear = nullptr;
            } else {
                it.M0 = F.P[0];
                it.M1 = F.P[1];
                it.nin = make_int3(C.n[0], C.n[1], C.n[2]);
                nout[0] = F.n[0]; nout[1] = F.n[1]; nout[2] = C.n[2];
                it.in = xv(P, l - 1);
                it.in2 = nullptr;
                it.out = xv(P, l);
                it.clear = Ls[l].y;
            }
            it.nout = make_int3(nout[0], nout[1], nout[2]);
            int gx = 0, gy = 0, wb = 0, ty = 0;
            size_t smem = 0;
            if (!transfer2_list_config<T>(it.M0, it.M1, nout, &gx, &gy, &wb, &ty, &smem))
                return "a transfer is outside the fused transfer kernel's range";
            it.gx = gx;
            it.gy = gy;
            r.wb = std::max(r.wb, wb);
            r.ty = ty;
            r.smem = std::max(r.smem, smem);
            r.put(it, gx * gy * nout[2], (int)j);
        }
        G.body.push_back(std::move(r));
        return "";
    }

    std::string coarse() {
        int kmax = 0;
        for (glls_problem* P : G.probs) kmax = std::max(kmax, coarse_of<T>(P).cr_levels);
        for (int l = 0; l < kmax; ++l) {
            WlRecord r;
            r.kind = WL_BCR_F;
            r.dbl = sizeof(T) == 8;
            r.l = l;
            for (size_t j = 0; j < G.probs.size(); ++j) {
                glls_problem* P = G.probs[j];
                const DevCoarse<T>& C = coarse_of<T>(P);
                if (C.cr_levels <= l) continue;
                const int a = C.nb >> l, nk = a / 2, ne = (a + 1) / 2;
                const int rows = (C.m + 7) / 8;
                BcrItem<T> it{C.fh[l], C.nb, C.m, C.ldm, C.index, rv(P, 0), levels_of<T>(P)[0].t1,
                              l == 0 ? nk + ne : nk, rows};
                r.smem = std::max(r.smem, 2 * sizeof(T) * (size_t)C.m);
                r.put(it, it.gx * rows, (int)j);
            }
            if (r.nitems) G.body.push_back(std::move(r));
        }
        {
            WlRecord r;
            r.kind = WL_COARSE;
            r.dbl = sizeof(T) == 8;
            for (size_t j = 0; j < G.probs.size(); ++j) {
                glls_problem* P = G.probs[j];
                const DevCoarse<T>& C = coarse_of<T>(P);
                const int k = C.cr_levels;
                CoarseItem<T> it{C.nr, C.ld, C.index, C.inv, k > 0 ? (const T*)levels_of<T>(P)[0].t1 : rv(P, 0),
                                 k > 0 ? nullptr : C.index, C.m, 1 << k, xv(P, 0)};
                long long blocks = (C.nr + 7) / 8;
                if (blocks > 2 * 152) blocks = 2 * 152;
                r.smem = std::max(r.smem, sizeof(T) * (size_t)C.ld);
                r.put(it, (int)blocks, (int)j);
            }
            if (r.smem > 200 * 1024) return "a coarsest dense system is too large for the work-list coarse kernel";
            G.body.push_back(std::move(r));
        }
        for (int l = kmax - 1; l >= 0; --l) {
            WlRecord r;
            r.kind = WL_BCR_B;
            r.dbl = sizeof(T) == 8;
            r.l = l;
            for (size_t j = 0; j < G.probs.size(); ++j) {
                glls_problem* P = G.probs[j];
                const DevCoarse<T>& C = coarse_of<T>(P);
                if (C.cr_levels <= l) continue;
                const int rows = (C.m + 7) / 8;
                BcrItem<T> it{C.agk[l], C.nb, C.m, C.ldm, C.index, levels_of<T>(P)[0].t1, xv(P, 0),
                              ((C.nb >> l) + 1) / 2, rows};
                r.smem = std::max(r.smem, 3 * sizeof(T) * (size_t)C.m);
                r.put(it, it.gx * rows, (int)j);
            }
            if (r.nitems) G.body.push_back(std::move(r));
        }
        return "";
    }

    // Algorithm 2 on level l (as cycle<T>)
    std::string cycle(int l) {
        if (l == 0) return coarse();
        const int d = 2;
        bool zero = true;
        std::string e;
        for (int s = 0; s < d && e.empty(); ++s)
            for (int k = 0; k < o.m && e.empty(); ++k) {
                e = smooth(l, s, zero);
                zero = false;
            }
        for (int g = 0; g < o.gamma && e.empty(); ++g) {
            e = apply(l);
            if (e.empty()) e = transfer(l, false);
            if (e.empty()) e = cycle(l - 1);
            if (e.empty()) e = transfer(l, true);
            for (int s = d - 1; s >= 0 && e.empty(); --s)
                for (int k = 0; k < o.m && e.empty(); ++k) e = smooth(l, s, false);
        }
        return e;
    }
};

// The outer iteration of a group (as outer_iteration): the gamma-cycle, the
// dots, the direction, the FP64 apply with its p.q partials, the update.
std::string build_group(WlGroup& G, const glls_solve_opts& o) {
    const bool mixed = o.precision == GLLS_PREC_MIXED;
    const int L = (int)G.probs[0]->L64.size() - 1;
    std::string e;
    if (mixed) {
        WlBuilder<float> b{G, o, true};
        e = b.cycle(L);
    } else {
        WlBuilder<double> b{G, o, false};
        e = b.cycle(L);
    }
    if (!e.empty()) return e;
    std::vector<FcgItem> items;
    WlRecord ap;
    ap.kind = WL_APPLY;
    ap.dbl = true;
    ap.mask = true;
    ap.dot = true;
    ap.ff = mixed && o.tol >= kFfMinTol;     // the outer apply in float-float where every item allows it
    for (size_t j = 0; j < G.probs.size(); ++j) {
        glls_problem* P = G.probs[j];
        const DevLevel<double>& F = P->L64[L].dev;
        double* prz = P->part;
        double* pzq = prz + kDotBlocks;
        double* prr = pzq + kDotBlocks;
        double* ppq = prr + kDotBlocks;
        FcgItem it{P->xk, P->rk, P->pk, P->qk, P->zk, mixed ? P->r32 : nullptr, mixed ? P->z32 : nullptr,
                   P->N, prz, pzq, prr, ppq, apply_list_blocks(F.p, F.E), nullptr, P->ticket};
        items.push_back(it);
        ap.p = F.p;
        ap.ff = ap.ff && F.dim == 2 && apply_ff_supported(F);
        ApplyItem<double> ai{F, P->pk, P->qk, ppq, nullptr};
        ap.put(ai, apply_list_blocks(F.p, F.E), (int)j);
    }
    // CTAs per problem of the outer-Krylov kernels: enough for the largest
    // problem of the group (about 16 values per thread), not kDotBlocks for
    // every one: each CTA also sums all of its problem's partials
    long long nmax = 1;
    for (glls_problem* P : G.probs) nmax = std::max(nmax, P->N);
    const int nblk = fcg_blocks(nmax);
    for (int step : {0, 1, -1, 2}) {
        if (step == -1) {
            G.body.push_back(ap);
            continue;
        }
        WlRecord r;
        r.kind = WL_FCG;
        r.step = step;
        r.dbl = true;
        r.blocks = nblk;
        for (size_t j = 0; j < items.size(); ++j) {
            const FcgItem& it = items[j];
            const unsigned char* b = reinterpret_cast<const unsigned char*>(&it);
            r.items.insert(r.items.end(), b, b + sizeof(FcgItem));
            r.start.push_back(0);
            r.owner.push_back((int)j);
            ++r.nitems;
        }
        G.body.push_back(std::move(r));
    }
    return "";
}

// Problem j of a group uses S = (plan block) + off_S + j S_COUNT: the FCG
// items get that pointer, every other item a pointer to its S_DONE flag,
// once the block is allocated.
void bind_scalars(WlGroup& G, unsigned char* base) {
    double* S = reinterpret_cast<double*>(base + G.off_S);
    for (auto& r : G.body)
        for (int i = 0; i < r.nitems; ++i) {
            double* Sj = S + (size_t)r.owner[i] * S_COUNT;
            if (r.kind == WL_FCG) {
                FcgItem it;
                std::memcpy(&it, r.items.data() + sizeof(FcgItem) * i, sizeof(FcgItem));
                it.S = Sj;
                std::memcpy(r.items.data() + sizeof(FcgItem) * i, &it, sizeof(FcgItem));
            } else {
                const double* done = Sj + S_DONE;
                std::memcpy(r.items.data() + r.item_bytes * i + r.done_at, &done, sizeof(done));
            }
        }
}

cudaError_t replay(const WlRecord& r, const unsigned char* base, int flexible, cudaStream_t st) {
    const void* items = base + r.off_items;
    const int* start = reinterpret_cast<const int*>(base + r.off_start);
    bool ok = true;
    switch (r.kind) {
        case WL_APPLY:
            if (r.ff) {
                ok = launch_apply_ff_list(r.p, (const ApplyItem<double>*)items, start, r.nitems, r.blocks, r.mask, st);
                break;
            }
            ok = r.dbl ? launch_apply_list<double>(r.p, (const ApplyItem<double>*)items, start, r.nitems, r.blocks,
                                                   r.mask, r.dot, st)
                       : launch_apply_list<float>(r.p, (const ApplyItem<float>*)items, start, r.nitems, r.blocks,
                                                  r.mask, r.dot, st);
            break;
        case WL_LINE:
            ok = r.dbl ? launch_line_block_list<double>(r.p, r.cv, items, start, r.nitems, r.blocks, r.threads, r.smem,
                                                        st)
                       : launch_line_block_list<float>(r.p, r.cv, items, start, r.nitems, r.blocks, r.threads, r.smem,
                                                       st);
            break;
        case WL_T2:
            ok = r.dbl ? launch_transfer2_list<double>(r.wb, r.ty, (const Transfer2Item<double>*)items, start,
                                                       r.nitems, r.blocks, r.smem, r.add, r.mask, st)
                       : launch_transfer2_list<float>(r.wb, r.ty, (const Transfer2Item<float>*)items, start, r.nitems,
                                                      r.blocks, r.smem, r.add, r.mask, st);
            break;
        case WL_BCR_F:
        case WL_BCR_B:
            if (r.dbl)
                launch_bcr_list<double>(r.kind == WL_BCR_F, r.l, (const BcrItem<double>*)items, start, r.nitems,
                                        r.blocks, r.smem, st);
            else
                launch_bcr_list<float>(r.kind == WL_BCR_F, r.l, (const BcrItem<float>*)items, start, r.nitems,
                                       r.blocks, r.smem, st);
            break;
        case WL_COARSE:
            if (r.dbl)
                launch_coarse_list<double>((const CoarseItem<double>*)items, start, r.nitems, r.blocks, r.smem, st);
            else
                launch_coarse_list<float>((const CoarseItem<float>*)items, start, r.nitems, r.blocks, r.smem, st);
            break;
        default:
            launch_fcg_list(r.step, (const FcgItem*)items, r.nitems, flexible, r.blocks, st);
    }
    if (!ok) return cudaErrorInvalidConfiguration;
    return cudaGetLastError();
}

// Captures the whole batched solve of W (all groups as graph branches).
cudaError_t capture_plan(WlPlan* W, const glls_solve_opts* o) {
    unsigned char* base = static_cast<unsigned char*>(W->dev);
    // GLLS_WORKLIST_PASSES=k (profiling aid): k passes of the loop body
    // captured inline instead of the device-side loop, so that a profiler
    // that does not list kernels inside conditional nodes sees them; the
    // solve then stops after k iterations
    const char* up = std::getenv("GLLS_WORKLIST_PASSES");
    const int unroll = up ? std::max(0, std::atoi(up)) : 0;
    const int flexible = o->krylov == GLLS_KRYLOV_FCG ? 1 : 0;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> joins(W->groups.size(), nullptr);
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (size_t i = 0; i < joins.size() && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&joins[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(W->master, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(fork, W->master);
    for (size_t gi = 0; gi < W->groups.size() && e == cudaSuccess; ++gi) {
        WlGroup& G = W->groups[gi];
        double* S = reinterpret_cast<double*>(base + G.off_S);
        const int n = (int)G.probs.size();
        e = cudaStreamWaitEvent(G.s1, fork, 0);
        for (int j = 0; j < n && e == cudaSuccess; ++j) {
            glls_problem* P = G.probs[j];
            solve_prologue(P, o, G.s1);
            e = cudaMemcpyAsync(S + (size_t)j * S_COUNT, P->S, sizeof(double) * S_COUNT, cudaMemcpyDeviceToDevice,
                                G.s1);
        }
        if (unroll > 0) {
            // profiling form: `unroll` passes of the body inline, no
            // conditional node (ncu lists the kernels of the passes)
            launch_solve_init(S, 0, o->tol, o->max_iter, G.s1, n, false);
            for (int k = 0; k < unroll && e == cudaSuccess; ++k) {
                for (const WlRecord& r : G.body)
                    if (e == cudaSuccess) e = replay(r, base, flexible, G.s1);
                launch_solve_cond(S, 0, o->max_iter, G.s1, n, false);
            }
        } else {
            cudaStreamCaptureStatus stt;
            cudaGraph_t capg = nullptr;
            cudaGraphConditionalHandle handle = 0;
            if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(G.s1, &stt, nullptr, &capg, nullptr, nullptr, nullptr);
            if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&handle, capg, 0, cudaGraphCondAssignDefault);
            if (e != cudaSuccess) break;
            launch_solve_init(S, handle, o->tol, o->max_iter, G.s1, n);
            const cudaGraphNode_t* deps = nullptr;
            size_t ndeps = 0;
            e = cudaStreamGetCaptureInfo(G.s1, &stt, nullptr, &capg, &deps, nullptr, &ndeps);
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = handle;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t cnode = nullptr;
            if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, capg, deps, nullptr, ndeps, &cp);
            if (e == cudaSuccess)
                e = cudaStreamUpdateCaptureDependencies(G.s1, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
            if (e == cudaSuccess) {
                cudaGraph_t body = cp.conditional.phGraph_out[0];
                e = cudaStreamBeginCaptureToGraph(G.s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    for (const WlRecord& r : G.body)
                        if (e == cudaSuccess) e = replay(r, base, flexible, G.s2);
                    launch_solve_cond(S, handle, o->max_iter, G.s2, n);
                    cudaError_t e2 = cudaStreamEndCapture(G.s2, &body);
                    if (e == cudaSuccess) e = e2;
                    if (e == cudaSuccess) G.kernels_iter = count_kernel_nodes(body);
                }
            }
        }
        for (int j = 0; j < n && e == cudaSuccess; ++j) {   // u = w + v; the scalars back to the problem
            glls_problem* P = G.probs[j];
            e = cudaMemcpyAsync(P->yk, P->xk, sizeof(double) * P->N, cudaMemcpyDeviceToDevice, G.s1);
            launch_axpy(P->yk, P->v, 1.0, P->N, G.s1);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(P->S, S + (size_t)j * S_COUNT, sizeof(double) * S_COUNT,
                                    cudaMemcpyDeviceToDevice, G.s1);
        }
        if (e == cudaSuccess) e = cudaEventRecord(joins[gi], G.s1);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(W->master, joins[gi], 0);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(W->master, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) W->kernels_fixed = count_kernel_nodes(graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&W->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (fork) cudaEventDestroy(fork);
    for (auto ev : joins)
        if (ev) cudaEventDestroy(ev);
    return e;
}

glls_status make_plan(glls_problem* const* probs, int n, const glls_solve_opts* o, WlPlan** out) {
    std::unique_ptr<WlPlan, void (*)(WlPlan*)> W(new WlPlan(), destroy_plan);
    W->probs.assign(probs, probs + n);
    W->key = *o;
    for (int i = 0; i < n; ++i) {
        glls_problem* P = probs[i];
        if (P->dim != 2) return fail(GLLS_ERR_INVALID, "work-list batch: 2-D problems only");
        if (P->smoother != GLLS_SMOOTHER_GLL) return fail(GLLS_ERR_INVALID, "work-list batch: GLL line-block smoother only");
        for (size_t l = 0; l < P->L64.size(); ++l) {
            const DevLevel<double>& L = P->L64[l].dev;
            if (L.p > 16 || L.N > (1LL << 31) - 1 || L.ne[0] >= 1024 || L.ne[1] >= 1024)
                return fail(GLLS_ERR_INVALID, "work-list batch: a level outside the specialised apply's range");
            if (l > 0 && (!L.blk[0] || !L.blk[1]))
                return fail(GLLS_ERR_INVALID, "work-list batch: a level without line blocks");
        }
        size_t gi = 0;
        while (gi < W->groups.size() && W->groups[gi].probs[0]->orders != P->orders) ++gi;
        if (gi == W->groups.size()) W->groups.emplace_back();
        W->groups[gi].probs.push_back(P);
        W->groups[gi].index.push_back(i);
    }
    // records, then one device block for every item array, start array and
    // group scalar array
    size_t bytes = 0;
    auto take = [&](size_t b) {
        const size_t at = bytes;
        bytes += (b + 255) / 256 * 256;
        return at;
    };
    for (auto& G : W->groups) {
        std::string err = build_group(G, *o);
        if (!err.empty()) return fail(GLLS_ERR_INVALID, "work-list batch: " + err);
        G.off_S = take(sizeof(double) * S_COUNT * G.probs.size());
        for (auto& r : G.body) {
            r.off_items = take(r.items.size());
            r.off_start = take(sizeof(int) * r.start.size());
        }
    }
    CK(dev_malloc(&W->dev, bytes));
    std::vector<unsigned char> host(bytes, 0);
    for (auto& G : W->groups) {
        bind_scalars(G, static_cast<unsigned char*>(W->dev));
        for (auto& r : G.body) {
            std::memcpy(host.data() + r.off_items, r.items.data(), r.items.size());
            std::memcpy(host.data() + r.off_start, r.start.data(), sizeof(int) * r.start.size());
        }
    }
    CK(cudaMemcpy(W->dev, host.data(), bytes, cudaMemcpyHostToDevice));
    CK(cudaStreamCreateWithFlags(&W->master, cudaStreamNonBlocking));
    for (auto& G : W->groups) {
        CK(cudaStreamCreateWithFlags(&G.s1, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&G.s2, cudaStreamNonBlocking));
    }
    CK(capture_plan(W.get(), o));
    *out = W.release();
    return GLLS_OK;
}

// After a breakdown the instance's work vectors can hold Inf or NaN where the
// solve kernels rely on zeros they never write (set-up leaves them zero: for
// instance boundary entries of the level iterates, where a prolongation of an
// infinite coarse value gives 0 * Inf).  They are cleared so that the next
// solve, in either precision, starts from the state set-up left.
template <typename T>
void clear_level_vectors(std::vector<LevelStore<T>>& Ls, int nrhs, cudaStream_t st) {
    for (auto& l : Ls) {
        const size_t bytes = sizeof(T) * (size_t)(l.dev.N * nrhs);
        T* vs[] = {l.r, l.x, l.y, l.t1, l.t2};
        for (T* v : vs) cudaMemsetAsync(v, 0, bytes, st);
    }
}

void clear_work_vectors(glls_problem* P, cudaStream_t st) {
    const long long NK = P->N * P->nrhs;
    double* vd[] = {P->xk, P->rk, P->pk, P->qk, P->zk};
    for (double* v : vd) cudaMemsetAsync(v, 0, sizeof(double) * NK, st);
    float* vf[] = {P->r32, P->z32};
    for (float* v : vf) cudaMemsetAsync(v, 0, sizeof(float) * NK, st);
    clear_level_vectors(P->L64, P->nrhs, st);
    clear_level_vectors(P->L32, P->nrhs, st);
    cudaStreamSynchronize(st);
}

}  // namespace

extern "C" {

const char* glls_last_error(void) { return g_last_error.c_str(); }

glls_status glls_gll(int p, double* xi, double* rho) {
    if (p < 1 || p > 64 || !xi) return fail(GLLS_ERR_INVALID, "glls_gll: need 1 <= p <= 64 and xi != NULL");
    std::vector<double> w;
    std::vector<double> x = gll_nodes(p, &w);
    std::memcpy(xi, x.data(), sizeof(double) * (p + 1));
    if (rho) std::memcpy(rho, w.data(), sizeof(double) * (p + 1));
    return GLLS_OK;
}

static glls_status problem_create(const glls_mesh_desc* desc, int nrhs, glls_problem** out) {
    if (!desc || !out) return fail(GLLS_ERR_INVALID, "null argument");
    *out = nullptr;
    if (desc->dim != 2 && desc->dim != 3) return fail(GLLS_ERR_INVALID, "dim must be 2 or 3");
    // the generic apply stages an element in shared memory: (p+1)^2 (2-D) or (p+1)^3 (3-D) nodes
    if (desc->order < 1 || desc->order > (desc->dim == 2 ? 64 : 16))
        return fail(GLLS_ERR_INVALID, "order must be in 1..64 (2-D) or 1..16 (3-D)");
    for (int a = 0; a < desc->dim; ++a)
        if (desc->nelem[a] < 1 || desc->nelem[a] > 4096) return fail(GLLS_ERR_INVALID, "nelem out of range");
    if (!desc->coords) return fail(GLLS_ERR_INVALID, "coords is NULL");
    bool multi = desc->nelem[0] > 1 || desc->nelem[1] > 1 || (desc->dim == 3 && desc->nelem[2] > 1);
    if (!multi && desc->order < 2) return fail(GLLS_ERR_INVALID, "a single element needs order >= 2");
    if (desc->smoother != GLLS_SMOOTHER_GLL && desc->smoother != GLLS_SMOOTHER_FEM &&
        desc->smoother != GLLS_SMOOTHER_GLL_BAND1)
        return fail(GLLS_ERR_INVALID, "bad smoother");
    if (desc->restriction != GLLS_RESTRICT_TRANSPOSE && desc->restriction != GLLS_RESTRICT_INTERP)
        return fail(GLLS_ERR_INVALID, "bad restriction");
    if (desc->summation != GLLS_SUM_ATOMIC && desc->summation != GLLS_SUM_COLORED)
        return fail(GLLS_ERR_INVALID, "bad summation");
    if (desc->smoother == GLLS_SMOOTHER_GLL && desc->order >= 2)
        for (int a = 0; a < desc->dim; ++a)
            if (!line_block_supported(desc->nelem[a] * desc->order - 1, desc->nelem[a]))
                return fail(GLLS_ERR_INVALID, "GLL line-block smoother: at most " + std::to_string(kMaxBlockSegments) +
                                                  " elements and " + std::to_string(kMaxBlockLine) +
                                                  " interior nodes per grid line");
    auto t0 = std::chrono::steady_clock::now();
    DeviceScope scope(desc->device);
    CK(scope.err);
    static std::once_flag once;
    static bool attrs_ok = false;
    std::call_once(once, [] {
        std::lock_guard<std::recursive_mutex> dev_lock(g_device_mutex);
        attrs_ok = init_kernel_attributes();
    });
    if (!attrs_ok) return fail(GLLS_ERR_CUDA, "could not set kernel shared-memory attributes");

    if (nrhs < 1 || nrhs > 4096) return fail(GLLS_ERR_INVALID, "nrhs must be in 1..4096");
    ProblemPtr P(new glls_problem());
    P->nrhs = nrhs;
    P->shared = std::make_shared<SharedData>();
    P->shared->device = desc->device;
    P->device = desc->device;
    P->dim = desc->dim;
    P->p = desc->order;
    P->smoother = desc->smoother;
    P->restriction = desc->restriction;
    for (int a = 0; a < 3; ++a) P->nelem[a] = a < desc->dim ? desc->nelem[a] : 1;
    std::vector<LevelHost> H;
    std::string err = build_levels(desc->dim, P->nelem, desc->order, desc->coords, desc->smoother,
                                   desc->restriction, H, P->setup_phase_ms);
    auto t_coarse = std::chrono::steady_clock::now();
    if (!err.empty()) return fail(GLLS_ERR_BREAKDOWN, err);
    for (auto& h : H) {
        if (h.N > 2147483647LL || h.E * h.nloc * h.ncomp > 2147483647LL)
            return fail(GLLS_ERR_INVALID, "problem too large for 32-bit node indexing");
        P->orders.push_back(h.p);
        for (long long i = 0; i < h.N; ++i) {
            // zero pivots would break cyclic reduction without pivoting
            bool inner = true;
            long long I = i % h.n[0], J = (i / h.n[0]) % h.n[1], K = i / ((long long)h.n[0] * h.n[1]);
            if (I == 0 || I == h.n[0] - 1 || J == 0 || J == h.n[1] - 1 ||
                (h.dim == 3 && (K == 0 || K == h.n[2] - 1)))
                inner = false;
            if (inner && !(h.diag[i] > 0.0)) return fail(GLLS_ERR_BREAKDOWN, "non-positive line-system diagonal");
        }
    }
    if (desc->coarse_solver < 0 || desc->coarse_solver > 2 || desc->coarse_cr_levels < 0)
        return fail(GLLS_ERR_INVALID, "coarse_solver must be GLLS_COARSE_* and coarse_cr_levels >= 0");
    CoarseHost C;
    err = build_coarse(H[0], desc->coarse_solver, desc->coarse_cr_levels, C);
    if (!err.empty())
        return fail(err.find("too large") != std::string::npos || err.find("more than") != std::string::npos
                        ? GLLS_ERR_INVALID
                        : GLLS_ERR_BREAKDOWN,
                    err);
    if (C.cr_levels > kMaxCrLevels) return fail(GLLS_ERR_INVALID, "too many block-CR levels");
    auto t_upload = std::chrono::steady_clock::now();
    P->setup_phase_ms[4] = std::chrono::duration<double, std::milli>(t_upload - t_coarse).count();

    std::lock_guard<std::recursive_mutex> dev_lock(g_device_mutex);
    glls_status st = upload_levels<double>(P.get(), H, P->L64);
    if (st != GLLS_OK) return st;
    st = upload_levels<float>(P.get(), H, P->L32);
    if (st != GLLS_OK) return st;
    for (auto& l : P->L64) l.dev.colored = desc->summation == GLLS_SUM_COLORED;
    for (auto& l : P->L32) l.dev.colored = desc->summation == GLLS_SUM_COLORED;
    {
        // float-float outer apply: the FP32 rounding remainders of the finest
        // level's FP64 geometric factors (the FP32 level holds the rounded
        // values)
        const size_t lf = H.size() - 1;
        DevLevel<double>& F64 = P->L64[lf].dev;
        if (F64.p >= 2 && F64.p <= (F64.dim == 2 ? 16 : 8)) {
            const std::vector<double>& G = H[lf].G;
            std::vector<float> lo(G.size());
            for (size_t i = 0; i < G.size(); ++i) lo[i] = (float)(G[i] - (double)(float)G[i]);
            CK(P->upload(&F64.Glo, lo));
            F64.Ghi = P->L32[lf].dev.G;
        }
    }
    st = upload_coarse<double>(P.get(), C, P->C64);
    if (st == GLLS_OK) st = upload_coarse<float>(P.get(), C, P->C32);
    if (st != GLLS_OK) return st;
    P->C32.index = P->C64.index;

    const LevelHost& F = H.back();
    P->N = F.N;
    P->N0 = H[0].N;
    CK(P->upload(&P->mass, F.mass));
    st = alloc_instance(P.get());
    if (st != GLLS_OK) return st;
    CK(cudaDeviceSynchronize());
    P->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    P->setup_phase_ms[5] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_upload).count();
    *out = P.release();
    return GLLS_OK;
}

static glls_status problem_clone(const glls_problem* src, int nrhs, glls_problem** out) {
    if (!src || !out) return fail(GLLS_ERR_INVALID, "null argument");
    *out = nullptr;
    if (nrhs < 1 || nrhs > 4096) return fail(GLLS_ERR_INVALID, "nrhs must be in 1..4096");
    DeviceScope scope(src->device);
    CK(scope.err);
    ProblemPtr P(new glls_problem());
    std::lock_guard<std::recursive_mutex> dev_lock(g_device_mutex);
    P->nrhs = nrhs;
    P->shared = src->shared;
    P->device = src->device;
    P->dim = src->dim;
    for (int a = 0; a < 3; ++a) P->nelem[a] = src->nelem[a];
    P->p = src->p;
    P->smoother = src->smoother;
    P->restriction = src->restriction;
    P->orders = src->orders;
    P->C64 = src->C64;
    P->C32 = src->C32;
    P->N = src->N;
    P->N0 = src->N0;
    P->mass = src->mass;
    P->L64.resize(src->L64.size());
    P->L32.resize(src->L32.size());
    for (size_t l = 0; l < src->L64.size(); ++l) {
        P->L64[l].dev = src->L64[l].dev;
        P->L32[l].dev = src->L32[l].dev;
    }
    glls_status st = alloc_level_vectors<double>(P.get(), P->L64);
    if (st == GLLS_OK) st = alloc_level_vectors<float>(P.get(), P->L32);
    if (st == GLLS_OK) st = alloc_instance(P.get());
    if (st != GLLS_OK) return st;
    CK(cudaDeviceSynchronize());
    *out = P.release();
    return GLLS_OK;
}

// Host allocations of the set-up (std::vector) report GLLS_ERR_OOM instead of
// throwing across the ABI.
glls_status glls_problem_create(const glls_mesh_desc* desc, glls_problem** out) {
    return glls_problem_create_nrhs(desc, 1, out);
}

glls_status glls_problem_create_nrhs(const glls_mesh_desc* desc, int nrhs, glls_problem** out) {
    try {
        return problem_create(desc, nrhs, out);
    } catch (const std::bad_alloc&) {
        return fail(GLLS_ERR_OOM, "host allocation failed during set-up");
    } catch (const std::exception& e) {
        return fail(GLLS_ERR_INVALID, std::string("set-up failed: ") + e.what());
    }
}

glls_status glls_problem_clone(const glls_problem* src, glls_problem** out) {
    return glls_problem_clone_nrhs(src, src ? src->nrhs : 1, out);
}

glls_status glls_problem_clone_nrhs(const glls_problem* src, int nrhs, glls_problem** out) {
    try {
        return problem_clone(src, nrhs, out);
    } catch (const std::bad_alloc&) {
        return fail(GLLS_ERR_OOM, "host allocation failed during clone");
    }
}

void glls_debug_fail_alloc_after(long long n) { g_alloc_countdown.store(n < 0 ? -1 : n); }

void glls_problem_destroy(glls_problem* P) {
    if (!P) return;
    std::lock_guard<std::recursive_mutex> dev_lock(g_device_mutex);
    forget_batches_of(P);
    DeviceScope scope(P->device);
    if (P->iter_exec) cudaGraphExecDestroy(P->iter_exec);
    if (P->solve_exec) cudaGraphExecDestroy(P->solve_exec);
    if (P->capture_stream) cudaStreamDestroy(P->capture_stream);
    if (P->capture_stream2) cudaStreamDestroy(P->capture_stream2);
    for (void* a : P->allocs) cudaFree(a);
    if (P->hostS) cudaFreeHost(P->hostS);
    delete P;
}

glls_status glls_problem_info(const glls_problem* P, glls_info* out) {
    if (!P || !out) return fail(GLLS_ERR_INVALID, "null argument");
    std::memset(out, 0, sizeof(*out));
    out->dim = P->dim;
    out->levels = (int)P->L64.size();
    for (size_t l = 0; l < P->L64.size() && l < 8; ++l) {
        out->order[l] = P->L64[l].dev.p;
        for (int a = 0; a < 3; ++a) out->nodes[l][a] = P->L64[l].dev.n[a];
        out->ndof[l] = P->L64[l].dev.N;
    }
    out->coarse_unknowns = P->C64.n;
    out->coarse_cr_levels = P->C64.cr_levels;
    out->coarse_dense_unknowns = P->C64.nr;
    out->device_bytes = P->bytes + (P->shared ? P->shared->bytes : 0);
    out->instance_bytes = P->bytes;
    out->nrhs = P->nrhs;
    for (int k = 0; k < 6; ++k) out->setup_phase_ms[k] = P->setup_phase_ms[k];
    return GLLS_OK;
}

glls_status glls_set_dirichlet(glls_problem* P, const double* g, int on_device, void* stream) {
    if (!P || !g) return fail(GLLS_ERR_INVALID, "null argument");
    DeviceScope scope(P->device);
    CK(scope.err);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(P->g, g, sizeof(double) * P->N, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    if (!on_device) CK(cudaStreamSynchronize(st));
    P->has_dirichlet = true;
    return GLLS_OK;
}

glls_status glls_set_rhs(glls_problem* P, const double* f, int on_device, void* stream) {
    if (!P || !f) return fail(GLLS_ERR_INVALID, "null argument");
    DeviceScope scope(P->device);
    CK(scope.err);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(P->f, f, sizeof(double) * P->N * P->nrhs,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    if (!on_device) CK(cudaStreamSynchronize(st));
    P->has_rhs = true;
    return GLLS_OK;
}

glls_status glls_lift_f64(glls_problem* P, const double* f, const double* g, double* f0, void* stream) {
    if (!P || !f || !g || !f0) return fail(GLLS_ERR_INVALID, "null argument");
    DeviceScope scope(P->device);
    CK(scope.err);
    cudaStream_t st = (cudaStream_t)stream;
    const int L = (int)P->L64.size() - 1;
    const DevLevel<double>& F = P->L64[L].dev;
    launch_boundary_only(g, P->v, F.n, F.dim, st);
    launch_apply<double>(F, P->v, P->yk, false, st);
    launch_lift_rhs(P->mass, f, P->yk, f0, F.n, F.dim, st);
    CK(cudaGetLastError());
    return GLLS_OK;
}

static glls_status solve_impl(glls_problem* P, const glls_solve_opts* o, double* u, int on_device, void* stream,
                              glls_stats* stats) {
    if (!P || !u) return fail(GLLS_ERR_INVALID, "null argument");
    if (P->nrhs > 1 && o && (o->use_graph != 2 || o->krylov == GLLS_KRYLOV_GMRES))
        return fail(GLLS_ERR_INVALID, "several right-hand sides: use_graph = 2 and FCG or PCG");
    glls_status s0 = check_opts(o);
    if (s0 != GLLS_OK) return s0;
    if (!P->has_rhs) return fail(GLLS_ERR_INVALID, "right-hand side not set");
    DeviceScope scope(P->device);
    CK(scope.err);
    cudaStream_t st = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    const long long N = P->N;
    if (!P->has_dirichlet) CK(cudaMemsetAsync(P->g, 0, sizeof(double) * N, st));
    int it = 0;
    double rel = 0.0;
    glls_status result = GLLS_OK;
    if (o->krylov == GLLS_KRYLOV_GMRES) {
        result = gmres_solve(P, o, st, &it, &rel);
        if (result != GLLS_OK && result != GLLS_ERR_NOT_CONVERGED) return result;
        CK(cudaMemcpyAsync(P->yk, P->xk, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        launch_axpy(P->yk, P->v, 1.0, N, st);
        CK(cudaMemcpyAsync(u, P->yk, sizeof(double) * N, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           st));
        CK(cudaStreamSynchronize(st));
        CK(cudaGetLastError());
        if (stats) {
            stats->iterations = it;
            stats->rel_residual = rel;
            stats->setup_ms = P->setup_ms;
            stats->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            stats->status = result;
            stats->kernels = 0;
        }
        return result;
    }
    if (o->use_graph == 2) {
        // whole solve on the device: one graph launch, one synchronisation
        glls_status gs = get_solve_graph(P, o);
        if (gs != GLLS_OK) return gs;
        CK(cudaGraphLaunch(P->solve_exec, st));
        CK(cudaMemcpyAsync(u, P->yk, sizeof(double) * N * P->nrhs,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(P->hostS, P->S, sizeof(double) * S_COUNT * P->nrhs, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        CK(cudaGetLastError());
        result = solve_result(P, P->hostS, stats,
                              std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
        if (result == GLLS_ERR_BREAKDOWN) fail(result, "breakdown in the outer iteration (p.Ap <= 0 or NaN)");
        if (result == GLLS_ERR_NOT_CONVERGED) fail(result, "max_iter reached");
        (void)it;
        (void)rel;
        return result;
    }
    // host-driven loop: prologue, then one outer iteration per launch
    solve_prologue(P, o, st);
    double init[S_COUNT] = {0};
    CK(cudaMemcpyAsync(P->hostS, P->S, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const double rr0 = P->hostS[S_RR0];
    init[S_RZ] = 1.0;
    init[S_RR0] = rr0;
    std::memcpy(P->hostS, init, sizeof(init));
    CK(cudaMemcpyAsync(P->S, P->hostS, sizeof(init), cudaMemcpyHostToDevice, st));
    if (!(rr0 >= 0.0) || !std::isfinite(rr0)) {
        result = fail(GLLS_ERR_BREAKDOWN, "non-finite right-hand side");
    } else if (rr0 > 0.0) {
        const double tol2 = o->tol * o->tol * rr0;
        if (o->use_graph) {
            glls_status gs = get_iteration_graph(P, o);
            if (gs != GLLS_OK) return gs;
        }
        const int every = o->check_every > 0 ? o->check_every : 1;
        result = GLLS_ERR_NOT_CONVERGED;
        while (it < o->max_iter) {
            if (o->use_graph) CK(cudaGraphLaunch(P->iter_exec, st));
            else outer_iteration(P, o, st);
            ++it;
            if (it % every == 0 || it == o->max_iter) {
                CK(cudaMemcpyAsync(P->hostS, P->S, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                if (P->hostS[S_FLAG] != 0.0 || !std::isfinite(P->hostS[S_RR])) {
                    result = fail(GLLS_ERR_BREAKDOWN, "breakdown in the outer iteration (p.Ap <= 0 or NaN)");
                    break;
                }
                if (P->hostS[S_RR] <= tol2) {
                    result = GLLS_OK;
                    break;
                }
            }
        }
        if (result == GLLS_ERR_NOT_CONVERGED) fail(GLLS_ERR_NOT_CONVERGED, "max_iter reached");
        rel = std::sqrt(P->hostS[S_RR] / rr0);
    }
    CK(cudaGetLastError());
    // u = w + v
    CK(cudaMemcpyAsync(P->yk, P->xk, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    launch_axpy(P->yk, P->v, 1.0, N, st);
    CK(cudaMemcpyAsync(u, P->yk, sizeof(double) * N, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    if (!on_device || stats) CK(cudaStreamSynchronize(st));
    if (stats) {
        stats->iterations = it;
        stats->rel_residual = rel;
        stats->setup_ms = P->setup_ms;
        stats->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        stats->status = result;
    }
    return result;
}

// stats is filled on every return: its status is the call's status even where
// the solve stopped before any iteration.
glls_status glls_solve(glls_problem* P, const glls_solve_opts* o, double* u, int on_device, void* stream,
                       glls_stats* stats) {
    const int k = P ? P->nrhs : 1;
    if (stats) std::memset(stats, 0, sizeof(*stats) * k);
    const glls_status r = solve_impl(P, o, u, on_device, stream, stats);
    if (r == GLLS_ERR_BREAKDOWN) {
        DeviceScope scope(P->device);
        if (scope.err == cudaSuccess) clear_work_vectors(P, (cudaStream_t)stream);
    }
    if (stats) {
        if (k == 1) {
            stats[0].status = r;
        } else if (r != GLLS_OK && r != GLLS_ERR_NOT_CONVERGED && r != GLLS_ERR_BREAKDOWN) {
            for (int j = 0; j < k; ++j) stats[j].status = r;   // nothing ran: every right-hand side failed
        }
    }
    return r;
}

glls_status glls_estimate_bytes(const glls_mesh_desc* desc, size_t* bytes) {
    if (!desc || !bytes) return fail(GLLS_ERR_INVALID, "null argument");
    if (desc->dim != 2 && desc->dim != 3) return fail(GLLS_ERR_INVALID, "dim must be 2 or 3");
    // the generic apply stages an element in shared memory: (p+1)^2 (2-D) or (p+1)^3 (3-D) nodes
    if (desc->order < 1 || desc->order > (desc->dim == 2 ? 64 : 16))
        return fail(GLLS_ERR_INVALID, "order must be in 1..64 (2-D) or 1..16 (3-D)");
    const int d = desc->dim;
    long long ne[3] = {1, 1, 1}, E = 1;
    for (int a = 0; a < d; ++a) {
        if (desc->nelem[a] < 1) return fail(GLLS_ERR_INVALID, "nelem must be >= 1");
        ne[a] = desc->nelem[a];
        E *= ne[a];
    }
    bool multi = true;                      // p = 1 has interior unknowns
    for (int a = 0; a < d; ++a) multi = multi && ne[a] > 1;
    std::vector<int> chain = order_chain(desc->order, multi);
    const int ncomp = d == 2 ? 3 : 6;
    double total = 0.0;
    long long Nfine = 0, n0 = 1;
    for (size_t c = 0; c < chain.size(); ++c) {
        const int p = chain[c];
        long long N = 1, nloc = 1, inner = 1;
        for (int a = 0; a < d; ++a) {
            N *= ne[a] * p + 1;
            nloc *= p + 1;
            inner *= ne[a] * p - 1;
        }
        if (c == 0) Nfine = N;
        if (c + 1 == chain.size()) n0 = inner;
        // G, diag, off, D in FP64 + FP32; packed (diag, off) pairs per direction; five level
        // vectors in each precision; transfer bands
        total += 12.0 * ((double)ncomp * E * nloc + (1 + d) * (double)N + (p + 1) * (p + 1)) + 12.0 * 5 * N;
        total += 24.0 * d * (double)N;
        if (c == 0 && p >= 2 && p <= (d == 2 ? 16 : 8)) total += 4.0 * ncomp * E * nloc;   // float-float G remainders
        total += 2.0 * d * (12.0 * (2 * p + 2) * (double)(ne[0] * p + 1) + 4.0 * (ne[0] * p + 1));
        if (desc->smoother == GLLS_SMOOTHER_GLL && p >= 2) {
            // condensed line blocks: per segment (p-1)p/2 + 2(p-1) values, per vertex 2 (FP64 + FP32)
            for (int s = 0; s < d; ++s) {
                double lines = 1.0;
                for (int a = 0; a < d; ++a)
                    if (a != s) lines *= (double)(ne[a] * p - 1);
                total += 12.0 * lines * ne[s] * ((p - 1) * p / 2.0 + 2.0 * (p - 1)) + 24.0 * lines * ne[s];
            }
        }
    }
    // coarsest solve: block-CR operators (FP64 + FP32) and the dense inverse of what is left
    const int p0 = chain.back();
    const int nb = (int)(ne[d - 1] * p0 - 1), m = nb > 0 ? (int)(n0 / nb) : 1;
    int k = 0;
    if (desc->coarse_solver == 2)
        k = std::min(desc->coarse_cr_levels > 0 ? desc->coarse_cr_levels : std::max(1, auto_cr_levels(nb, m)),
                     max_cr_levels(nb));
    else if (desc->coarse_solver == 0)
        k = auto_cr_levels(nb, m);
    if (k == 0 && (long long)nb * m > 16384 && desc->coarse_solver != 1)   // as build_coarse
        k = std::max(1, std::min(max_cr_levels(nb), auto_cr_levels(nb, m)));
    const double ldm = (double)((m + 3) / 4 * 4);
    for (int l = 0; l < k; ++l) {
        const int a = nb >> l;
        total += 12.0 * (2.0 * (a / 2) + 3.0 * ((a + 1) / 2)) * m * ldm;
    }
    const long long nr = (long long)(nb >> k) * m;
    const double ld64 = (double)((nr + 1) / 2 * 2), ld32 = (double)((nr + 3) / 4 * 4);
    total += 8.0 * n0 + (double)nr * (8.0 * ld64 + 4.0 * ld32);
    total += 8.0 * (11.0 * Nfine) + 8.0 * Nfine + 8.0 * std::max<double>(2 * kMaxReduceBlocks, E + 1) + 64.0;
    total += 4.0 * 2.0 * Nfine;                                          // r32, z32
    *bytes = (size_t)total;
    return GLLS_OK;
}

glls_status glls_solve_batch(glls_problem* const* probs, int n, const glls_solve_opts* o, double* const* u,
                             int on_device, void* stream, glls_stats* stats) {
    if (!probs || n < 1 || !u) return fail(GLLS_ERR_INVALID, "glls_solve_batch: need n >= 1 problems and outputs");
    if (stats) std::memset(stats, 0, sizeof(*stats) * n);
    glls_status s0 = check_opts(o);
    if (s0 != GLLS_OK) return s0;
    const int dev = probs[0] ? probs[0]->device : 0;
    for (int i = 0; i < n; ++i) {
        if (!probs[i] || !u[i]) return fail(GLLS_ERR_INVALID, "glls_solve_batch: null problem or output");
        if (probs[i]->device != dev) return fail(GLLS_ERR_INVALID, "glls_solve_batch: problems on different devices");
        if (!probs[i]->has_rhs) return fail(GLLS_ERR_INVALID, "glls_solve_batch: right-hand side not set");
        if (probs[i]->nrhs != 1)
            return fail(GLLS_ERR_INVALID, "glls_solve_batch: problems with one right-hand side only (glls_solve "
                                          "takes several)");
        for (int j = 0; j < i; ++j)
            if (probs[j] == probs[i]) return fail(GLLS_ERR_INVALID, "glls_solve_batch: a problem appears twice");
    }
    DeviceScope scope(dev);
    CK(scope.err);
    cudaStream_t st = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    for (int i = 0; i < n; ++i)
        if (!probs[i]->has_dirichlet) CK(cudaMemsetAsync(probs[i]->g, 0, sizeof(double) * probs[i]->N, st));
    cudaGraphExec_t exec = nullptr;
    {
        // lock order: device, then batch (as in glls_problem_destroy)
        std::lock_guard<std::recursive_mutex> dev_lock(g_device_mutex);
        std::lock_guard<std::mutex> lock(g_batch_mutex);
        std::vector<glls_problem*> key(probs, probs + n);
        for (size_t i = 0; i < g_batches.size(); ++i)
            if (g_batches[i].probs == key && same_solve_key(g_batches[i].key, *o)) {
                BatchEntry hit = g_batches[i];
                g_batches.erase(g_batches.begin() + i);
                g_batches.push_back(hit);
                exec = hit.exec;
                break;
            }
        if (!exec) {
            BatchEntry be;
            be.probs = key;
            be.key = *o;
            CK(cudaStreamCreateWithFlags(&be.master, cudaStreamNonBlocking));
            cudaEvent_t fork = nullptr;
            std::vector<cudaEvent_t> joins(n, nullptr);
            cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
            for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&joins[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaStreamBeginCapture(be.master, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                e = cudaEventRecord(fork, be.master);
                for (int i = 0; i < n && e == cudaSuccess; ++i) {
                    glls_problem* P = probs[i];
                    e = cudaStreamWaitEvent(P->capture_stream, fork, 0);
                    if (e == cudaSuccess) e = capture_solve(P, o, P->capture_stream, P->capture_stream2);
                    if (e == cudaSuccess) e = cudaEventRecord(joins[i], P->capture_stream);
                    if (e == cudaSuccess) e = cudaStreamWaitEvent(be.master, joins[i], 0);
                }
                cudaGraph_t graph = nullptr;
                cudaError_t e2 = cudaStreamEndCapture(be.master, &graph);
                if (e == cudaSuccess) e = e2;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&be.exec, graph, 0);
                if (graph) cudaGraphDestroy(graph);
            }
            if (fork) cudaEventDestroy(fork);
            for (auto ev : joins)
                if (ev) cudaEventDestroy(ev);
            if (e != cudaSuccess) {
                cudaStreamDestroy(be.master);
                CK(e);
            }
            exec = be.exec;
            g_batches.push_back(be);
            if (g_batches.size() > 8) {
                cudaGraphExecDestroy(g_batches.front().exec);
                cudaStreamDestroy(g_batches.front().master);
                g_batches.erase(g_batches.begin());
            }
        }
    }
    CK(cudaGraphLaunch(exec, st));
    for (int i = 0; i < n; ++i) {
        glls_problem* P = probs[i];
        CK(cudaMemcpyAsync(u[i], P->yk, sizeof(double) * P->N,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(P->hostS, P->S, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    const double t_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    glls_status worst = GLLS_OK;
    for (int i = 0; i < n; ++i) {
        glls_status r = solve_result(probs[i], probs[i]->hostS, stats ? &stats[i] : nullptr, t_ms);
        if (r == GLLS_ERR_BREAKDOWN) clear_work_vectors(probs[i], st);
        if (r != GLLS_OK && worst == GLLS_OK) worst = r;
    }
    if (worst == GLLS_ERR_BREAKDOWN) fail(worst, "breakdown in at least one problem of the batch");
    if (worst == GLLS_ERR_NOT_CONVERGED) fail(worst, "at least one problem of the batch reached max_iter");
    return worst;
}

glls_status glls_solve_batch_worklist(glls_problem* const* probs, int n, const glls_solve_opts* o, double* const* u,
                                      int on_device, void* stream, glls_stats* stats) {
    if (!probs || n < 1 || !u) return fail(GLLS_ERR_INVALID, "glls_solve_batch_worklist: need n >= 1 problems and outputs");
    if (stats) std::memset(stats, 0, sizeof(*stats) * n);
    glls_status s0 = check_opts(o);
    if (s0 != GLLS_OK) return s0;
    if (o->krylov == GLLS_KRYLOV_GMRES) return fail(GLLS_ERR_INVALID, "glls_solve_batch_worklist: FCG or PCG only");
    const int dev = probs[0] ? probs[0]->device : 0;
    for (int i = 0; i < n; ++i) {
        if (!probs[i] || !u[i]) return fail(GLLS_ERR_INVALID, "glls_solve_batch_worklist: null problem or output");
        if (probs[i]->device != dev) return fail(GLLS_ERR_INVALID, "glls_solve_batch_worklist: problems on different devices");
        if (!probs[i]->has_rhs) return fail(GLLS_ERR_INVALID, "glls_solve_batch_worklist: right-hand side not set");
        if (probs[i]->nrhs != 1) return fail(GLLS_ERR_INVALID, "glls_solve_batch_worklist: one right-hand side per problem");
        if (probs[i]->L64.back().dev.colored)
            return fail(GLLS_ERR_INVALID, "glls_solve_batch_worklist: coloured summation (GLLS_SUM_COLORED) is not "
                                          "in the work-list kernels; use glls_solve_batch");
        for (int j = 0; j < i; ++j)
            if (probs[j] == probs[i]) return fail(GLLS_ERR_INVALID, "glls_solve_batch_worklist: a problem appears twice");
    }
    DeviceScope scope(dev);
    CK(scope.err);
    cudaStream_t st = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    for (int i = 0; i < n; ++i)
        if (!probs[i]->has_dirichlet) CK(cudaMemsetAsync(probs[i]->g, 0, sizeof(double) * probs[i]->N, st));
    cudaGraphExec_t exec = nullptr;
    long long kfix = 0;
    std::vector<std::pair<std::vector<int>, long long>> loops;   // problems of a group, kernels per pass
    {
        std::lock_guard<std::recursive_mutex> dev_lock(g_device_mutex);
        std::lock_guard<std::mutex> lock(g_batch_mutex);
        std::vector<glls_problem*> key(probs, probs + n);
        for (size_t i = 0; i < g_wplans.size(); ++i)
            if (g_wplans[i]->probs == key && same_solve_key(g_wplans[i]->key, *o)) {
                WlPlan* hit = g_wplans[i];
                g_wplans.erase(g_wplans.begin() + i);
                g_wplans.push_back(hit);
                exec = hit->exec;
                kfix = hit->kernels_fixed;
                for (const auto& G : hit->groups) loops.emplace_back(G.index, G.kernels_iter);
                break;
            }
        if (!exec) {
            WlPlan* W = nullptr;
            glls_status ps = make_plan(probs, n, o, &W);
            if (ps != GLLS_OK) return ps;
            g_wplans.push_back(W);
            if (g_wplans.size() > 4) {
                destroy_plan(g_wplans.front());
                g_wplans.erase(g_wplans.begin());
            }
            exec = W->exec;
            kfix = W->kernels_fixed;
            for (const auto& G : W->groups) loops.emplace_back(G.index, G.kernels_iter);
        }
    }
    CK(cudaGraphLaunch(exec, st));
    for (int i = 0; i < n; ++i) {
        glls_problem* P = probs[i];
        CK(cudaMemcpyAsync(u[i], P->yk, sizeof(double) * P->N,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(P->hostS, P->S, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    const double t_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    glls_status worst = GLLS_OK;
    for (int i = 0; i < n; ++i) {
        glls_status r = solve_result(probs[i], probs[i]->hostS, stats ? &stats[i] : nullptr, t_ms);
        if (r == GLLS_ERR_BREAKDOWN) clear_work_vectors(probs[i], st);
        if (r != GLLS_OK && worst == GLLS_OK) worst = r;
    }
    if (stats) {
        // kernels of the whole launch, reported on the first problem: the
        // fixed nodes plus each group's loop body times its passes (the
        // group loops while any of its problems is active)
        long long total = kfix;
        for (const auto& g : loops) {
            double passes = 0;
            for (int i : g.first) passes = std::max(passes, probs[i]->hostS[S_ITER]);
            total += g.second * (long long)passes;
        }
        for (int i = 0; i < n; ++i) stats[i].kernels = i == 0 ? total : 0;
    }
    if (worst == GLLS_ERR_BREAKDOWN) fail(worst, "breakdown in at least one problem of the batch");
    if (worst == GLLS_ERR_NOT_CONVERGED) fail(worst, "at least one problem of the batch reached max_iter");
    return worst;
}

glls_status glls_autotune(glls_problem* P, int* chosen, float* best_us) {
    if (!P) return fail(GLLS_ERR_INVALID, "null problem");
    DeviceScope scope(P->device);
    CK(scope.err);
    const size_t cells = P->L64.size() * 2 * 3;
    if (chosen) std::fill(chosen, chosen + cells, 0);
    if (best_us) std::fill(best_us, best_us + cells, 0.f);
    glls_status s = tune_levels<float>(P, P->L32, 0, chosen, best_us);
    if (s == GLLS_OK) s = tune_levels<double>(P, P->L64, 1, chosen, best_us);
    // captured graphs hold the previous tiles
    if (P->iter_exec) { cudaGraphExecDestroy(P->iter_exec); P->iter_exec = nullptr; }
    if (P->solve_exec) { cudaGraphExecDestroy(P->solve_exec); P->solve_exec = nullptr; }
    forget_batches_of(P);
    return s;
}

// The outer iteration's FP64 apply: y = A_l x with the per-CTA partial sums
// of x.(A x) fused into the kernel (the consumer adds them).
glls_status glls_apply_partials_f64(glls_problem* P, int level, const double* x, double* y, double* partials,
                                    int capacity, int* count, void* stream) {
    glls_status s = check_level(P, level, false);
    if (s != GLLS_OK) return s;
    if (!x || !y || !partials || !count) return fail(GLLS_ERR_INVALID, "null argument");
    const DevLevel<double>& L = P->L64[level].dev;
    const int n = dot_partials_of(L);
    *count = n;
    if (capacity < n) return fail(GLLS_ERR_INVALID, "partials: need " + std::to_string(n) + " entries");
    DeviceScope scope(P->device);
    CK(scope.err);
    launch_apply<double>(L, x, y, true, (cudaStream_t)stream, true, partials, partials, nullptr);
    CK(cudaGetLastError());
    return GLLS_OK;
}

// The same product in float-float arithmetic, as the mixed-precision outer
// iteration launches it where the level allows (apply_ff.cu).
glls_status glls_apply_partials_ff(glls_problem* P, int level, const double* x, double* y, double* partials,
                                   int capacity, int* count, void* stream) {
    glls_status s = check_level(P, level, false);
    if (s != GLLS_OK) return s;
    if (!x || !y || !partials || !count) return fail(GLLS_ERR_INVALID, "null argument");
    const DevLevel<double>& L = P->L64[level].dev;
    if (!apply_ff_supported(L))
        return fail(GLLS_ERR_INVALID, "float-float apply: the finest level of a problem with 2 <= p <= 16 (2-D) "
                                      "or 2 <= p <= 8 (3-D) and atomic summation only");
    const int n = apply_ff_partials(L);
    *count = n;
    if (capacity < n) return fail(GLLS_ERR_INVALID, "partials: need " + std::to_string(n) + " entries");
    DeviceScope scope(P->device);
    CK(scope.err);
    if (!launch_apply_ff(L, x, y, true, partials, (cudaStream_t)stream, 1)) return fail(GLLS_ERR_CUDA, "launch failed");
    CK(cudaGetLastError());
    return GLLS_OK;
}

#define LEVEL_OPS(SUF, T)                                                                                      \
    glls_status glls_apply_multi_##SUF(glls_problem* P, int level, const T* x, T* y, int nrhs, void* stream) {  \
        glls_status s = check_level(P, level, false);                                                           \
        if (s != GLLS_OK) return s;                                                                             \
        if (!x || !y || nrhs < 1 || nrhs > 4096) return fail(GLLS_ERR_INVALID, "null vector or bad nrhs");      \
        DeviceScope scope(P->device);                                                                           \
        CK(scope.err);                                                                                          \
        CK(launch_apply<T>(levels_of<T>(P)[level].dev, x, y, true, (cudaStream_t)stream, false, nullptr,        \
                           nullptr, nullptr, nrhs));                                                            \
        CK(cudaGetLastError());                                                                                 \
        return GLLS_OK;                                                                                         \
    }                                                                                                           \
    glls_status glls_apply_##SUF(glls_problem* P, int level, const T* x, T* y, void* stream) {                  \
        glls_status s = check_level(P, level, false);                                                           \
        if (s != GLLS_OK) return s;                                                                             \
        if (!x || !y) return fail(GLLS_ERR_INVALID, "null vector");                                             \
        DeviceScope scope(P->device);                                                                           \
        CK(scope.err);                                                                                          \
        launch_apply<T>(levels_of<T>(P)[level].dev, x, y, true, (cudaStream_t)stream);                          \
        CK(cudaGetLastError());                                                                                 \
        return GLLS_OK;                                                                                         \
    }                                                                                                           \
    glls_status glls_line_solve_##SUF(glls_problem* P, int level, int axis, const T* g, T* x, void* stream) {   \
        glls_status s = check_level(P, level, false);                                                           \
        if (s != GLLS_OK) return s;                                                                             \
        if (axis < 0 || axis >= P->dim) return fail(GLLS_ERR_INVALID, "axis out of range");                     \
        if (!g || !x) return fail(GLLS_ERR_INVALID, "null vector");                                             \
        DeviceScope scope(P->device);                                                                           \
        CK(scope.err);                                                                                          \
        launch_line_solve<T>(levels_of<T>(P)[level].dev, axis, 0, g, nullptr, nullptr, x, T(1),                 \
                             (cudaStream_t)stream);                                                             \
        CK(cudaGetLastError());                                                                                 \
        return GLLS_OK;                                                                                         \
    }                                                                                                           \
    glls_status glls_smooth_##SUF(glls_problem* P, int level, int axis, T alpha, const T* r, T* x,              \
                                  void* stream) {                                                               \
        glls_status s = check_level(P, level, false);                                                           \
        if (s != GLLS_OK) return s;                                                                             \
        if (axis < 0 || axis >= P->dim) return fail(GLLS_ERR_INVALID, "axis out of range");                     \
        if (!r || !x) return fail(GLLS_ERR_INVALID, "null vector");                                             \
        DeviceScope scope(P->device);                                                                           \
        CK(scope.err);                                                                                          \
        smooth<T>(P, level, axis, alpha, r, x, false, (cudaStream_t)stream);                                    \
        CK(cudaGetLastError());                                                                                 \
        return GLLS_OK;                                                                                         \
    }                                                                                                           \
    glls_status glls_line_update_##SUF(glls_problem* P, int level, int axis, T alpha, const T* r, T* y, T* x,    \
                                       void* stream) {                                                          \
        glls_status s = check_level(P, level, false);                                                           \
        if (s != GLLS_OK) return s;                                                                             \
        if (axis < 0 || axis >= P->dim) return fail(GLLS_ERR_INVALID, "axis out of range");                     \
        if (!r || !y || !x) return fail(GLLS_ERR_INVALID, "null vector");                                       \
        DeviceScope scope(P->device);                                                                           \
        CK(scope.err);                                                                                          \
        launch_line_solve<T>(levels_of<T>(P)[level].dev, axis, 1, nullptr, r, y, x, alpha, (cudaStream_t)stream); \
        CK(cudaGetLastError());                                                                                 \
        return GLLS_OK;                                                                                         \
    }                                                                                                           \
    glls_status glls_restrict_##SUF(glls_problem* P, int level, const T* r, const T* x, T* rc, void* stream) {  \
        glls_status s = check_level(P, level, true);                                                            \
        if (s != GLLS_OK) return s;                                                                             \
        if (!r || !x || !rc) return fail(GLLS_ERR_INVALID, "null vector");                                      \
        DeviceScope scope(P->device);                                                                           \
        CK(scope.err);                                                                                          \
        auto& Ls = levels_of<T>(P);                                                                             \
        launch_apply<T>(Ls[level].dev, x, Ls[level].y, true, (cudaStream_t)stream, true);                       \
        restrict_residual<T>(P, level, r, Ls[level].y, rc, (cudaStream_t)stream);                               \
        CK(cudaMemsetAsync(Ls[level].y, 0, sizeof(T) * Ls[level].dev.N, (cudaStream_t)stream));                 \
        CK(cudaGetLastError());                                                                                 \
        return GLLS_OK;                                                                                         \
    }                                                                                                           \
    glls_status glls_prolong_add_##SUF(glls_problem* P, int level, const T* e, T* x, void* stream) {            \
        glls_status s = check_level(P, level, true);                                                            \
        if (s != GLLS_OK) return s;                                                                             \
        if (!e || !x) return fail(GLLS_ERR_INVALID, "null vector");                                             \
        DeviceScope scope(P->device);                                                                           \
        CK(scope.err);                                                                                          \
        prolong_add<T>(P, level, e, x, (cudaStream_t)stream);                                                   \
        CK(cudaGetLastError());                                                                                 \
        return GLLS_OK;                                                                                         \
    }                                                                                                           \
    glls_status glls_coarse_solve_##SUF(glls_problem* P, const T* r, T* e, void* stream) {                      \
        if (!P || !r || !e) return fail(GLLS_ERR_INVALID, "null argument");                                    \
        DeviceScope scope(P->device);                                                                           \
        CK(scope.err);                                                                                          \
        launch_coarse<T>(coarse_of<T>(P), levels_of<T>(P)[0].dev.N, r, e, levels_of<T>(P)[0].t1,               \
                         (cudaStream_t)stream);                                                                        \
        CK(cudaGetLastError());                                                                                 \
        return GLLS_OK;                                                                                         \
    }                                                                                                           \
    glls_status glls_precondition_##SUF(glls_problem* P, const glls_solve_opts* o, const T* r, T* z,            \
                                        void* stream) {                                                         \
        if (!P || !r || !z) return fail(GLLS_ERR_INVALID, "null argument");                                     \
        glls_status s = check_opts(o);                                                                          \
        if (s != GLLS_OK) return s;                                                                             \
        DeviceScope scope(P->device);                                                                           \
        CK(scope.err);                                                                                          \
        CK(cudaMemsetAsync(z, 0, sizeof(T) * levels_of<T>(P).back().dev.N, (cudaStream_t)stream));               \
        cycle<T>(P, (int)P->L64.size() - 1, r, z, o->gamma, o->m, (T)o->alpha, (cudaStream_t)stream);           \
        CK(cudaGetLastError());                                                                                 \
        return GLLS_OK;                                                                                         \
    }

LEVEL_OPS(f64, double)
LEVEL_OPS(f32, float)

}  // extern "C"

// ===========================================================================
// Restriction without any device allocation
// ===========================================================================
// Scratch for glls_restrict_noalloc_f32: the apply output y and two transfer
// temporaries, each kNoAllocMaxNodes floats (3 MiB in total).  Being a
// file-scope __device__ array it exists once on every device that loads the
// library, for the life of the process, and every call shares it.
namespace {

constexpr long long kNoAllocMaxNodes = 1LL << 18;
static __device__ __align__(256) float g_noalloc_scratch[3 * kNoAllocMaxNodes];

std::mutex g_noalloc_mutex;
float* g_noalloc_addr[128] = {nullptr};   // device address of the array, per device ordinal

// Host code must not use g_noalloc_scratch as a pointer: its host-side symbol
// is a stand-in, not a device address.  The device address is looked up once
// per device, with that device current.
glls_status noalloc_scratch(int device, float** out) {
    if (device < 0 || device >= 128) return fail(GLLS_ERR_INVALID, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return fail(GLLS_ERR_CUDA, std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") + cudaGetErrorString(e));
        g_noalloc_addr[device] = static_cast<float*>(p);
    }
    *out = g_noalloc_addr[device];
    return GLLS_OK;
}

}  // namespace

extern "C" glls_status glls_restrict_noalloc_f32(glls_problem* P, int level, const float* r, const float* x,
                                                 float* rc, void* stream) {
    glls_status s = check_level(P, level, true);
    if (s != GLLS_OK) return s;
    if (!r || !x || !rc) return fail(GLLS_ERR_INVALID, "null vector");
    const DevLevel<float>& F = P->L32[level].dev;
    const DevLevel<float>& C = P->L32[level - 1].dev;
    if (F.N > kNoAllocMaxNodes)
        return fail(GLLS_ERR_INVALID, "glls_restrict_noalloc_f32: level has " + std::to_string(F.N) +
                                          " nodes, more than the fixed scratch limit of " +
                                          std::to_string(kNoAllocMaxNodes));
    DeviceScope scope(P->device);
    CK(scope.err);
    float* base = nullptr;
    s = noalloc_scratch(P->device, &base);
    if (s != GLLS_OK) return s;
    float* y = base;
    float* t[2] = {base + kNoAllocMaxNodes, base + 2 * kNoAllocMaxNodes};
    cudaStream_t st = (cudaStream_t)stream;
    // y must start at zero: the apply sums element contributions into it
    CK(launch_apply<float>(F, x, y, true, st, false));
    int cur[3] = {F.n[0], F.n[1], F.n[2]};
    const float* in = r;
    const float* in2 = y;
    for (int a = 0; a < F.dim; ++a) {
        int nxt[3] = {cur[0], cur[1], cur[2]};
        nxt[a] = C.n[a];
        const bool last = a == F.dim - 1;
        float* out = last ? rc : t[a % 2];
        launch_transfer<float>(F.R[a], a, cur, nxt, in, in2, out, false, last, st);
        in = out;
        in2 = nullptr;
        for (int k = 0; k < 3; ++k) cur[k] = nxt[k];
    }
    CK(cudaGetLastError());
    return GLLS_OK;
}
