// Device-side data layout of the GLL p-multigrid solver and the host
// launchers of its kernels (kernels.cu).
//
// Layout in HBM, per level and precision T (double or float):
//   nodal vectors   : global grid, x fastest, N = n0*n1*n2 entries
//   G               : [ncomp][E * nloc] geometry factors, element-major, local
//                     node index q = (k*(p+1) + j)*(p+1) + i
//   diag, off[s]    : band-1 line-system coefficients on the global grid;
//                     off[s][node] couples node and node + e_s
//   blk[s], vband[s]: Def. 3.2 line blocks condensed per element segment
//                     (GLL smoother, p >= 2), see DevLevel
//   D               : (p+1)^2 derivative matrix, D[i*(p+1)+j] = pi_j'(xi_i)
//   P[a], R[a]      : fixed-width row bands of the 1-D transfer matrices
//
// Several right-hand sides (nrhs > 1 in the launchers): a vector argument
// holds nrhs consecutive copies of its level's grid, right-hand side j at
// offset j N.  Kernels that read level data (apply, line solves, transfers,
// coarsest solve) put the right-hand side fastest in their CTA order, so the
// nrhs CTAs that read one element, line or block tile run together and the
// tile comes from HBM about once per launch.  Per-right-hand-side partial
// sums, tickets and Krylov scalars follow one another (stride given where
// they are used).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <utility>

namespace glls {

// Programmatic dependent launch.  Kernels are launched with programmatic
// stream serialisation, so the CTAs of the next kernel in a stream (or graph)
// may be scheduled while the previous kernel drains.  Every kernel therefore
// starts with grid_dep_sync(): it waits until the preceding kernel has
// completed and its writes are visible, then lets the following kernel begin
// launching.  Because each kernel waits before it touches memory, ordering is
// transitive along the stream exactly as without the attribute.
__device__ __forceinline__ void grid_dep_sync() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// False when GLLS_PDL=0 is set in the environment (plain stream order).
bool pdl_enabled();

template <typename... K, typename... A>
inline cudaError_t launch_k(void (*kern)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

template <typename T>
struct DevBand {
    int rows = 0, cols = 0, width = 0;
    const int* start = nullptr;
    const T* coef = nullptr;
    // largest input span (max start + width - min start) of 32 / 8
    // consecutive rows: the shared-memory window of a fused transfer tile
    int span32 = 0, span8 = 0;
};

template <typename T>
struct Vec2Of;
template <>
struct Vec2Of<float> { using type = float2; };
template <>
struct Vec2Of<double> { using type = double2; };

template <typename T>
struct DevLevel {
    int dim = 2, p = 1, n1 = 2, nloc = 4, ncomp = 3;
    int ne[3] = {1, 1, 1};
    int n[3] = {1, 1, 1};
    long long N = 0, E = 0;
    const T* G = nullptr;
    const T* D = nullptr;
    const T* diag = nullptr;
    const T* off[3] = {nullptr, nullptr, nullptr};
    // (diag, off[s]) interleaved per direction: one 8/16-byte load per node
    const typename Vec2Of<T>::type* band[3] = {nullptr, nullptr, nullptr};
    DevBand<T> P[3], R[3];
    int lpb[3] = {4, 4, 4};   // band-1 line-solve tile (lines per CTA) per direction, set by the autotuner
    int lbc[3] = {0, 0, 0};   // line-block lines per CTA per direction, set by the autotuner (0: launch heuristic)
    int colored = 0;          // direct stiffness summation by element colours (bitwise reproducible; see launch_apply)
    // float-float form of G (finest FP64 level, 2-D 2 <= p <= 16, 3-D
    // 2 <= p <= 8; null elsewhere): Ghi = the FP32 level's G (the FP64 factors rounded to
    // nearest), Glo = their FP32 rounding remainders (apply_ff.cu)
    const float* Ghi = nullptr;
    const float* Glo = nullptr;
    // Def. 3.2 line blocks condensed per element segment (GLL smoother, p >= 2;
    // null otherwise): blk[s] [ncoef][nlines * ne[s]] = packed K_I^-1, w_L,
    // w_R per segment; vband[s] [nlines][ne[s] - 1] = vertex Schur complement
    // (diagonal, coupling to the next vertex).  See lines_block.cu.
    const T* blk[3] = {nullptr, nullptr, nullptr};
    const typename Vec2Of<T>::type* vband[3] = {nullptr, nullptr, nullptr};
};

// Exact coarsest solve: cr_levels levels of block cyclic reduction over the
// blocks of the slowest grid axis (Thm. 3.8 with m > 1, Cor. 3.9), then the
// dense inverse of the remaining system (cr_levels = 0: of the whole system).
// Unknowns are numbered lexicographically, so block b (0-based) holds unknowns
// b m .. b m + m - 1.  At level l (h = 2^l) the active blocks are
// b = (t + 1) h - 1, t = 0 .. (nb >> l) - 1; even t are eliminated, odd t kept.
constexpr int kMaxCrLevels = 16;
template <typename T>
struct DevCoarse {
    long long n = 0;                    // interior unknowns
    const long long* index = nullptr;   // interior node of each unknown
    long long nr = 0;                   // unknowns of the densely solved system
    long long ld = 0;                   // padded row length of inv (multiple of 16 bytes)
    const T* inv = nullptr;             // dense nr x nr inverse, row-major, leading dimension ld
    int nb = 1, m = 0, ldm = 0;         // blocks, block size, padded row length of the m x m blocks
    int cr_levels = 0;
    const T* fh[kMaxCrLevels] = {};     // level l: [kept][2][m][ldm]: L_i A_{i-h}^-1, U_i A_{i+h}^-1
    const T* agk[kMaxCrLevels] = {};    // level l: [elim][3][m][ldm]: A_j^-1, A_j^-1 L_j, A_j^-1 U_j
};

// ---- work lists: one launch over the tiles of several problems ----------
// Item j of a work-list launch owns the CTAs [start[j], start[j + 1]) of a
// one-dimensional grid (start has nitems + 1 entries, start[0] = 0); every
// item carries its own level data and vectors, so problems of different
// sizes share a launch; an item whose problem has stopped (done flag set)
// returns at once.  Returns the item of CTA b by bisection.
__device__ __forceinline__ int work_item(const int* __restrict__ start, int nitems, int b) {
    int lo = 0, hi = nitems - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename T>
struct ApplyItem {               // y (+)= A x on one problem's level; dot partials (FP64 outer apply) in part
    DevLevel<T> L;
    const T* x;
    T* y;
    double* part;
    const double* done;          // the problem's stop flag (nonzero: its CTAs return at once), or null
};

template <typename T>
struct Transfer2Item {           // both in-plane factors of a restriction or prolongation (transfer2_kernel)
    DevBand<T> M0, M1;
    int3 nin, nout;
    const T* in;
    const T* in2;
    T* out;
    T* clear;
    int gx, gy;                  // the item's tile grid (x: 32 outputs of axis 0, y: TY outputs of axis 1)
    const double* done;
};

template <typename T>
struct CoarseItem {              // dense part of the coarsest solve (coarse_kernel)
    long long n, ld;
    const long long* index;
    const T* inv;
    const T* src;
    const long long* src_index;
    int m, H;
    T* e;
    const double* done;
};

template <typename T>
struct BcrItem {                 // one block-CR level of one problem (bcr_forward/backward_kernel)
    const T* ops;                // fh[l] (forward) or agk[l] (backward)
    int nb, m, ldm;
    const long long* index;
    const T* src;                // forward: r; backward: w
    T* dst;                      // forward: w; backward: e
    int gx, rows;                // the item's CTA grid
    const double* done;
};

struct FcgItem {                 // one problem's outer Krylov vectors, partial sums and scalars
    double *x, *r, *p, *q, *z;
    float *r32, *z32;            // FP32 copies (mixed precision), else null
    long long n;
    double *prz, *pzq, *prr, *ppq;
    int npq;                     // partials of p.q (CTAs of the problem's FP64 apply)
    double* S;
    unsigned* ticket;
};

int apply_list_blocks(int p, long long E);
template <typename T>
bool launch_apply_list(int p, const ApplyItem<T>* items, const int* start, int nitems, int blocks, bool mask,
                       bool dot, cudaStream_t st);
// Float-float outer apply with p.(A p) partials (apply_ff.cu): the finest
// level of 2-D problems with 2 <= p <= 16 and of 3-D problems with
// 2 <= p <= 8 (false elsewhere).  y seams zero on entry.
bool apply_ff_supported(const DevLevel<double>& L);
int apply_ff_partials(const DevLevel<double>& L);   // dot partials (CTAs) per right-hand side
bool launch_apply_ff(const DevLevel<double>& L, const double* x, double* y, bool mask, double* part,
                     cudaStream_t st, int nrhs);
bool launch_apply_ff_list(int p, const ApplyItem<double>* items, const int* start, int nitems, int blocks, bool mask,
                          cudaStream_t st);
// The float-float apply serves solves with tol >= kFfMinTol: its rounding
// (about 2^-44 relative per contraction) parts the recurrence residual from
// the true one near 1e-13.
constexpr double kFfMinTol = 1e-12;
template <typename T>
bool transfer2_list_config(const DevBand<T>& M0, const DevBand<T>& M1, const int nout[3], int* gx, int* gy,
                           int* wb, int* ty, size_t* smem);
template <typename T>
bool launch_transfer2_list(int wb, int ty, const Transfer2Item<T>* items, const int* start, int nitems, int blocks,
                           size_t smem, bool add, bool mask, cudaStream_t st);
template <typename T>
void launch_coarse_list(const CoarseItem<T>* items, const int* start, int nitems, int blocks, size_t smem,
                        cudaStream_t st);
template <typename T>
void launch_bcr_list(bool forward, int l, const BcrItem<T>* items, const int* start, int nitems, int blocks,
                     size_t smem, cudaStream_t st);
// blocks: CTAs per item (<= kDotBlocks), the same for every item: each item's
// partial sums of r.z, z.q and r.r have that many entries
void launch_fcg_list(int step, const FcgItem* items, int nitems, int flexible, int blocks, cudaStream_t st);
template <typename T>
size_t line_block_item_bytes();
template <typename T>
size_t line_block_item_done_offset();
template <typename T>
int line_block_list_item(const DevLevel<T>& L, int s, int mode, const T* g, const T* r, T* y, T* x, T alpha,
                         void* item, int* blocks, int* threads, size_t smem[2], int* cv);
bool line_block_list_specialised(int p, int cv);
template <typename T>
bool launch_line_block_list(int p, int cv, const void* items, const int* start, int nitems, int blocks, int threads,
                            size_t smem, cudaStream_t st);

// Opt every kernel into up to 200 KB of dynamic shared memory (call once per
// device, outside stream capture).
bool init_kernel_attributes();
constexpr size_t kMaxDynSmemBytes = 200 * 1024;

// Specialised fast paths (apply.cu with apply_eo.cu and apply_col.cu for
// 3-D, lines.cu); they return false when the case is outside their compiled
// range and the generic kernels take over.
// dot: if non-null, also accumulate sum_e x_e^T (A_e x_e) = x.(A x) for x
// zero on the boundary; the last block writes it to dot[0] using `part` and
// `ticket` (see launch_dots).
template <typename T>
bool launch_apply_fixed(const DevLevel<T>& L, const T* x, T* y, bool mask, double* dot, double* part,
                        unsigned* ticket, cudaStream_t st, int nrhs = 1);
template <typename T>
bool launch_line_warp(const DevLevel<T>& L, int s, int mode, const T* g, const T* r, T* y, T* x, T alpha,
                      cudaStream_t st, int nrhs = 1);
bool init_line_warp_attributes();
// Line solves with the condensed Def. 3.2 line blocks (lines_block.cu), used
// whenever L.blk[s] is set; lines of at most kMaxBlockLine unknowns and
// kMaxBlockSegments elements (checked at set-up).  Returns false only outside
// that range or when the launch fails.
constexpr int kMaxBlockLine = 2047;
constexpr int kMaxBlockSegments = 256;
bool line_block_supported(int n, int E);
template <typename T>
bool launch_line_block(const DevLevel<T>& L, int s, int mode, const T* g, const T* r, T* y, T* x, T alpha,
                       cudaStream_t st, int nrhs = 1);
bool init_line_block_attributes();
// 3-D FP32 apply with one thread per element column (apply_col.cu), p <= 3
// (the orders the even-odd kernel does not take); no x.(A x) product.
// Returns false outside that range.
bool launch_apply_col(const DevLevel<float>& L, const float* x, float* y, bool mask, cudaStream_t st,
                      int nrhs = 1);
bool init_apply_col_attributes();
// 3-D apply with one thread per element grid line and even-odd derivative
// sweeps (apply_eo.cu), for the orders apply_eo_selected names, with the
// optional x.(A x) partials (one per CTA, apply_eo_blocks of them).
bool apply_eo_selected(int dim, int p, bool f64);
template <typename T>
bool launch_apply_eo(const DevLevel<T>& L, const T* x, T* y, bool mask, double* dot, double* part,
                     unsigned* ticket, cudaStream_t st, int nrhs = 1);
int apply_eo_blocks(int p, long long E);
bool init_apply_eo_attributes();

// ---- launchers (all asynchronous on `st`) ---------------------------------
// y = A x; mask: boundary rows of y are not written.  y_is_zero: the caller
// guarantees y == 0 on entry (otherwise it is zeroed first).  dot, part,
// ticket: optional x.(A x) into dot[0] (FP64 only).  Returns the status of
// the zeroing (cudaSuccess when y_is_zero); launch errors are left to
// cudaGetLastError.
template <typename T>
cudaError_t launch_apply(const DevLevel<T>& L, const T* x, T* y, bool mask, cudaStream_t st, bool y_is_zero = false,
                  double* dot = nullptr, double* part = nullptr, unsigned* ticket = nullptr, int nrhs = 1);

// Line solves along axis s.  mode 0: x = B_s^-1 g; mode 1: x += alpha
// B_s^-1 (r - y) and y is reset to 0 where read; mode 2: x += alpha B_s^-1 r;
// mode 3: x = alpha B_s^-1 r.  Only interior entries of x are written.
template <typename T>
void launch_line_solve(const DevLevel<T>& L, int s, int mode, const T* g, const T* r, T* y,
                       T* x, T alpha, cudaStream_t st, int nrhs = 1);

// One tensor-product factor of a transfer: out = M in (or in - in2) along
// axis a; grids nin/nout differ only along a.  add: out += ...; mask: zero
// the output's boundary nodes; clear (optional, output-grid sized): set to 0.
template <typename T>
void launch_transfer(const DevBand<T>& M, int a, const int nin[3], const int nout[3], const T* in,
                     const T* in2, T* out, bool add, bool mask, cudaStream_t st, T* clear = nullptr, int nrhs = 1);

// The first two tensor-product factors of a transfer in one launch: out =
// M1 (M0 (in - in2)) along axes 0 and 1, for every index of axis 2 (nin and
// nout differ along axes 0 and 1 only).  add / mask / clear as for
// launch_transfer (mask only when these are the last factors, i.e. in 2-D).
// Returns false when the tile window does not fit in shared memory (the
// caller then runs the two passes separately).
template <typename T>
bool launch_transfer2(const DevBand<T>& M0, const DevBand<T>& M1, const int nin[3], const int nout[3], const T* in,
                      const T* in2, T* out, bool add, bool mask, cudaStream_t st, T* clear = nullptr, int nrhs = 1);

// e = A_0^-1 r on the interior of the coarsest level; e's boundary entries
// are zeroed first unless e_boundary_zero.  w: scratch of C.n values (used
// when C.cr_levels > 0; must not alias r or e).
template <typename T>
void launch_coarse(const DevCoarse<T>& C, long long N0, const T* r, T* e, T* w, cudaStream_t st,
                   bool e_boundary_zero = false, int nrhs = 1);

// ---- vector kernels -------------------------------------------------------
template <typename Ti, typename To>
void launch_cast(const Ti* in, To* out, long long n, cudaStream_t st);
template <typename T>
void launch_zero_boundary(T* v, const int n[3], int dim, cudaStream_t st, int nrhs = 1);

// Deterministic dot products in one launch: partial sums per block into
// `part` (ndots * nblocks); the last block adds them in block order into
// S[slot0] (and S[slot1]).  `ticket` is a zero-initialised counter that the
// kernel resets.
constexpr int kDotBlocks = 304;   // 2 x 152 SMs
// CTAs per right-hand side of the outer-iteration kernels (dots, direction,
// update) for vectors of n values: about 16 values per thread, between 16
// and kDotBlocks (each CTA also sums all of the apply's partials, so more
// CTAs than the vector needs cost more than they hide)
inline int fcg_blocks(long long n) {
    const long long b = (n + 4095) / 4096;
    return (int)(b < 16 ? 16 : b > kDotBlocks ? kDotBlocks : b);
}
constexpr int kMaxReduceBlocks = 8192;
void launch_dots(const double* a0, const double* b0, const double* a1, const double* b1, int ndots,
                 long long n, double* part, double* S, int slot0, int slot1, unsigned* ticket, cudaStream_t st, int nrhs = 1);
// Outer-iteration dots without a grid-wide finish: kDotBlocks per-block
// partials of r.z into prz and of z.q into pzq; z is first taken from z32
// when given (z = double(z32)); q is reset to 0 after it is read.
void launch_dots_rz_zq(const double* r, double* z, const float* z32, double* q, long long n, double* prz, double* pzq,
                       cudaStream_t st, int nrhs = 1);

// Krylov scalar slots in the device array S.
// Per right-hand side j the slots sit at S + j * S_COUNT.  S_DONE: 0 while
// iterating, 1 converged, 2 broken down; S_ITS: iterations when it stopped.
enum Slot { S_RZ = 0, S_PQ, S_RR, S_RZNEW, S_ZQ, S_RR0, S_ALPHA, S_FLAG, S_TOL2, S_ITER, S_DONE, S_ITS, S_COUNT };

// q-independent update: p.q (npq partials from the apply) and r.z (nrz
// partials) are summed in every block, alpha = r.z / p.q; x += alpha p;
// r -= alpha q; r.r partials into prr; the last block writes S_RR, S_RZ,
// S_ALPHA, S_PQ and flags breakdown in S_FLAG.  r32 (optional): also
// r32 = float(r) for the FP32 gamma-cycle.
void launch_fcg_update(double* x, double* r, const double* p, const double* q, long long n, const double* ppq,
                       int npq, const double* prz, int nrz, double* prr, double* S, unsigned* ticket, float* r32,
                       cudaStream_t st, int nrhs = 1);
// p = z + beta p with beta = -S_ALPHA zq / S_RZ (flexible) or rz_new / S_RZ,
// rz_new and zq summed from the nd partials of launch_dots_rz_zq.
void launch_fcg_direction(double* p, const double* z, long long n, const double* prz, const double* pzq, int nd,
                          const double* S, int flexible, cudaStream_t st, int nrhs = 1);
// Dot partials launch_apply writes for L when asked for x.(A x) without a ticket.
template <typename T>
int apply_dot_partials(const DevLevel<T>& L);
// f0 = M f - y on interior nodes (0 on the boundary); v = g on the boundary, 0 inside.
void launch_lift_rhs(const double* mass, const double* f, const double* y, double* f0, const int n[3], int dim,
                     cudaStream_t st, int nrhs = 1);
void launch_boundary_only(const double* g, double* v, const int n[3], int dim, cudaStream_t st);
// y += a x; nrhs vectors of n values each, x the same for all when x_shared
void launch_axpy(double* y, const double* x, double a, long long n, cudaStream_t st, int nrhs = 1,
                 bool x_shared = false);
// GMRES: h[j] = V_j . w (j < k1, deterministic, part holds 64 k1 partials);
// w += sign sum_j h[j] V_j; out = in / sqrt(nrm2[0]).
void launch_multidot(const double* V, long long ld, int k1, const double* w, long long n, double* part, double* h,
                     unsigned* ticket, cudaStream_t st);
void launch_gs_update(double* w, const double* V, long long ld, int k1, const double* h, long long n, double sign,
                      cudaStream_t st);
void launch_scale_by_norm(double* out, const double* in, const double* nrm2, long long n, cudaStream_t st);

// Device-side solve loop: after S_RR0 is computed, initialise S and set the
// WHILE handle (r0 != 0); at the end of each iteration count it and set the
// handle to (r.r > tol^2 r0.r0, it < maxit, no breakdown).
// set_cond = false: update the scalars without setting the conditional
// (unrolled loops captured without a conditional node)
void launch_solve_init(double* S, cudaGraphConditionalHandle h, double tol, int maxit, cudaStream_t st, int nrhs = 1,
                       bool set_cond = true);
void launch_solve_cond(double* S, cudaGraphConditionalHandle h, int maxit, cudaStream_t st, int nrhs = 1,
                       bool set_cond = true);

}  // namespace glls
