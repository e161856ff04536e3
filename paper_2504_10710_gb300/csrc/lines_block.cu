// Line smoothing with the Def. 3.2 line blocks R A_p P (GLL smoother,
// levels with p >= 2).
//
// A line's block couples every pair of its nodes that share an element, so it
// is the sum of (p+1) x (p+1) element-segment blocks overlapping at the
// element-boundary vertices.  The set-up (setup.cpp, line_blocks) condenses
// it: one step of Algorithm 1 with S = the block diagonal of the segment
// interiors K_I (Thm. 3.8: exact when S inverts those blocks exactly) leaves
// the Schur complement on the vertices (Prop. 3.7), which is tridiagonal and
// is solved by cyclic reduction (Cor. 3.9).  Per segment the set-up stores
// K_I^-1 (upper triangle) and w_L, w_R = K_I^-1 K_{I,v} for its two vertices;
// per line the vertex system.  One application of the block inverse to g:
//   z   = K_I^-1 g_I                          every segment
//   c_v = g_v - w_R(v-1) . g_I(v-1) - w_L(v) . g_I(v)     (c = R (g - K x))
//   S nu = c                                  vertex CR, one warp per line
//   x_I = z - w_L nu_left - w_R nu_right,  x_v = nu_v       (y = x + P e)
//
// A CTA owns LPC <= min(16, 256 / E) lines of one direction (E segments
// each) with LPC E threads (rounded up to a warp), one segment task per
// thread; small levels take fewer lines per CTA so that every SM gets work.  All
// global loads are issued at entry: the line values (coalesced: along the
// line for x-lines, across adjacent lines for strided directions), the
// vertex systems, and each thread's segment operator into registers; after
// one barrier the segment work, the vertex CR (one warp per line, warps
// taking a second line when LPC > 8) and the back substitution run in
// registers and shared memory, and the results are stored.  P is the
// compile-time order (2..8); P = 0 takes the order at run time, reads its
// operator from global memory inside the loops and accumulates K_I^-1 g_I in
// shared memory.
#include "async_copy.cuh"
#include "cr_warp.cuh"
#include "device.cuh"

#include <algorithm>
#include <cstddef>
#include <cstring>

namespace glls {
namespace {

template <typename T>
struct BlockLineArgs {
    int n, nlines, stride, m1, st1, st2, contiguous, mode;
    int p, E, span, cv, lpc;
    int nrhs;           // right-hand sides (vectors of N values each)
    long long N;
    long long ntask;
    T alpha;
    const T* blk;                              // [ncoef][ntask]
    const typename Vec2Of<T>::type* vband;     // [nlines][E - 1]
    const T* g;
    const T* r;
    T* y;
    T* x;
    const double* done;                        // work lists: the problem's stop flag, or null
};

constexpr int kBlockThreads = 256;
constexpr int kMaxLinesPerCta = 16;

// SMs of the current device (cached per process: one device type).
int sm_count() {
    static const int n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        return cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0 ? v : 152;
    }();
    return n;
}

// shared-memory index with one pad word per 32
__device__ __forceinline__ int padk(int k) { return k + (k >> 5); }



// Vertex system of one line (E - 1 unknowns; vertex k is line unknown
// (k + 1) p - 1), right-hand side c_k = g_v - dr[k] - dl[k + 1], operator
// from shared memory (vb: diagonal and coupling to the next vertex per
// vertex); the solution overwrites the vertex entries of `line`.
template <typename T, int C>
__device__ __forceinline__ void vertex_solve(T* line, const T* dl, const T* dr, const T* vb, int E, int p,
                                             int lane) {
    const int nv = E - 1;
    T a[C], l[C], u[C], g[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const int k = C * lane + j;
        if (k < nv) {
            a[j] = vb[2 * k];
            u[j] = k < nv - 1 ? vb[2 * k + 1] : T(0);
            l[j] = k > 0 ? vb[2 * k - 1] : T(0);
            g[j] = line[padk((k + 1) * p - 1)] - dr[k] - dl[k + 1];
        } else {
            a[j] = T(1); l[j] = T(0); u[j] = T(0); g[j] = T(0);
        }
    }
    warp_cr_solve<T, C>(a, l, u, g, lane);
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const int k = C * lane + j;
        if (k < nv) line[padk((k + 1) * p - 1)] = g[j];
    }
}

// Segment operator of one task in registers (compile-time order).
template <typename T, int P>
struct SegOp {
    static constexpr int MI = P > 1 ? P - 1 : 1;
    static constexpr int NPK = MI * (MI + 1) / 2;
    T t[NPK], wl[MI], wr[MI];
};

// MODE 0: x = B^-1 g.  MODE 1: x += alpha B^-1 (r - y), and y is reset to 0
// on element-boundary nodes (the apply that produced y plain-stores element-
// interior nodes and adds into element-boundary ones).  MODE 2: x += alpha
// B^-1 r.  MODE 3: x = alpha B^-1 r.
// Register budget: FP32 four CTAs per SM (<= 64 registers), three for order 8
// and the run-time order (<= 85: the 42 operator values of a segment stay in
// registers), FP64 two (<= 128).
// The CTA body for block `blk` of the launch of A (any block size of at
// least lpc E threads, rounded to whole warps).
template <typename T, int P, int CV>
__device__ __forceinline__ void line_block_body(BlockLineArgs<T> A, int blk) {
    // right-hand side fastest in the CTA order (see device.cuh): the nrhs CTAs
    // of one line group read the same segment operators
    const int rhs = blk % A.nrhs, bx = blk / A.nrhs;
    {
        const long long vo = (long long)rhs * A.N;
        if (A.g) A.g += vo;
        if (A.r) A.r += vo;
        if (A.y) A.y += vo;
        A.x += vo;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = A.n, E = A.E, span = A.span, mode = A.mode, LPC = A.lpc;
    const int p = P > 0 ? P : A.p;
    const int mi = p - 1, npk = mi * (mi + 1) / 2;
    const long long ntask = A.ntask;
    T* sg = reinterpret_cast<T*>(smem_raw);   // [LPC][span]: g, then z / nu, then B^-1 g
    T* sx = sg + LPC * span;                  // [LPC][span]: x on entry (MODE 1, 2)
    T* sy = sx + LPC * span;                  // [LPC][span]: y on entry (MODE 1)
    T* sdl = sy + LPC * span;                 // [LPC][E]: w_L . g_I per segment
    T* sdr = sdl + LPC * E;                   // [LPC][E]: w_R . g_I
    T* svb = sdr + LPC * E;                   // [LPC][2 (E - 1)]: vertex systems
    T* sz = svb + 2 * LPC * (E - 1);          // [LPC][span]: z accumulation (P = 0)
    // orders above 8 keep the segment operators in shared memory (too many
    // for registers): the run-time order, and compile-time orders 9..12
    constexpr bool SMOP = P == 0 || P > 8;
    T* sop = P == 0 ? sz + LPC * span : sz;   // [ncoef][blockDim]: segment operators (SMOP)
    const int l0 = bx * LPC;
    const int Wc = min(LPC, A.nlines - l0);
    const int tid = threadIdx.x;
    // first node of line w of this CTA (interior indices c1, c2 of the other axes)
    auto line_base = [&](int w) {
        const int li = l0 + w;
        return (li % A.m1 + 1) * A.st1 + (li / A.m1 + 1) * A.st2;
    };
    // this thread's segment task and its operator, loaded before anything waits
    const int ntk = Wc * E;
    const bool has_task = tid < ntk;
    const int tw = has_task ? tid / E : 0, te = has_task ? tid - tw * E : 0;
    const T* bp = A.blk + ((long long)(l0 + tw) * E + te);
    SegOp<T, SMOP ? 2 : P> op;            // registers (orders 2..8 only)
    if constexpr (P > 0 && !SMOP) {
        if (has_task) {
#pragma unroll
            for (int c = 0; c < SegOp<T, P>::NPK; ++c) op.t[c] = __ldg(bp + (long long)c * ntask);
#pragma unroll
            for (int i = 0; i < P - 1; ++i) {
                op.wl[i] = __ldg(bp + (long long)(npk + i) * ntask);
                op.wr[i] = __ldg(bp + (long long)(npk + mi + i) * ntask);
            }
        }
    }
    // operator rows are as long as this launch item's own thread count (a
    // work-list block may be larger; its extra threads have no segment)
    const int opstride = min(kBlockThreads, max(32, (LPC * E + 31) / 32 * 32));
    if constexpr (SMOP) {
        // the thread's segment operator is copied to shared memory with the
        // line values and read from there in the loops
        if (has_task) {
            const int ncoef = npk + 2 * mi;
            for (int c = 0; c < ncoef; ++c) cp_async(sop + c * opstride + tid, bp + (long long)c * ntask);
        }
    }
    auto opc = [&](int c) { return sop[c * opstride + tid]; };   // coefficient c of this thread's segment (SMOP)
    auto op_t = [&](int c) -> T {
        if constexpr (SMOP) return opc(c);
        else return op.t[c];
    };
    auto op_wl = [&](int i) -> T {
        if constexpr (SMOP) return opc(npk + i);
        else return op.wl[i];
    };
    auto op_wr = [&](int i) -> T {
        if constexpr (SMOP) return opc(npk + mi + i);
        else return op.wr[i];
    };

    // line values, staged without divisions by asynchronous copies (every
    // copy of the tile in flight at once): x-lines are walked along the line
    // by whole warps (coalesced along x); strided directions by threads that
    // each keep one line of the CTA and step over its rows, adjacent threads
    // on adjacent lines (coalesced across the lines)
    const bool contig = A.contiguous != 0;
    const int nthr = blockDim.x, nwarp = nthr >> 5;
    const int rows_per_pass = nthr / LPC;     // strided: rows covered per pass
    const int sw = contig ? 0 : tid % LPC, sk0 = contig ? 0 : tid / LPC;
    const bool s_active = !contig && sw < Wc && sk0 < rows_per_pass;
    const int s_base = s_active ? line_base(sw) : 0;
    auto stage = [&](int w, int k, int node) {
        const int o = w * span + padk(k);
        cp_async(sg + o, (mode == 0 ? A.g : A.r) + node);
        if (mode == 1) cp_async(sy + o, A.y + node);
        if (mode == 1 || mode == 2) cp_async(sx + o, A.x + node);
    };
    if (contig) {
        for (int w = tid >> 5; w < Wc; w += nwarp) {
            const int b = line_base(w);
#pragma unroll 2
            for (int k = tid & 31; k < n; k += 32) stage(w, k, b + (k + 1) * A.stride);
        }
    } else if (s_active) {
#pragma unroll 2
        for (int k = sk0; k < n; k += rows_per_pass) stage(sw, k, s_base + (k + 1) * A.stride);
    }
    // vertex systems of the CTA's lines (contiguous in global memory)
    if (E > 1) {
        const T* vsrc = reinterpret_cast<const T*>(A.vband + (long long)l0 * (E - 1));
        const int nvb = 2 * Wc * (E - 1);
        for (int i = tid; i < nvb; i += nthr) cp_async(svb + i, vsrc + i);
    }
    cp_async_wait_all();
    __syncthreads();
    if (mode == 1) {          // g = r - y (pad slots hold unused values)
        for (int i = tid; i < Wc * span; i += nthr) sg[i] -= sy[i];
        __syncthreads();
    }

    // ---- segments: z = K_I^-1 g_I and the two vertex dots
    T z[P > 1 ? P - 1 : 1];
    if (has_task) {
        T* line = sg + tw * span;
        const int base = te * p;   // line unknown of the segment's first interior node
        T dl = T(0), dr = T(0);
        if constexpr (P > 0) {
            T gi[P - 1];
#pragma unroll
            for (int i = 0; i < P - 1; ++i) {
                gi[i] = line[padk(base + i)];
                z[i] = T(0);
            }
            int c = 0;
#pragma unroll
            for (int i = 0; i < P - 1; ++i)
#pragma unroll
                for (int j = i; j < P - 1; ++j) {
                    const T t = op_t(c++);
                    z[i] += t * gi[j];
                    if (j != i) z[j] += t * gi[i];
                }
#pragma unroll
            for (int i = 0; i < P - 1; ++i) {
                dl += op_wl(i) * gi[i];
                dr += op_wr(i) * gi[i];
            }
        } else {
            T* zz = sz + tw * span;
            for (int i = 0; i < mi; ++i) zz[padk(base + i)] = T(0);
            int c = 0;
            for (int i = 0; i < mi; ++i) {
                const T gi_ = line[padk(base + i)];
                T zi = T(0);
                for (int j = i; j < mi; ++j) {
                    const T t = opc(c);
                    ++c;
                    zi += t * line[padk(base + j)];
                    if (j != i) zz[padk(base + j)] += t * gi_;
                }
                zz[padk(base + i)] += zi;
                dl += opc(npk + i) * gi_;
                dr += opc(npk + mi + i) * gi_;
            }
        }
        // each task reads and writes only its own segment's interior nodes
        if constexpr (P > 0) {
#pragma unroll
            for (int i = 0; i < P - 1; ++i) line[padk(base + i)] = z[i];
        } else {
            const T* zz = sz + tw * span;
            for (int i = 0; i < mi; ++i) line[padk(base + i)] = zz[padk(base + i)];
        }
        sdl[tw * E + te] = dl;
        sdr[tw * E + te] = dr;
    }
    __syncthreads();

    // ---- vertex systems, one warp per line
    const int warp = tid >> 5, lane = tid & 31;
    if (E > 1) {
        for (int w = warp; w < Wc; w += nwarp) {
            T* line = sg + w * span;
            const T* vb = svb + 2 * w * (E - 1);
            vertex_solve<T, CV>(line, sdl + w * E, sdr + w * E, vb, E, p, lane);
        }
    }
    __syncthreads();

    // ---- segments: x_I = z - w_L nu_left - w_R nu_right
    if (has_task) {
        T* line = sg + tw * span;
        const int base = te * p;
        const T nl = te > 0 ? line[padk(base - 1)] : T(0);
        const T nr = te < E - 1 ? line[padk(base + mi)] : T(0);
        if constexpr (P > 0) {
#pragma unroll
            for (int i = 0; i < P - 1; ++i) line[padk(base + i)] = z[i] - (op_wl(i) * nl + op_wr(i) * nr);
        } else {
            for (int i = 0; i < mi; ++i) {
                const T wl = opc(npk + i);
                const T wr = opc(npk + mi + i);
                line[padk(base + i)] -= wl * nl + wr * nr;
            }
        }
    }
    __syncthreads();

    // seam test: the line lies on an element boundary of another axis, or the
    // node is a vertex of the line
    auto put = [&](int w, int k, int base, bool line_seam) {
        const int node = base + (k + 1) * A.stride;
        const T v = sg[w * span + padk(k)];
        A.x[node] = mode == 0 ? v : (mode == 3 ? A.alpha * v : sx[w * span + padk(k)] + A.alpha * v);
        // the next apply stores element-interior nodes and adds into the
        // element-boundary ones: only those must be reset
        if (mode == 1 && (line_seam || (k + 1) % p == 0)) A.y[node] = T(0);
    };
    auto seam_of = [&](int w) {
        const int li = l0 + w;
        return ((li % A.m1 + 1) % p == 0) || (A.st2 != 0 && (li / A.m1 + 1) % p == 0);
    };
    if (contig) {
        for (int w = tid >> 5; w < Wc; w += nwarp) {
            const int b = line_base(w);
            const bool ls = seam_of(w);
#pragma unroll 2
            for (int k = tid & 31; k < n; k += 32) put(w, k, b, ls);
        }
    } else if (s_active) {
        const bool ls = seam_of(sw);
#pragma unroll 2
        for (int k = sk0; k < n; k += rows_per_pass) put(sw, k, s_base, ls);
    }
}

template <typename T, int P, int CV>
__global__ void __launch_bounds__(kBlockThreads, sizeof(T) == 8 ? 2 : (P >= 8 || P == 0 ? 3 : 4))
    line_block_kernel(BlockLineArgs<T> A) {
    grid_dep_sync();
    line_block_body<T, P, CV>(A, blockIdx.x);
}

// Work-list form: item j (one problem's level, direction and vectors) owns
// the CTAs [start[j], start[j + 1]).
template <typename T, int P, int CV>
__global__ void __launch_bounds__(kBlockThreads, sizeof(T) == 8 ? 2 : (P >= 8 || P == 0 ? 3 : 4))
    line_block_list_kernel(const BlockLineArgs<T>* __restrict__ items, const int* __restrict__ start, int nitems) {
    grid_dep_sync();
    const int j = work_item(start, nitems, blockIdx.x);
    if (items[j].done && *items[j].done != 0.0) return;
    line_block_body<T, P, CV>(items[j], blockIdx.x - start[j]);
}

template <typename T, int P>
size_t block_smem(int lpc, int span, int E) {
    return sizeof(T) * ((size_t)lpc * span * (P == 0 ? 4 : 3) + 2 * (size_t)lpc * E + 2 * (size_t)lpc * (E - 1));
}

// Shared memory of the run-time-order instance's segment operators for a
// block of `threads` threads at order p.
template <typename T>
size_t op_smem(int p, int threads) {
    const size_t mi = (size_t)(p - 1);
    return sizeof(T) * (mi * (mi + 1) / 2 + 2 * mi) * (size_t)threads;
}

// Orders 2..12 are compiled for vertex chunks of 1 and 2 per lane (lines of
// up to 65 elements); longer lines and other orders take the run-time order.
template <typename T, int P, int CV>
bool launch_pc(BlockLineArgs<T> A, cudaStream_t st) {
    // lines per CTA: at most 256 segment tasks and 16 lines; the autotuner's
    // choice for the level and direction when it has made one (A.lpc > 0),
    // else fewer while the level would have less than about four CTAs per SM
    // (small levels are latency bound: more, smaller CTAs run their phases
    // side by side)
    const int most = std::min(kMaxLinesPerCta, std::max(1, kBlockThreads / A.E));
    int lpc = most;
    if (A.lpc > 0) lpc = std::min(A.lpc, most);
    else
        while (lpc > 1 && (long long)(A.nlines + lpc - 1) / lpc * A.nrhs < 4 * sm_count()) lpc /= 2;
    auto thr = [&](int c) { return std::min(kBlockThreads, std::max(32, (c * A.E + 31) / 32 * 32)); };
    auto sm = [&](int c) {
        return block_smem<T, P>(c, A.span, A.E) + (P == 0 || P > 8 ? op_smem<T>(A.p, thr(c)) : 0);
    };
    while (lpc > 1 && sm(lpc) > kMaxDynSmemBytes) lpc /= 2;
    const size_t smem = sm(lpc);
    if (smem > kMaxDynSmemBytes) return false;
    A.lpc = lpc;
    const int threads = thr(lpc);
    const long long blocks = (long long)(A.nlines + lpc - 1) / lpc * A.nrhs;
    if (blocks > 0x7fffffffLL) return false;
    return launch_k(line_block_kernel<T, P, CV>, (unsigned)blocks, threads, smem, st, A) == cudaSuccess;
}

template <typename T, int P>
bool launch_p(BlockLineArgs<T> A, cudaStream_t st) {
    if constexpr (P > 0) {
        if (A.cv == 1) return launch_pc<T, P, 1>(A, st);
        if (A.cv == 2) return launch_pc<T, P, 2>(A, st);
        return launch_p<T, 0>(A, st);
    } else {
        switch (A.cv) {
            case 1: return launch_pc<T, 0, 1>(A, st);
            case 2: return launch_pc<T, 0, 2>(A, st);
            case 4: return launch_pc<T, 0, 4>(A, st);
            default: return launch_pc<T, 0, 8>(A, st);
        }
    }
}

template <typename T, int P>
bool set_attr_p() {
    const int lim = (int)kMaxDynSmemBytes;
    if constexpr (P > 0) {
        const void* fns[] = {(const void*)line_block_kernel<T, P, 1>, (const void*)line_block_kernel<T, P, 2>,
                             (const void*)line_block_list_kernel<T, P, 1>,
                             (const void*)line_block_list_kernel<T, P, 2>};
        for (const void* f : fns)
            if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess) return false;
        return true;
    } else {
        const void* fns[] = {(const void*)line_block_kernel<T, 0, 1>, (const void*)line_block_kernel<T, 0, 2>,
                             (const void*)line_block_kernel<T, 0, 4>, (const void*)line_block_kernel<T, 0, 8>,
                             (const void*)line_block_list_kernel<T, 0, 1>,
                             (const void*)line_block_list_kernel<T, 0, 2>,
                             (const void*)line_block_list_kernel<T, 0, 4>,
                             (const void*)line_block_list_kernel<T, 0, 8>};
        for (const void* f : fns)
            if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess) return false;
        return true;
    }
}

template <typename T>
bool set_attr_t() {
    return set_attr_p<T, 0>() && set_attr_p<T, 2>() && set_attr_p<T, 3>() && set_attr_p<T, 4>() &&
           set_attr_p<T, 5>() && set_attr_p<T, 6>() && set_attr_p<T, 7>() && set_attr_p<T, 8>() &&
           set_attr_p<T, 9>() && set_attr_p<T, 10>() && set_attr_p<T, 11>() && set_attr_p<T, 12>();
}

}  // namespace

bool init_line_block_attributes() { return set_attr_t<float>() && set_attr_t<double>(); }

bool line_block_supported(int n, int E) { return n <= kMaxBlockLine && E <= kMaxBlockSegments; }

namespace {

// Fills A for a line solve of L along s; 0: nothing to do, -1: outside the
// supported range, 1: ready.
template <typename T>
int make_args(BlockLineArgs<T>& A, const DevLevel<T>& L, int s, int mode, const T* g, const T* r, T* y, T* x,
              T alpha, int nrhs) {
    A.nrhs = nrhs;
    A.N = L.N;
    A.n = L.n[s] - 2;
    if (A.n <= 0) return 0;
    A.E = L.ne[s];
    if (!line_block_supported(A.n, A.E) || L.N > (1LL << 31) - 1) return -1;
    int o1, o2;
    if (s == 0) { o1 = 1; o2 = 2; } else if (s == 1) { o1 = 0; o2 = 2; } else { o1 = 0; o2 = 1; }
    const int strides[3] = {1, L.n[0], L.n[0] * L.n[1]};
    A.m1 = L.n[o1] - 2;
    const int m2 = L.dim == 3 ? L.n[o2] - 2 : 1;
    A.nlines = A.m1 * m2;
    if (A.nlines <= 0) return 0;
    A.ntask = (long long)A.nlines * A.E;
    A.stride = strides[s];
    A.st1 = strides[o1];
    A.st2 = L.dim == 3 ? strides[o2] : 0;
    A.contiguous = s == 0;
    A.mode = mode;
    A.p = L.p;
    A.span = (A.n - 1) + ((A.n - 1) >> 5) + 1;
    A.span = (A.span + 3) / 4 * 4;
    A.lpc = L.lbc[s];                  // 0: the launch heuristic
    const int nv = A.E - 1;
    A.cv = nv <= 32 ? 1 : (nv <= 64 ? 2 : (nv <= 128 ? 4 : 8));
    A.alpha = alpha;
    A.blk = L.blk[s];
    A.vband = L.vband[s];
    A.g = g;
    A.r = r;
    A.y = y;
    A.x = x;
    A.done = nullptr;
    return 1;
}

template <typename T, int P, int CV>
bool launch_list_pc(const void* items, const int* start, int nitems, int blocks, int threads, size_t smem,
                    cudaStream_t st) {
    return launch_k(line_block_list_kernel<T, P, CV>, (unsigned)blocks, threads, smem, st,
                    static_cast<const BlockLineArgs<T>*>(items), start, nitems) == cudaSuccess;
}

template <typename T, int P>
bool launch_list_p(int cv, const void* items, const int* start, int nitems, int blocks, int threads, size_t smem,
                   cudaStream_t st) {
    if constexpr (P > 0) {
        if (cv == 1) return launch_list_pc<T, P, 1>(items, start, nitems, blocks, threads, smem, st);
        if (cv == 2) return launch_list_pc<T, P, 2>(items, start, nitems, blocks, threads, smem, st);
        return launch_list_p<T, 0>(cv, items, start, nitems, blocks, threads, smem, st);
    } else {
        switch (cv) {
            case 1: return launch_list_pc<T, 0, 1>(items, start, nitems, blocks, threads, smem, st);
            case 2: return launch_list_pc<T, 0, 2>(items, start, nitems, blocks, threads, smem, st);
            case 4: return launch_list_pc<T, 0, 4>(items, start, nitems, blocks, threads, smem, st);
            default: return launch_list_pc<T, 0, 8>(items, start, nitems, blocks, threads, smem, st);
        }
    }
}

}  // namespace

template <typename T>
size_t line_block_item_bytes() {
    return sizeof(BlockLineArgs<T>);
}

template <typename T>
size_t line_block_item_done_offset() {
    return offsetof(BlockLineArgs<T>, done);
}

// One work-list item: the line solve of L along s (as launch_line_block,
// one right-hand side), written into `item` (line_block_item_bytes bytes);
// its CTA count, block size, vertex chunk (cv, 1..8) and dynamic shared
// memory for the order-specialised instance (smem[0]) and the run-time-order
// instance (smem[1]).  Lines per CTA as for a single launch, without the
// small-level split (a work-list launch has the CTAs of all its items).
// 0: nothing to do; -1: unsupported.
template <typename T>
int line_block_list_item(const DevLevel<T>& L, int s, int mode, const T* g, const T* r, T* y, T* x, T alpha,
                         void* item, int* blocks, int* threads, size_t smem[2], int* cv) {
    BlockLineArgs<T> A;
    const int k = make_args<T>(A, L, s, mode, g, r, y, x, alpha, 1);
    if (k <= 0) return k;
    // the run-time-order instance and orders 9..12 also hold the segment
    // operators of the item's own threads
    auto thr = [&](int c) { return std::min(kBlockThreads, std::max(32, (c * A.E + 31) / 32 * 32)); };
    auto sm1 = [&](int c) { return block_smem<T, 0>(c, A.span, A.E) + op_smem<T>(A.p, thr(c)); };
    int lpc = std::min(kMaxLinesPerCta, std::max(1, kBlockThreads / A.E));
    while (lpc > 1 && sm1(lpc) > kMaxDynSmemBytes) lpc /= 2;
    if (sm1(lpc) > kMaxDynSmemBytes) return -1;
    A.lpc = lpc;
    smem[0] = block_smem<T, 2>(lpc, A.span, A.E) + (A.p > 8 ? op_smem<T>(A.p, thr(lpc)) : 0);
    smem[1] = sm1(lpc);
    *threads = thr(lpc);
    *blocks = (A.nlines + lpc - 1) / lpc;
    *cv = A.cv;
    std::memcpy(item, &A, sizeof(A));
    return 1;
}

// Whether launch_line_block_list(p, cv, ...) runs the order-specialised
// instance (smem[0] of the items) or the run-time-order one (smem[1]).
bool line_block_list_specialised(int p, int cv) { return p >= 2 && p <= 12 && cv <= 2; }

// One launch over the items (all of order p; cv: the largest vertex chunk of
// the items).
template <typename T>
bool launch_line_block_list(int p, int cv, const void* items, const int* start, int nitems, int blocks, int threads,
                            size_t smem, cudaStream_t st) {
    if (nitems < 1 || blocks < 1) return true;
    switch (line_block_list_specialised(p, cv) ? p : 0) {
        case 2: return launch_list_p<T, 2>(cv, items, start, nitems, blocks, threads, smem, st);
        case 3: return launch_list_p<T, 3>(cv, items, start, nitems, blocks, threads, smem, st);
        case 4: return launch_list_p<T, 4>(cv, items, start, nitems, blocks, threads, smem, st);
        case 5: return launch_list_p<T, 5>(cv, items, start, nitems, blocks, threads, smem, st);
        case 6: return launch_list_p<T, 6>(cv, items, start, nitems, blocks, threads, smem, st);
        case 7: return launch_list_p<T, 7>(cv, items, start, nitems, blocks, threads, smem, st);
        case 8: return launch_list_p<T, 8>(cv, items, start, nitems, blocks, threads, smem, st);
        case 9: return launch_list_p<T, 9>(cv, items, start, nitems, blocks, threads, smem, st);
        case 10: return launch_list_p<T, 10>(cv, items, start, nitems, blocks, threads, smem, st);
        case 11: return launch_list_p<T, 11>(cv, items, start, nitems, blocks, threads, smem, st);
        case 12: return launch_list_p<T, 12>(cv, items, start, nitems, blocks, threads, smem, st);
        default: return launch_list_p<T, 0>(cv, items, start, nitems, blocks, threads, smem, st);
    }
}

template size_t line_block_item_bytes<float>();
template size_t line_block_item_bytes<double>();
template size_t line_block_item_done_offset<float>();
template size_t line_block_item_done_offset<double>();
template int line_block_list_item<float>(const DevLevel<float>&, int, int, const float*, const float*, float*, float*,
                                         float, void*, int*, int*, size_t*, int*);
template int line_block_list_item<double>(const DevLevel<double>&, int, int, const double*, const double*, double*,
                                          double*, double, void*, int*, int*, size_t*, int*);
template bool launch_line_block_list<float>(int, int, const void*, const int*, int, int, int, size_t, cudaStream_t);
template bool launch_line_block_list<double>(int, int, const void*, const int*, int, int, int, size_t, cudaStream_t);

template <typename T>
bool launch_line_block(const DevLevel<T>& L, int s, int mode, const T* g, const T* r, T* y, T* x, T alpha,
                       cudaStream_t st, int nrhs) {
    BlockLineArgs<T> A;
    const int k = make_args<T>(A, L, s, mode, g, r, y, x, alpha, nrhs);
    if (k <= 0) return k == 0;
    switch (L.p) {
        case 2: return launch_p<T, 2>(A, st);
        case 3: return launch_p<T, 3>(A, st);
        case 4: return launch_p<T, 4>(A, st);
        case 5: return launch_p<T, 5>(A, st);
        case 6: return launch_p<T, 6>(A, st);
        case 7: return launch_p<T, 7>(A, st);
        case 8: return launch_p<T, 8>(A, st);
        case 9: return launch_p<T, 9>(A, st);
        case 10: return launch_p<T, 10>(A, st);
        case 11: return launch_p<T, 11>(A, st);
        case 12: return launch_p<T, 12>(A, st);
        default: return launch_p<T, 0>(A, st);
    }
}

template bool launch_line_block<float>(const DevLevel<float>&, int, int, const float*, const float*, float*, float*,
                                       float, cudaStream_t, int);
template bool launch_line_block<double>(const DevLevel<double>&, int, int, const double*, const double*, double*,
                                        double*, double, cudaStream_t, int);

}  // namespace glls
