// Line solves by cyclic reduction with one warp per grid line: the band-1
// line systems (Def. 3.1/3.2), and the vertex systems of the condensed line
// blocks (lines_block.cu) through the same warp_cr_solve (cr_warp.cuh).
//
// The band-1 system of a line is staged through shared memory with coalesced
// loads (adjacent lines of a CTA are adjacent in memory for strided
// directions), then each lane holds a contiguous chunk of C unknowns in
// registers and the warp runs cyclic reduction (cr_warp.cuh).  A line of n
// unknowns is padded to 32 C with decoupled identity rows.
#include "cr_warp.cuh"
#include "device.cuh"

namespace glls {
namespace {

template <typename T>
struct WarpLineArgs {
    int n, nlines, stride, m1, st1, st2, contiguous, mode;
    int p;              // element order: element-boundary nodes are multiples of p
    int nrhs;           // right-hand sides (vectors of N values each)
    long long N;
    T alpha;
    const typename Vec2Of<T>::type* band;   // (diag, off) per node
    const T* g;
    const T* r;
    T* y;
    T* x;
};

// shared-memory index with one pad word per 32: lane-chunk reads are conflict free
__device__ __forceinline__ int padi(int k) { return k + (k >> 5); }

// MODE 0: x = B^-1 g.  MODE 1: x += alpha B^-1 (r - y), and y is reset to 0
// on element-boundary nodes (the apply that produced y plain-stores element-
// interior nodes and adds into element-boundary ones, so its consumer
// restores the zeros the next apply needs).  MODE 2: x += alpha B^-1 r.
// MODE 3: x = alpha B^-1 r (first smoothing step from x = 0).
template <typename T, int C, int LPB, int MODE>
__global__ void __launch_bounds__(32 * LPB) line_warp_kernel(WarpLineArgs<T> A) {
    grid_dep_sync();
    // right-hand side fastest in the CTA order (see device.cuh)
    const int rhs = blockIdx.x % A.nrhs, bx = blockIdx.x / A.nrhs;
    {
        const long long off = (long long)rhs * A.N;
        if (A.g) A.g += off;
        if (A.r) A.r += off;
        if (A.y) A.y += off;
        A.x += off;
    }
    constexpr int SPAN = 32 * C + C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sd = reinterpret_cast<T*>(smem_raw);
    T* so = sd + LPB * SPAN;
    T* sg = so + LPB * SPAN;
    __shared__ int sbase[LPB];
    __shared__ int sseam[LPB];   // the whole line lies on element boundaries
    const int n = A.n;
    const int l0 = bx * LPB;
    const int Wc = min(LPB, A.nlines - l0);
    const int tid = threadIdx.x;
    if (tid < LPB) {
        const int li = l0 + tid;
        const int c1 = li % A.m1 + 1, c2 = li / A.m1 + 1;
        sbase[tid] = c1 * A.st1 + c2 * A.st2;
        sseam[tid] = (c1 % A.p == 0) || (A.st2 != 0 && c2 % A.p == 0);
    }
    __syncthreads();
    // staged loads: every thread has at most C elements per array, all issued
    // back to back.  x-lines: warp w reads line w; strided lines: the LPB
    // threads of a row group read LPB adjacent lines.
    const bool contig = A.contiguous != 0;
    const int lw = contig ? (tid >> 5) : (tid & (LPB - 1));
    const int lk = contig ? (tid & 31) : (tid / LPB);
    const int lnode = lw < Wc ? sbase[lw] : 0;
    const bool lseam = lw < Wc && sseam[lw] != 0;
    // x (MODE 1, 2) is read here with the band and the right-hand side, so the
    // update after the solve waits on no further global load
    T vd[C], vo[C], vg[C], out[C];
#pragma unroll
    for (int m = 0; m < C; ++m) {
        const int k = lk + 32 * m;
        vd[m] = T(1); vo[m] = T(0); vg[m] = T(0); out[m] = T(0);
        if (lw < Wc && k < n) {
            const int node = lnode + (k + 1) * A.stride;
            const auto b = __ldg(A.band + node);
            vd[m] = b.x;
            vo[m] = k < n - 1 ? b.y : T(0);
            if (MODE == 0) vg[m] = A.g[node];
            else if (MODE == 1) vg[m] = A.r[node] - A.y[node];
            else vg[m] = A.r[node];
            if (MODE == 1 || MODE == 2) out[m] = A.x[node];
        }
    }
#pragma unroll
    for (int m = 0; m < C; ++m) {
        const int k = lk + 32 * m;
        if (lw < Wc && k < n) {
            const int sidx = lw * SPAN + padi(k);
            sd[sidx] = vd[m];
            so[sidx] = vo[m];
            sg[sidx] = vg[m];
        }
    }
    __syncthreads();

    const int w = tid >> 5, lane = tid & 31;
    if (w < Wc) {
        T a[C], l[C], u[C], g[C];
        const int base = w * SPAN;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const int k = C * lane + j;
            if (k < n) {
                a[j] = sd[base + padi(k)];
                u[j] = so[base + padi(k)];
                g[j] = sg[base + padi(k)];
                l[j] = k > 0 ? so[base + padi(k - 1)] : T(0);
            } else {
                a[j] = T(1); u[j] = T(0); l[j] = T(0); g[j] = T(0);
            }
        }
        warp_cr_solve<T, C>(a, l, u, g, lane);
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const int k = C * lane + j;
            if (k < n) sg[base + padi(k)] = g[j];
        }
    }
    __syncthreads();
    // (k + 1) mod p along this thread's nodes k = lk + 32 m, stepped without division
    const int p = A.p, step = 32 % p;
    int rem = (lk + 1) % p;
#pragma unroll
    for (int m = 0; m < C; ++m) {
        const int k = lk + 32 * m;
        if (lw < Wc && k < n) {
            const T v = sg[lw * SPAN + padi(k)];
            A.x[lnode + (k + 1) * A.stride] = MODE == 0 ? v : (MODE == 3 ? A.alpha * v : out[m] + A.alpha * v);
            // the next apply stores element-interior nodes and adds into the
            // element-boundary ones: only those must be reset
            if (MODE == 1 && (lseam || rem == 0)) A.y[lnode + (k + 1) * A.stride] = T(0);
        }
        rem += step;
        if (rem >= p) rem -= p;
    }
}

// Lines per CTA (the tile the autotuner chooses among): 2, 4, 8, or 16 (FP32).
template <typename T, int C, int LPB>
void launch_lpb(const WarpLineArgs<T>& A, cudaStream_t st) {
    const size_t smem = sizeof(T) * 3 * LPB * (32 * C + C);
    const int blocks = (A.nlines + LPB - 1) / LPB * A.nrhs;
    switch (A.mode) {
        case 0: launch_k(line_warp_kernel<T, C, LPB, 0>, blocks, 32 * LPB, smem, st, A); break;
        case 1: launch_k(line_warp_kernel<T, C, LPB, 1>, blocks, 32 * LPB, smem, st, A); break;
        case 2: launch_k(line_warp_kernel<T, C, LPB, 2>, blocks, 32 * LPB, smem, st, A); break;
        default: launch_k(line_warp_kernel<T, C, LPB, 3>, blocks, 32 * LPB, smem, st, A); break;
    }
}

template <typename T, int C>
void launch_c(const WarpLineArgs<T>& A, int lpb, cudaStream_t st) {
    if (lpb == 16) {
        // 16 lines per CTA (512 threads): FP32 with at most 16 unknowns per
        // lane only (register and shared-memory budget); otherwise 8
        if constexpr (sizeof(T) == 4 && C <= 16) {
            launch_lpb<T, C, 16>(A, st);
            return;
        }
        lpb = 8;
    }
    if (lpb == 2) launch_lpb<T, C, 2>(A, st);
    else if (lpb == 8) launch_lpb<T, C, 8>(A, st);
    else launch_lpb<T, C, 4>(A, st);
}

template <typename T, int C, int LPB>
bool set_attr_lpb() {
    const int lim = 160 * 1024;
    return cudaFuncSetAttribute((const void*)line_warp_kernel<T, C, LPB, 0>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess &&
           cudaFuncSetAttribute((const void*)line_warp_kernel<T, C, LPB, 1>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess &&
           cudaFuncSetAttribute((const void*)line_warp_kernel<T, C, LPB, 2>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess &&
           cudaFuncSetAttribute((const void*)line_warp_kernel<T, C, LPB, 3>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
}

template <typename T, int C>
bool set_attr() {
    bool ok = set_attr_lpb<T, C, 2>() && set_attr_lpb<T, C, 4>() && set_attr_lpb<T, C, 8>();
    if constexpr (sizeof(T) == 4 && C <= 16) ok = ok && set_attr_lpb<T, C, 16>();
    return ok;
}

}  // namespace

bool init_line_warp_attributes() {
    bool ok = set_attr<float, 1>() && set_attr<float, 2>() && set_attr<float, 4>() && set_attr<float, 8>() &&
              set_attr<float, 16>() && set_attr<float, 32>();
    ok = ok && set_attr<double, 1>() && set_attr<double, 2>() && set_attr<double, 4>() && set_attr<double, 8>() &&
         set_attr<double, 16>();
    return ok;
}

template <typename T>
bool launch_line_warp(const DevLevel<T>& L, int s, int mode, const T* g, const T* r, T* y, T* x, T alpha,
                      cudaStream_t st, int nrhs) {
    WarpLineArgs<T> A;
    A.nrhs = nrhs;
    A.N = L.N;
    A.n = L.n[s] - 2;
    const int cmax = sizeof(T) == 4 ? 32 : 16;
    if (A.n > 32 * cmax || L.N > (1LL << 31) - 1) return false;
    if (A.n <= 0) return true;
    int o1, o2;
    if (s == 0) { o1 = 1; o2 = 2; } else if (s == 1) { o1 = 0; o2 = 2; } else { o1 = 0; o2 = 1; }
    const int strides[3] = {1, L.n[0], L.n[0] * L.n[1]};
    A.m1 = L.n[o1] - 2;
    const int m2 = L.dim == 3 ? L.n[o2] - 2 : 1;
    A.nlines = A.m1 * m2;
    if (A.nlines <= 0) return true;
    A.stride = strides[s];
    A.st1 = strides[o1];
    A.st2 = L.dim == 3 ? strides[o2] : 0;
    A.contiguous = s == 0;
    A.mode = mode;
    A.p = L.p;
    A.alpha = alpha;
    A.band = L.band[s];
    A.g = g;
    A.r = r;
    A.y = y;
    A.x = x;
    int C = 1;
    while (32 * C < A.n) C *= 2;
    const int lpb = L.lpb[s];
    switch (C) {
        case 1: launch_c<T, 1>(A, lpb, st); break;
        case 2: launch_c<T, 2>(A, lpb, st); break;
        case 4: launch_c<T, 4>(A, lpb, st); break;
        case 8: launch_c<T, 8>(A, lpb, st); break;
        case 16: launch_c<T, 16>(A, lpb, st); break;
        default:
            if constexpr (sizeof(T) == 4) { launch_c<T, 32>(A, lpb, st); break; }
            return false;
    }
    return true;
}

template bool launch_line_warp<float>(const DevLevel<float>&, int, int, const float*, const float*, float*,
                                      float*, float, cudaStream_t, int);
template bool launch_line_warp<double>(const DevLevel<double>&, int, int, const double*, const double*,
                                       double*, double*, double, cudaStream_t, int);

}  // namespace glls
