// sm_103a kernels of the GLL p-multigrid gamma-cycle solver.
//
//   apply_kernel     y = A_l x, eq. (discreteBilinear): per element, x is staged
//                    in shared memory, reference gradients by sum factorisation
//                    (one 1-D contraction with D per axis), the pointwise
//                    geometric factors G, then the transposed contractions;
//                    element-interior nodes are stored, shared nodes summed
//                    with atomics (direct stiffness summation).
//   line_kernel      B_s^-1 on every interior grid line along axis s: the band-1
//                    line system (Def. 3.1/3.2) staged in shared memory and
//                    solved in place by cyclic reduction written as the direct
//                    multigrid of Algorithm 1 / Thm. 3.8 / Cor. 3.9.
//   transfer_kernel  one axis of the tensor-product transfers P_l, R_l (Sec. 3.3).
//   coarse_kernel    dense inverse times vector: A_0^-1 r, or the inverse of the
//                    system left after block cyclic reduction.
//   bcr_*_kernel     block cyclic reduction of the coarsest level over grid
//                    lines / planes (Thm. 3.8 with m > 1, Cor. 3.9): forward
//                    elimination and back substitution, one launch per level.
//   dots / fcg_*     FP64 outer-Krylov vector operations with scalars kept in
//                    device memory, deterministic two-stage reductions.
#include "device.cuh"
#include "reduce.cuh"

#include <climits>
#include <cstdio>
#include <cstdlib>
#include <type_traits>

namespace glls {

namespace {

__device__ __forceinline__ bool on_boundary(long long g, const int n[3], int dim) {
    long long I = g % n[0];
    long long J = (g / n[0]) % n[1];
    if (I == 0 || I == n[0] - 1 || J == 0 || J == n[1] - 1) return true;
    if (dim == 3) {
        long long K = g / ((long long)n[0] * n[1]);
        if (K == 0 || K == n[2] - 1) return true;
    }
    return false;
}

// ---------------------------------------------------------------------------
// stiffness apply
// ---------------------------------------------------------------------------
// Element e of a launch: the e-th element in lexicographic order, or with
// colour >= 0 the e-th element (lexicographic within the colour) whose
// coordinate parities (ex & 1, ey & 1, ez & 1) are the bits of colour.
// Elements of one colour are at least two apart along some axis, so no two of
// them share a node.
template <int DIM>
__device__ __forceinline__ void element_coords(long long e, const int* ne, int colour, long long& ex, long long& ey,
                                               long long& ez) {
    if (colour < 0) {
        ex = e % ne[0];
        ey = (e / ne[0]) % ne[1];
        ez = DIM == 3 ? e / ((long long)ne[0] * ne[1]) : 0;
        return;
    }
    const int cx = colour & 1, cy = (colour >> 1) & 1, cz = (colour >> 2) & 1;
    const long long m0 = (ne[0] - cx + 1) / 2, m1 = (ne[1] - cy + 1) / 2;
    ex = 2 * (e % m0) + cx;
    ey = 2 * ((e / m0) % m1) + cy;
    ez = DIM == 3 ? 2 * (e / (m0 * m1)) + cz : 0;
}

// Elements of colour c (as above) on a grid of ne elements per axis.
inline long long colour_elements(const int* ne, int dim, int c) {
    long long n = 1;
    for (int a = 0; a < dim; ++a) n *= (ne[a] - ((c >> a) & 1) + 1) / 2;
    return n;
}

// y = A x over the elements of the launch.  colour < 0: all elements, seam
// nodes accumulated with atomics (their summation order follows the
// scheduling).  colour >= 0: the elements of one colour, seam nodes updated
// with a plain read-add-write (no other element of the launch touches them);
// the 2^dim colour launches in order 0, 1, ... add every seam node's
// contributions in a fixed order, so y is the same bits on every run.
template <typename T, int DIM>
__global__ void __launch_bounds__(256) apply_kernel(DevLevel<T> L, const T* __restrict__ x, T* __restrict__ y,
                                                    int mask, int epc, int nrhs, int colour, long long nelem) {
    grid_dep_sync();
    // right-hand side fastest in the CTA order (see device.cuh)
    const int rhs = blockIdx.x % nrhs;
    const long long bx = blockIdx.x / nrhs;
    x += (long long)rhs * L.N;
    y += (long long)rhs * L.N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sD = reinterpret_cast<T*>(smem_raw);
    const int n1 = L.n1, nloc = L.nloc, p = L.p;
    T* sx = sD + n1 * n1;
    T* sw = sx + epc * nloc;
    for (int t = threadIdx.x; t < n1 * n1; t += blockDim.x) sD[t] = L.D[t];
    const long long e0 = bx * epc;
    const int ecount = (int)min((long long)epc, nelem - e0);
    const int total = ecount * nloc;
    const long long EN = L.E * nloc;

    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int el = t / nloc, q = t - el * nloc;
        const int i = q % n1, j = (q / n1) % n1, k = DIM == 3 ? q / (n1 * n1) : 0;
        long long ex, ey, ez;
        element_coords<DIM>(e0 + el, L.ne, colour, ex, ey, ez);
        const long long g = ((ez * p + k) * L.n[1] + (ey * p + j)) * L.n[0] + (ex * p + i);
        sx[t] = x[g];
    }
    __syncthreads();

    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int el = t / nloc, q = t - el * nloc;
        const int i = q % n1, j = (q / n1) % n1, k = DIM == 3 ? q / (n1 * n1) : 0;
        const T* xe = sx + el * nloc;
        T gr[3] = {T(0), T(0), T(0)};
        // reference gradient: contraction with D along each axis
        for (int m = 0; m < n1; ++m) {
            gr[0] += sD[i * n1 + m] * xe[(k * n1 + j) * n1 + m];
            gr[1] += sD[j * n1 + m] * xe[(k * n1 + m) * n1 + i];
            if (DIM == 3) gr[2] += sD[k * n1 + m] * xe[(m * n1 + j) * n1 + i];
        }
        long long ex, ey, ez;
        element_coords<DIM>(e0 + el, L.ne, colour, ex, ey, ez);
        const long long gq = ((ez * L.ne[1] + ey) * L.ne[0] + ex) * nloc + q;   // geometry factors of the element
        if (DIM == 2) {
            const T g00 = L.G[gq], g01 = L.G[EN + gq], g11 = L.G[2 * EN + gq];
            sw[t] = g00 * gr[0] + g01 * gr[1];
            sw[epc * nloc + t] = g01 * gr[0] + g11 * gr[1];
        } else {
            const T g00 = L.G[gq], g01 = L.G[EN + gq], g02 = L.G[2 * EN + gq];
            const T g11 = L.G[3 * EN + gq], g12 = L.G[4 * EN + gq], g22 = L.G[5 * EN + gq];
            sw[t] = g00 * gr[0] + g01 * gr[1] + g02 * gr[2];
            sw[epc * nloc + t] = g01 * gr[0] + g11 * gr[1] + g12 * gr[2];
            sw[2 * epc * nloc + t] = g02 * gr[0] + g12 * gr[1] + g22 * gr[2];
        }
    }
    __syncthreads();

    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int el = t / nloc, q = t - el * nloc;
        const int i = q % n1, j = (q / n1) % n1, k = DIM == 3 ? q / (n1 * n1) : 0;
        const T* w0 = sw + el * nloc;
        const T* w1 = sw + epc * nloc + el * nloc;
        const T* w2 = sw + 2 * epc * nloc + el * nloc;
        T v = T(0);
        for (int m = 0; m < n1; ++m) {
            v += sD[m * n1 + i] * w0[(k * n1 + j) * n1 + m];
            v += sD[m * n1 + j] * w1[(k * n1 + m) * n1 + i];
            if (DIM == 3) v += sD[m * n1 + k] * w2[(m * n1 + j) * n1 + i];
        }
        long long ex, ey, ez;
        element_coords<DIM>(e0 + el, L.ne, colour, ex, ey, ez);
        const long long g = ((ez * p + k) * L.n[1] + (ey * p + j)) * L.n[0] + (ex * p + i);
        const bool inner = i > 0 && i < p && j > 0 && j < p && (DIM == 2 || (k > 0 && k < p));
        if (inner) {
            y[g] = v;
        } else {
            if (mask && on_boundary(g, L.n, DIM)) continue;
            if (colour < 0) atomicAdd(&y[g], v);
            else y[g] += v;
        }
    }
}

// ---------------------------------------------------------------------------
// line solves by cyclic reduction
// ---------------------------------------------------------------------------
template <typename T>
struct LineArgs {
    int n;              // unknowns per line
    long long nlines;
    int W;              // lines per CTA
    long long stride;   // node stride along the line
    int m1;             // interior extent of the faster other axis
    long long st1, st2; // node strides of the two other axes
    int contiguous;
    int mode;
    T alpha;
    const T* diag;
    const T* off;
    const T* g;
    const T* r;
    T* y;
    T* x;
};

template <typename T>
__global__ void __launch_bounds__(256) line_kernel(LineArgs<T> A) {
    grid_dep_sync();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = A.n;
    const long long l0 = (long long)blockIdx.x * A.W;
    const int Wc = (int)min((long long)A.W, A.nlines - l0);
    T* sa = reinterpret_cast<T*>(smem_raw);
    T* sl = sa + A.W * n;
    T* su = sl + A.W * n;
    T* sg = su + A.W * n;
    const int total = Wc * n;

    auto node_of = [&](int w, int kk) -> long long {
        const long long li = l0 + w;
        const long long c1 = li % A.m1 + 1, c2 = li / A.m1 + 1;
        return c1 * A.st1 + c2 * A.st2 + (long long)(kk + 1) * A.stride;
    };

    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        int w, kk;
        if (A.contiguous) { w = t / n; kk = t - w * n; } else { kk = t / Wc; w = t - kk * Wc; }
        const long long g = node_of(w, kk);
        const int s = w * n + kk;
        sa[s] = A.diag[g];
        su[s] = kk < n - 1 ? A.off[g] : T(0);
        sl[s] = kk > 0 ? A.off[g - A.stride] : T(0);
        if (A.mode == 0) {
            sg[s] = A.g[g];
        } else if (A.mode == 1) {
            sg[s] = A.r[g] - A.y[g];
            A.y[g] = T(0);
        } else {
            sg[s] = A.r[g];
        }
    }
    __syncthreads();

    // forward reduction: eliminate the odd multiples of h into the even ones
    int h = 1;
    while (n / h > 1) {
        const int cnt = n / (2 * h);
        for (int t = threadIdx.x; t < Wc * cnt; t += blockDim.x) {
            const int w = t / cnt, c = t - w * cnt;
            const int i = (c + 1) * 2 * h - 1;   // 0-based position of 1-based (c+1)*2h
            const int il = w * n + i - h, ic = w * n + i, ir = w * n + i + h;
            const T al = -sl[ic] / sa[il];
            T be = T(0), ur = T(0), lr = T(0), gr = T(0);
            if (i + h < n) { be = -su[ic] / sa[ir]; ur = su[ir]; lr = sl[ir]; gr = sg[ir]; }
            sa[ic] = sa[ic] + al * su[il] + be * lr;
            sg[ic] = sg[ic] + al * sg[il] + be * gr;
            sl[ic] = al * sl[il];
            su[ic] = be * ur;
        }
        __syncthreads();
        h *= 2;
    }
    for (int w = threadIdx.x; w < Wc; w += blockDim.x) sg[w * n + h - 1] = sg[w * n + h - 1] / sa[w * n + h - 1];
    __syncthreads();
    // back substitution: odd multiples of h from their solved neighbours
    for (h /= 2; h >= 1; h /= 2) {
        const int cnt = (n / h + 1) / 2;
        for (int t = threadIdx.x; t < Wc * cnt; t += blockDim.x) {
            const int w = t / cnt, c = t - w * cnt;
            const int i = (2 * c + 1) * h - 1;
            const int ic = w * n + i;
            const T xl = i - h >= 0 ? sg[ic - h] : T(0);
            const T xr = i + h < n ? sg[ic + h] : T(0);
            sg[ic] = (sg[ic] - sl[ic] * xl - su[ic] * xr) / sa[ic];
        }
        __syncthreads();
    }

    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        int w, kk;
        if (A.contiguous) { w = t / n; kk = t - w * n; } else { kk = t / Wc; w = t - kk * Wc; }
        const long long g = node_of(w, kk);
        const T v = sg[w * n + kk];
        if (A.mode == 0) A.x[g] = v;
        else if (A.mode == 3) A.x[g] = A.alpha * v;
        else A.x[g] += A.alpha * v;
    }
}

// ---------------------------------------------------------------------------
// transfers
// ---------------------------------------------------------------------------
// WB: compile-time bound on the band width, so that all loads of a row are
// issued back to back (WB = 0: runtime loop for very wide bands).
template <typename T, int WB>
__global__ void transfer_kernel(DevBand<T> M, int a, int3 nin, int3 nout, const T* __restrict__ in,
                                const T* __restrict__ in2, T* __restrict__ out, int add, int mask, int dim,
                                T* __restrict__ clear, int nrhs) {
    grid_dep_sync();
    const int total = nout.x * nout.y * nout.z;
    const long long tin = (long long)nin.x * nin.y * nin.z;
    const int sin_a = a == 0 ? 1 : (a == 1 ? nin.x : nin.x * nin.y);
    const int W = M.width;
    const long long all = (long long)total * nrhs;
    for (long long gidx = blockIdx.x * (long long)blockDim.x + threadIdx.x; gidx < all;
         gidx += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(gidx / total), idx = (int)(gidx - (long long)j * total);
        const T* in_j = in + j * tin;
        const T* in2_j = in2 ? in2 + j * tin : nullptr;
        T* out_j = out + (long long)j * total;
        if (clear) clear[gidx] = T(0);
        const int c0 = idx % nout.x, c1 = (idx / nout.x) % nout.y, c2 = idx / (nout.x * nout.y);
        if (mask) {
            const bool bnd = c0 == 0 || c0 == nout.x - 1 || c1 == 0 || c1 == nout.y - 1 ||
                             (dim == 3 && (c2 == 0 || c2 == nout.z - 1));
            if (bnd) { if (!add) out_j[idx] = T(0); continue; }
        }
        const int K = a == 0 ? c0 : (a == 1 ? c1 : c2);
        const int b0 = a == 0 ? 0 : c0, b1 = a == 1 ? 0 : c1, b2 = a == 2 ? 0 : c2;
        const int base = (b2 * nin.y + b1) * nin.x + b0 + M.start[K] * sin_a;
        const T* cf = M.coef + K * W;
        T v = T(0);
        if (WB > 0) {
            T cv[WB > 0 ? WB : 1], iv[WB > 0 ? WB : 1];
#pragma unroll
            for (int k = 0; k < (WB > 0 ? WB : 1); ++k) {
                cv[k] = T(0);
                iv[k] = T(0);
                if (k < W) {
                    cv[k] = cf[k];
                    iv[k] = in2_j ? in_j[base + k * sin_a] - in2_j[base + k * sin_a] : in_j[base + k * sin_a];
                }
            }
#pragma unroll
            for (int k = 0; k < (WB > 0 ? WB : 1); ++k) v += cv[k] * iv[k];
        } else {
            for (int k = 0; k < W; ++k)
                v += cf[k] * (in2_j ? in_j[base + k * sin_a] - in2_j[base + k * sin_a] : in_j[base + k * sin_a]);
        }
        out_j[idx] = add ? out_j[idx] + v : v;
    }
}

// ---------------------------------------------------------------------------
// coarsest solve: dense inverse times vector, one warp per row
// ---------------------------------------------------------------------------
// Position, in the block-ordered unknown numbering, of unknown t of the
// system left after k block-CR levels (H = 2^k): block (t / m + 1) H - 1.
__device__ __forceinline__ long long reduced_pos(long long t, int m, int H) {
    const long long b = t / m;
    return ((b + 1) * H - 1) * m + (t - b * m);
}

// Dense inverse times vector.  The input is gathered into shared memory:
// src[src_index[pos(t)]] (nodal source) or src[pos(t)] (block-ordered
// source); row i of the result goes to e[index[pos(i)]].
template <typename T>
__device__ __forceinline__ void coarse_body(long long n, long long ld, const long long* __restrict__ index,
                                            const T* __restrict__ inv, const T* __restrict__ src,
                                            const long long* __restrict__ src_index, int m, int H, T* __restrict__ e,
                                            int nrhs, long long vstride, int blk, int nblk) {
    // right-hand side fastest in the CTA order (see device.cuh); src and e
    // hold vstride values per right-hand side
    const int rhs = blk % nrhs;
    const long long bx = blk / nrhs, nbx = nblk / nrhs;
    src += rhs * vstride;
    e += rhs * vstride;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* rs = reinterpret_cast<T*>(smem_raw);
    for (long long t = threadIdx.x; t < ld; t += blockDim.x) {
        T v = T(0);
        if (t < n) {
            const long long q = reduced_pos(t, m, H);
            v = src_index ? src[src_index[q]] : src[q];
        }
        rs[t] = v;
    }
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int wpb = blockDim.x / 32;
    constexpr int V = 16 / sizeof(T);   // elements per 16-byte vector
    using Vec = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    // each lane keeps U row chunks in flight (independent loads and partial
    // sums), so a row costs about one memory latency instead of one per chunk
    constexpr int U = sizeof(T) == 4 ? 16 : 8;
    const long long nvec = ld / V;
    for (long long row = bx * wpb + warp; row < n; row += nbx * wpb) {
        const long long out = lane == 0 ? index[reduced_pos(row, m, H)] : 0;   // in flight with the row
        const Vec* a = reinterpret_cast<const Vec*>(inv + row * ld);
        T part[U];
#pragma unroll
        for (int u = 0; u < U; ++u) part[u] = T(0);
        for (long long j0 = lane; j0 < nvec; j0 += 32 * U) {
            Vec v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long j = j0 + 32LL * u;
                if (j < nvec) v[u] = __ldg(a + j);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long j = j0 + 32LL * u;
                if (j < nvec) {
                    const T* vv = reinterpret_cast<const T*>(&v[u]);
#pragma unroll
                    for (int q = 0; q < V; ++q) part[u] += vv[q] * rs[j * V + q];
                }
            }
        }
        T s = T(0);
#pragma unroll
        for (int u = 0; u < U; ++u) s += part[u];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) e[out] = s;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) coarse_kernel(long long n, long long ld, const long long* __restrict__ index,
                                                     const T* __restrict__ inv, const T* __restrict__ src,
                                                     const long long* __restrict__ src_index, int m, int H,
                                                     T* __restrict__ e, int nrhs, long long vstride) {
    grid_dep_sync();
    coarse_body<T>(n, ld, index, inv, src, src_index, m, H, e, nrhs, vstride, blockIdx.x, gridDim.x);
}

template <typename T>
__global__ void __launch_bounds__(256) coarse_list_kernel(const CoarseItem<T>* __restrict__ items,
                                                          const int* __restrict__ start, int nitems) {
    grid_dep_sync();
    const int j = work_item(start, nitems, blockIdx.x);
    const CoarseItem<T>& it = items[j];
    if (it.done && *it.done != 0.0) return;
    coarse_body<T>(it.n, it.ld, it.index, it.inv, it.src, it.src_index, it.m, it.H, it.e, 1, 0,
                   blockIdx.x - start[j], start[j + 1] - start[j]);
}

// Rows of a block per CTA in the block-CR kernels: one per warp, so that a
// level with few blocks still spreads over many CTAs.
constexpr int kBcrRows = 8;

// Block CR forward step at level l (h = 2^l), one CTA per (kept block,
// kBcrRows rows): for kept block b = (2q + 2) h - 1,
//   w_b = src_b - (L_b A_{b-h}^-1) w_{b-h} - (U_b A_{b+h}^-1) w_{b+h}
// (the c = R (g - M x) step of Algorithm 1 with x = S^-1 g).  At level 0 the
// source is the nodal right-hand side r gathered through index, and CTAs
// past the kept blocks copy the eliminated blocks into w; deeper levels
// update w in place (they read only blocks eliminated at this level).
template <typename T>
__device__ __forceinline__ void bcr_forward_body(const T* __restrict__ FH, int l, int nb, int m, int ldm,
                                                 const long long* __restrict__ index, const T* __restrict__ r, T* w,
                                                 int nrhs, long long nvec, int bx, int by) {
    const int rhs = bx % nrhs;
    r += rhs * nvec;
    w += rhs * nvec;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* xl = reinterpret_cast<T*>(smem_raw);
    T* xr = xl + m;
    const int h = 1 << l, nk = (nb >> l) / 2;
    const int row0 = by * kBcrRows;
    const bool lvl0 = l == 0;
    const int q = bx / nrhs;
    if (q >= nk) {                                   // level 0: copy eliminated block 2 (q - nk)
        const long long b = 2LL * (q - nk);
        for (int rr = threadIdx.x; rr < kBcrRows; rr += blockDim.x) {
            const int row = row0 + rr;
            if (row < m) w[b * m + row] = r[index[b * m + row]];
        }
        return;
    }
    const long long b = (2LL * q + 2) * h - 1, lb = b - h, rb = b + h;
    const bool right = rb < nb;
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
        xl[c] = lvl0 ? r[index[lb * m + c]] : w[lb * m + c];
        xr[c] = right ? (lvl0 ? r[index[rb * m + c]] : w[rb * m + c]) : T(0);
    }
    __syncthreads();
    const T* F = FH + (size_t)q * 2 * m * ldm;
    const T* Hm = F + (size_t)m * ldm;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int rr = warp; rr < kBcrRows; rr += 8) {
        const int row = row0 + rr;
        if (row >= m) break;
        T s = T(0);
        for (int c = lane; c < m; c += 32) s += F[(size_t)row * ldm + c] * xl[c] + Hm[(size_t)row * ldm + c] * xr[c];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const long long o = b * m + row;
            w[o] = (lvl0 ? r[index[o]] : w[o]) - s;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) bcr_forward_kernel(const T* __restrict__ FH, int l, int nb, int m, int ldm,
                                                          const long long* __restrict__ index,
                                                          const T* __restrict__ r, T* w, int nrhs, long long nvec) {
    grid_dep_sync();
    bcr_forward_body<T>(FH, l, nb, m, ldm, index, r, w, nrhs, nvec, blockIdx.x, blockIdx.y);
}

// Block CR back substitution at level l, one CTA per (eliminated block,
// kBcrRows rows): for b = (2s + 1) h - 1,
//   x_b = A_b^-1 w_b - (A_b^-1 L_b) x_{b-h} - (A_b^-1 U_b) x_{b+h}
// (y = x + P e of Algorithm 1); the kept neighbours' values are already in
// e (solved at deeper levels), read and written through index.
template <typename T>
__device__ __forceinline__ void bcr_backward_body(const T* __restrict__ AGK, int l, int nb, int m, int ldm,
                                                  const long long* __restrict__ index, const T* __restrict__ w, T* e,
                                                  int nrhs, long long nvec, int bx, int by) {
    const int rhs = bx % nrhs;
    w += rhs * nvec;
    e += rhs * nvec;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* xw = reinterpret_cast<T*>(smem_raw);
    T* xl = xw + m;
    T* xr = xl + m;
    const int h = 1 << l;
    const int row0 = by * kBcrRows;
    const long long s_ = bx / nrhs;
    const long long b = (2 * s_ + 1) * h - 1, lb = b - h, rb = b + h;
    const bool left = lb >= 0, right = rb < nb;
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
        xw[c] = w[b * m + c];
        xl[c] = left ? e[index[lb * m + c]] : T(0);
        xr[c] = right ? e[index[rb * m + c]] : T(0);
    }
    __syncthreads();
    const T* Ai = AGK + (size_t)s_ * 3 * m * ldm;
    const T* G = Ai + (size_t)m * ldm;
    const T* K = G + (size_t)m * ldm;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int rr = warp; rr < kBcrRows; rr += 8) {
        const int row = row0 + rr;
        if (row >= m) break;
        T v = T(0);
        for (int c = lane; c < m; c += 32) {
            const size_t o = (size_t)row * ldm + c;
            v += Ai[o] * xw[c] - G[o] * xl[c] - K[o] * xr[c];
        }
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) e[index[b * m + row]] = v;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) bcr_backward_kernel(const T* __restrict__ AGK, int l, int nb, int m, int ldm,
                                                           const long long* __restrict__ index,
                                                           const T* __restrict__ w, T* e, int nrhs, long long nvec) {
    grid_dep_sync();
    bcr_backward_body<T>(AGK, l, nb, m, ldm, index, w, e, nrhs, nvec, blockIdx.x, blockIdx.y);
}

// Work-list forms of both block-CR steps: item j owns the CTAs [start[j],
// start[j + 1]) (its gx x rows grid, x fastest).
template <typename T>
__global__ void __launch_bounds__(256) bcr_list_kernel(const BcrItem<T>* __restrict__ items,
                                                       const int* __restrict__ start, int nitems, int l, int forward) {
    grid_dep_sync();
    const int j = work_item(start, nitems, blockIdx.x);
    const BcrItem<T>& it = items[j];
    if (it.done && *it.done != 0.0) return;
    const int local = blockIdx.x - start[j];
    const int bx = local % it.gx, by = local / it.gx;
    if (forward)
        bcr_forward_body<T>(it.ops, l, it.nb, it.m, it.ldm, it.index, it.src, it.dst, 1, 0, bx, by);
    else
        bcr_backward_body<T>(it.ops, l, it.nb, it.m, it.ldm, it.index, it.src, it.dst, 1, 0, bx, by);
}

// Fused two-factor transfer: a CTA of 32 x 8 threads computes a 32 x TY tile
// of outputs (I, J) of one axis-2 plane.  Its input window (rows of axis 1 x
// columns of axis 0 that the tile's bands touch) is staged in shared memory
// as in - in2, contracted along axis 0 into t (window rows x 32), then along
// axis 1:  out(I, J) = sum_k M1(J, k) sum_q M0(I, q) in(q, s1(J) + k).
// Band rows are held in registers (width bucket WB >= both widths).
template <typename T, int WB, int TY>
__device__ __forceinline__ void transfer2_body(const DevBand<T>& M0, const DevBand<T>& M1, int3 nin, int3 nout,
                                               const T* __restrict__ in, const T* __restrict__ in2,
                                               T* __restrict__ out, int add, int mask, T* __restrict__ clear, int bx,
                                               int by, int z) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int win[4];                       // column lo, column count, row lo, row count
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int I0 = bx * 32, J0 = by * TY;
    const int W0 = M0.width, W1 = M1.width;
    const int I = I0 + tx;
    const bool okI = I < nout.x;
    const int s0 = okI ? M0.start[I] : 0;
    T c0[WB];
#pragma unroll
    for (int k = 0; k < WB; ++k) c0[k] = okI && k < W0 ? M0.coef[(size_t)I * W0 + k] : T(0);
    if (ty == 0) {
        int lo = okI ? s0 : INT_MAX, hi = okI ? s0 + W0 : INT_MIN;
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        const int J = J0 + tx;
        const bool okJ = tx < TY && J < nout.y;
        const int s1 = okJ ? M1.start[J] : 0;
        int rlo = okJ ? s1 : INT_MAX, rhi = okJ ? s1 + W1 : INT_MIN;
        for (int o = 16; o > 0; o >>= 1) {
            rlo = min(rlo, __shfl_xor_sync(0xffffffffu, rlo, o));
            rhi = max(rhi, __shfl_xor_sync(0xffffffffu, rhi, o));
        }
        if (tx == 0) {
            win[0] = lo;
            win[1] = hi - lo;
            win[2] = rlo;
            win[3] = rhi - rlo;
        }
    }
    __syncthreads();
    const int clo = win[0], ncol = win[1], rlo = win[2], nrow = win[3];
    T* sin = reinterpret_cast<T*>(smem_raw);      // nrow x ncol
    T* st = sin + (size_t)M1.span8 * M0.span32;   // nrow x 32
    const size_t pin = (size_t)nin.x * nin.y, pout = (size_t)nout.x * nout.y;
    const T* inz = in + z * pin;
    const T* in2z = in2 ? in2 + z * pin : nullptr;
    // staged in rounds of U loads per thread, all issued before any is used
    constexpr int U = 4;
    const int total = nrow * ncol;
    for (int base = threadIdx.x; base < total; base += 256 * U) {
        T a[U], b[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + 256 * u;
            a[u] = T(0);
            b[u] = T(0);
            if (idx < total) {
                const int r = idx / ncol, c = idx - r * ncol;
                const size_t g = (size_t)(rlo + r) * nin.x + clo + c;
                a[u] = inz[g];
                if (in2z) b[u] = in2z[g];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + 256 * u;
            if (idx < total) sin[idx] = a[u] - b[u];
        }
    }
    __syncthreads();
    // lanes past the last output column read column 0 of the window (their
    // coefficients are zero), never outside it
    const int coff = okI ? s0 - clo : 0;
    for (int r = ty; r < nrow; r += 8) {
        const T* row = sin + (size_t)r * ncol + coff;
        T v = T(0);
#pragma unroll
        for (int k = 0; k < WB; ++k)
            if (k < W0) v += c0[k] * row[k];
        st[r * 32 + tx] = v;
    }
    __syncthreads();
    if (!okI) return;
    for (int jj = ty; jj < TY; jj += 8) {
        const int J = J0 + jj;
        if (J >= nout.y) break;
        const size_t o = z * pout + (size_t)J * nout.x + I;
        if (clear) clear[o] = T(0);
        if (mask && (I == 0 || I == nout.x - 1 || J == 0 || J == nout.y - 1)) {
            if (!add) out[o] = T(0);
            continue;
        }
        const int s1 = M1.start[J];
        const T* c1 = M1.coef + (size_t)J * W1;
        const T* col = st + (s1 - rlo) * 32 + tx;
        T cv[WB];
#pragma unroll
        for (int k = 0; k < WB; ++k) cv[k] = k < W1 ? c1[k] : T(0);
        T v = T(0);
#pragma unroll
        for (int k = 0; k < WB; ++k)
            if (k < W1) v += cv[k] * col[k * 32];
        out[o] = add ? out[o] + v : v;
    }
}

template <typename T, int WB, int TY>
__global__ void __launch_bounds__(256) transfer2_kernel(DevBand<T> M0, DevBand<T> M1, int3 nin, int3 nout,
                                                        const T* __restrict__ in, const T* __restrict__ in2,
                                                        T* __restrict__ out, int add, int mask, T* __restrict__ clear) {
    grid_dep_sync();
    transfer2_body<T, WB, TY>(M0, M1, nin, nout, in, in2, out, add, mask, clear, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Work-list form: item j owns the CTAs [start[j], start[j + 1]), its
// gx x gy x (planes) tile grid, x fastest.
template <typename T, int WB, int TY>
__global__ void __launch_bounds__(256) transfer2_list_kernel(const Transfer2Item<T>* __restrict__ items,
                                                             const int* __restrict__ start, int nitems, int add,
                                                             int mask) {
    grid_dep_sync();
    const int j = work_item(start, nitems, blockIdx.x);
    const Transfer2Item<T>& it = items[j];
    if (it.done && *it.done != 0.0) return;
    const int local = blockIdx.x - start[j];
    const int bx = local % it.gx, rest = local / it.gx;
    transfer2_body<T, WB, TY>(it.M0, it.M1, it.nin, it.nout, it.in, it.in2, it.out, add, mask, it.clear, bx,
                              rest % it.gy, rest / it.gy);
}

// ---------------------------------------------------------------------------
// vector kernels
// ---------------------------------------------------------------------------
template <typename Ti, typename To>
__global__ void cast_kernel(const Ti* __restrict__ in, To* __restrict__ out, long long n) {
    grid_dep_sync();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = static_cast<To>(in[i]);
}

template <typename T>
__global__ void zero_boundary_kernel(T* v, int3 n, int dim, int nrhs) {
    grid_dep_sync();
    const long long total = (long long)n.x * n.y * n.z;
    const int nn[3] = {n.x, n.y, n.z};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total * nrhs;
         i += (long long)gridDim.x * blockDim.x)
        if (on_boundary(i % total, nn, dim)) v[i] = T(0);
}

__global__ void __launch_bounds__(256) dots_kernel(const double* __restrict__ a0, const double* __restrict__ b0,
                                                   const double* __restrict__ a1, const double* __restrict__ b1,
                                                   int ndots, long long n, double* part, double* S, int slot0,
                                                   int slot1, unsigned* ticket, int rotate) {
    grid_dep_sync();
    // right-hand side blockIdx.y: vectors at j n, partials at j ndots
    // gridDim.x, scalars at j S_COUNT, ticket j
    const long long j = blockIdx.y;
    a0 += j * n;
    b0 += j * n;
    if (ndots > 1) {
        a1 += j * n;
        b1 += j * n;
    }
    part += j * ndots * gridDim.x;
    S += j * S_COUNT;
    if (ticket) ticket += j;
    __shared__ double red[32];
    double s0 = 0.0, s1 = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        s0 += a0[i] * b0[i];
        if (ndots > 1) s1 += a1[i] * b1[i];
    }
    double t0 = block_sum(s0, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t0;
    if (ndots > 1) {
        double t1 = block_sum(s1, red);
        if (threadIdx.x == 0) part[gridDim.x + blockIdx.x] = t1;
    }
    if (ticket && last_block(ticket)) {
        finalize_partials(part, ndots, gridDim.x, S, slot0, slot1, red);
        if (threadIdx.x == 0) {
            if (rotate) S[S_RZ] = S[S_RZNEW];
            *ticket = 0u;
        }
    }
}

// Elements per thread per trip of the FCG vector kernels' grid-stride loops.
constexpr int kVecU = 4;

// Sum of n partials in a fixed order (every block gets the same value);
// valid in thread 0.
__device__ __forceinline__ double sum_partials(const double* part, int n, double* red) {
    double s = 0.0;
    int i = threadIdx.x;
    const int b = blockDim.x;
    for (; i + 3 * b < n; i += 4 * b) {      // four loads in flight, added in the same order
        const double a0 = __ldcg(part + i), a1 = __ldcg(part + i + b), a2 = __ldcg(part + i + 2 * b),
                     a3 = __ldcg(part + i + 3 * b);
        s += a0;
        s += a1;
        s += a2;
        s += a3;
    }
    for (; i < n; i += b) s += __ldcg(part + i);
    return block_sum(s, red);
}

// Outer-iteration dots, grid-stride over kDotBlocks CTAs: per-block partials
// of r.z into prz and of z.q into pzq (summed by the consumers); z is taken
// from z32 when given (z = double(z32)); q is reset to 0 after it is read.
__device__ __forceinline__ void dots_rz_zq_body(const double* __restrict__ r, double* __restrict__ z,
                                                const float* __restrict__ z32, double* __restrict__ q, long long n,
                                                double* __restrict__ prz, double* __restrict__ pzq) {
    __shared__ double red[32];
    double s0 = 0.0, s1 = 0.0;
    // kVecU elements per thread per trip, all loads issued before use (same
    // summation order as a plain grid-stride loop)
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; i0 < n; i0 += kVecU * stride) {
        double rv[kVecU], zv[kVecU], qv[kVecU];
#pragma unroll
        for (int u = 0; u < kVecU; ++u) {
            const long long i = i0 + u * stride;
            rv[u] = zv[u] = qv[u] = 0.0;
            if (i < n) {
                rv[u] = r[i];
                zv[u] = z32 ? (double)z32[i] : z[i];
                qv[u] = q[i];
            }
        }
#pragma unroll
        for (int u = 0; u < kVecU; ++u) {
            const long long i = i0 + u * stride;
            if (i < n) {
                if (z32) z[i] = zv[u];
                s0 += rv[u] * zv[u];
                s1 += zv[u] * qv[u];
                q[i] = 0.0;
            }
        }
    }
    const double t0 = block_sum(s0, red);
    if (threadIdx.x == 0) prz[blockIdx.x] = t0;
    const double t1 = block_sum(s1, red);
    if (threadIdx.x == 0) pzq[blockIdx.x] = t1;
}

__global__ void __launch_bounds__(256) dots_rz_zq_kernel(const double* __restrict__ r, double* __restrict__ z,
                                                         const float* __restrict__ z32, double* __restrict__ q,
                                                         long long n, double* __restrict__ prz,
                                                         double* __restrict__ pzq) {
    grid_dep_sync();
    const long long jr = blockIdx.y;       // right-hand side
    dots_rz_zq_body(r + jr * n, z + jr * n, z32 ? z32 + jr * n : nullptr, q + jr * n, n, prz + jr * gridDim.x,
                    pzq + jr * gridDim.x);
}

// q-independent update: every block sums the partials of p.q (npq, from the
// apply) and of r.z (nrz), alpha = r.z / p.q; x += alpha p; r -= alpha q;
// partials of r.r into prr; the last block publishes S_RR, S_RZ (for the next
// direction), S_ALPHA, S_PQ and the breakdown flag.
__device__ __forceinline__ void fcg_update_body(double* __restrict__ x, double* __restrict__ r,
                                                const double* __restrict__ p, const double* __restrict__ q,
                                                long long n, const double* ppq, int npq, const double* prz, int nrz,
                                                double* prr, double* S, unsigned* ticket, float* __restrict__ r32) {
    // a right-hand side that has stopped keeps its x and r
    const bool active = S[S_DONE] == 0.0;
    __shared__ double red[32];
    __shared__ double sh[3];
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long ifirst = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double xv[kVecU], rv[kVecU], pv[kVecU], qv[kVecU];
    auto load = [&](long long i0) {
#pragma unroll
        for (int u = 0; u < kVecU; ++u) {
            const long long i = i0 + u * stride;
            xv[u] = rv[u] = pv[u] = qv[u] = 0.0;
            if (i < n) {
                xv[u] = x[i];
                rv[u] = r[i];
                pv[u] = p[i];
                qv[u] = q[i];
            }
        }
    };
    // the first trip's vectors are in flight while the partials are summed
    if (active) load(ifirst);
    const double pq = sum_partials(ppq, npq, red);
    const double rz = sum_partials(prz, nrz, red);
    if (threadIdx.x == 0) {
        sh[0] = rz / pq;                    // FP64 division once per block
        sh[1] = pq;
        sh[2] = rz;
    }
    __syncthreads();
    const double alpha = sh[0];
    double s = 0.0;
    for (long long i0 = ifirst; active && i0 < n; i0 += kVecU * stride) {
        if (i0 != ifirst) load(i0);
#pragma unroll
        for (int u = 0; u < kVecU; ++u) {
            const long long i = i0 + u * stride;
            if (i < n) {
                x[i] = xv[u] + alpha * pv[u];
                const double ri = rv[u] - alpha * qv[u];
                r[i] = ri;
                if (r32) r32[i] = (float)ri;
                s += ri * ri;
            }
        }
    }
    const double t = block_sum(s, red);
    if (threadIdx.x == 0) prr[blockIdx.x] = t;
    if (last_block(ticket)) {
        if (active) {
            finalize_partials(prr, 1, gridDim.x, S, S_RR, S_RR, red);
            if (threadIdx.x == 0) {
                S[S_ALPHA] = alpha;
                S[S_PQ] = sh[1];
                S[S_RZ] = sh[2];
                if (!(sh[1] > 0.0) || !isfinite(alpha)) S[S_FLAG] = 1.0;
            }
        }
        if (threadIdx.x == 0) *ticket = 0u;
    }
}

__global__ void __launch_bounds__(256) fcg_update_kernel(double* __restrict__ x, double* __restrict__ r,
                                                         const double* __restrict__ p, const double* __restrict__ q,
                                                         long long n, const double* ppq, int npq, const double* prz,
                                                         int nrz, double* prr, double* S, unsigned* ticket,
                                                         float* __restrict__ r32) {
    grid_dep_sync();
    const long long jr = blockIdx.y;       // right-hand side
    fcg_update_body(x + jr * n, r + jr * n, p + jr * n, q + jr * n, n, ppq + jr * npq, npq, prz + jr * nrz, nrz,
                    prr + jr * gridDim.x, S + jr * S_COUNT, ticket + jr, r32 ? r32 + jr * n : nullptr);
}

// p = z + beta p, beta = -alpha zq / rz_old (flexible) or rz_new / rz_old
// (Fletcher-Reeves), with rz_new and zq summed from the dots' partials in
// every block and rz_old, alpha from the previous update.
__device__ __forceinline__ void fcg_direction_body(double* __restrict__ p, const double* __restrict__ z,
                                                   long long n, const double* prz, const double* pzq, int nd,
                                                   const double* __restrict__ S, int flexible) {
    if (S[S_DONE] != 0.0) return;           // stopped: p is no longer used
    __shared__ double red[32];
    __shared__ double sh_beta;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long ifirst = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double zv[kVecU], pv[kVecU];
    auto load = [&](long long i0) {
#pragma unroll
        for (int u = 0; u < kVecU; ++u) {
            const long long i = i0 + u * stride;
            zv[u] = pv[u] = 0.0;
            if (i < n) {
                zv[u] = z[i];
                pv[u] = p[i];
            }
        }
    };
    load(ifirst);      // in flight while the partials are summed
    const double rz_new = sum_partials(prz, nd, red);
    const double zq = sum_partials(pzq, nd, red);
    if (threadIdx.x == 0) sh_beta = flexible ? -S[S_ALPHA] * zq / S[S_RZ] : rz_new / S[S_RZ];
    __syncthreads();
    const double beta = sh_beta;
    for (long long i0 = ifirst; i0 < n; i0 += kVecU * stride) {
        if (i0 != ifirst) load(i0);
#pragma unroll
        for (int u = 0; u < kVecU; ++u) {
            const long long i = i0 + u * stride;
            if (i < n) p[i] = zv[u] + beta * pv[u];
        }
    }
}

__global__ void __launch_bounds__(256) fcg_direction_kernel(double* __restrict__ p, const double* __restrict__ z,
                                                            long long n, const double* prz, const double* pzq, int nd,
                                                            const double* __restrict__ S, int flexible) {
    grid_dep_sync();
    const long long jr = blockIdx.y;       // right-hand side
    fcg_direction_body(p + jr * n, z + jr * n, n, prz + jr * nd, pzq + jr * nd, nd, S + jr * S_COUNT, flexible);
}

// Work-list form of the three outer-iteration kernels: item blockIdx.y is one
// problem (its own vectors, length, partials and scalars), kDotBlocks CTAs
// each.  step 0: dots r.z, z.q; 1: direction; 2: update.
__global__ void __launch_bounds__(256) fcg_list_kernel(const FcgItem* __restrict__ items, int step, int flexible) {
    grid_dep_sync();
    const FcgItem& it = items[blockIdx.y];
    if (step == 0)
        dots_rz_zq_body(it.r, it.z, it.z32, it.q, it.n, it.prz, it.pzq);
    else if (step == 1)
        fcg_direction_body(it.p, it.z, it.n, it.prz, it.pzq, (int)gridDim.x, it.S, flexible);
    else
        fcg_update_body(it.x, it.r, it.p, it.q, it.n, it.ppq, it.npq, it.prz, (int)gridDim.x, it.prr, it.S,
                        it.ticket, it.r32);
}

// ---- GMRES helpers (Arnoldi with classical Gram-Schmidt, twice) ----------
// h[j] = V_j . w for j < k1; V rows of length n with leading dimension ld.
__global__ void __launch_bounds__(256) multidot_kernel(const double* __restrict__ V, long long ld, int k1,
                                                       const double* __restrict__ w, long long n,
                                                       double* part, double* h, unsigned* ticket) {
    grid_dep_sync();
    __shared__ double red[32];
    const int j = blockIdx.y;
    const double* v = V + (long long)j * ld;
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s += v[i] * w[i];
    const double t = block_sum(s, red);
    if (threadIdx.x == 0) part[j * gridDim.x + blockIdx.x] = t;
    if (last_block_of(ticket, gridDim.x * gridDim.y)) {
        for (int jj = 0; jj < k1; ++jj) {
            double a = 0.0;
            for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) a += __ldcg(part + jj * gridDim.x + b);
            const double tt = block_sum(a, red);
            if (threadIdx.x == 0) h[jj] = tt;
        }
        if (threadIdx.x == 0) *ticket = 0u;
    }
}

// w -= sum_{j < k1} h[j] V_j ;  x += sum_{j < k1} h[j] V_j when sign > 0
__global__ void gs_update_kernel(double* __restrict__ w, const double* __restrict__ V, long long ld, int k1,
                                 const double* __restrict__ h, long long n, double sign) {
    grid_dep_sync();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double a = 0.0;
        for (int j = 0; j < k1; ++j) a += h[j] * V[(long long)j * ld + i];
        w[i] += sign * a;
    }
}

// out = in / sqrt(nrm2[0])
__global__ void scale_by_norm_kernel(double* __restrict__ out, const double* __restrict__ in,
                                     const double* __restrict__ nrm2, long long n) {
    grid_dep_sync();
    __shared__ double sh_s;
    if (threadIdx.x == 0) sh_s = 1.0 / sqrt(nrm2[0]);
    __syncthreads();
    const double s = sh_s;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = in[i] * s;
}

// Device-side loop control for the captured solve graph (conditional WHILE
// node): solve_init_kernel runs once after r0.r0 is known, solve_cond_kernel
// ends every outer iteration.
// With several right-hand sides the loop runs while any of them is still
// iterating; each one stops (S_DONE, S_ITS) when it converges or breaks down.
__global__ void solve_init_kernel(double* S0, cudaGraphConditionalHandle h, double tol, int maxit, int nrhs,
                                  int set_cond) {
    grid_dep_sync();
    if (threadIdx.x != 0) return;
    bool go = false;
    for (int j = 0; j < nrhs; ++j) {
        double* S = S0 + (long long)j * S_COUNT;
        const double rr0 = S[S_RR0];
        S[S_RR] = rr0;
        S[S_TOL2] = tol * tol * rr0;
        S[S_ITER] = 0.0;
        S[S_RZ] = 1.0;
        S[S_ALPHA] = 0.0;
        S[S_FLAG] = 0.0;
        S[S_ZQ] = 0.0;
        S[S_PQ] = 0.0;
        S[S_RZNEW] = 0.0;
        S[S_ITS] = 0.0;
        S[S_DONE] = 0.0;
        if (!isfinite(rr0)) {
            S[S_FLAG] = 1.0;
            S[S_DONE] = 2.0;
        } else if (!(rr0 > 0.0)) {
            S[S_DONE] = 1.0;
        }
        go = go || S[S_DONE] == 0.0;
    }
    if (set_cond) cudaGraphSetConditional(h, go && maxit > 0 ? 1u : 0u);
}

__global__ void solve_cond_kernel(double* S0, cudaGraphConditionalHandle h, int maxit, int nrhs, int set_cond) {
    grid_dep_sync();
    if (threadIdx.x != 0) return;
    bool any = false;
    double it = 0.0;
    for (int j = 0; j < nrhs; ++j) {
        double* S = S0 + (long long)j * S_COUNT;
        it = S[S_ITER] + 1.0;
        S[S_ITER] = it;
        if (S[S_DONE] != 0.0) continue;
        const double rr = S[S_RR];
        if (!isfinite(rr) || S[S_FLAG] != 0.0) {
            S[S_FLAG] = 1.0;
            S[S_DONE] = 2.0;
            S[S_ITS] = it;
        } else if (rr <= S[S_TOL2]) {
            S[S_DONE] = 1.0;
            S[S_ITS] = it;
        } else {
            any = true;
        }
    }
    if (set_cond) cudaGraphSetConditional(h, any && it < (double)maxit ? 1u : 0u);
}

// f and f0 hold nrhs vectors; mass and y (A v of the shared lifting) one.
__global__ void lift_rhs_kernel(const double* __restrict__ mass, const double* __restrict__ f,
                                const double* __restrict__ y, double* __restrict__ f0, int3 n, int dim, int nrhs) {
    grid_dep_sync();
    const long long total = (long long)n.x * n.y * n.z;
    const int nn[3] = {n.x, n.y, n.z};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total * nrhs;
         i += (long long)gridDim.x * blockDim.x) {
        const long long li = i % total;
        f0[i] = on_boundary(li, nn, dim) ? 0.0 : mass[li] * f[i] - y[li];
    }
}

__global__ void boundary_only_kernel(const double* __restrict__ g, double* __restrict__ v, int3 n, int dim) {
    grid_dep_sync();
    const long long total = (long long)n.x * n.y * n.z;
    const int nn[3] = {n.x, n.y, n.z};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
        v[i] = on_boundary(i, nn, dim) ? g[i] : 0.0;
}

// y (nrhs vectors of n values) += a x; x one vector for all when x_shared
__global__ void axpy_kernel(double* __restrict__ y, const double* __restrict__ x, double a, long long n, int nrhs,
                            int x_shared) {
    grid_dep_sync();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n * nrhs;
         i += (long long)gridDim.x * blockDim.x)
        y[i] += a * x[x_shared ? i % n : i];
}

inline int grid_for(long long n, int threads = 256) {
    long long b = (n + threads - 1) / threads;
    if (b > 152LL * 16) b = 152LL * 16;
    if (b < 1) b = 1;
    return (int)b;
}

// Dynamic shared memory above 48 KB needs an opt-in per kernel; it is set
// once for every kernel at library initialisation (init_kernel_attributes),
// never during stream capture.
constexpr int kMaxDynSmem = 200 * 1024;

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_apply(const DevLevel<T>& L, const T* x, T* y, bool mask, cudaStream_t st, bool y_is_zero,
                         double* dot, double* part, unsigned* ticket, int nrhs) {
    if (!y_is_zero) {
        const cudaError_t e = cudaMemsetAsync(y, 0, sizeof(T) * L.N * nrhs, st);
        if (e != cudaSuccess) return e;
    }
    // coloured summation: the node-per-thread kernel once per element colour
    if (!L.colored && launch_apply_fixed<T>(L, x, y, mask, dot, part, ticket, st, nrhs)) return cudaSuccess;
    int epc = 256 / L.nloc;
    if (epc < 1) epc = 1;
    const size_t smem = sizeof(T) * (L.n1 * L.n1 + (size_t)epc * L.nloc * (1 + L.dim));
    const int ncolour = L.colored ? 1 << L.dim : 1;
    for (int c = 0; c < ncolour; ++c) {
        const int colour = L.colored ? c : -1;
        const long long nelem = L.colored ? colour_elements(L.ne, L.dim, c) : L.E;
        if (nelem == 0) continue;
        const long long blocks = (nelem + epc - 1) / epc * nrhs;
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
        const cudaError_t e =
            L.dim == 2 ? launch_k(apply_kernel<T, 2>, (unsigned)blocks, 256, smem, st, L, x, y, mask ? 1 : 0, epc,
                                  nrhs, colour, nelem)
                       : launch_k(apply_kernel<T, 3>, (unsigned)blocks, 256, smem, st, L, x, y, mask ? 1 : 0, epc,
                                  nrhs, colour, nelem);
        if (e != cudaSuccess) return e;
    }
    // orders outside the specialised range: x.(A x) as a separate product
    if (dot) {
        if constexpr (sizeof(T) == 8) {
            if (ticket)    // single right-hand side only
                launch_dots(reinterpret_cast<const double*>(x), reinterpret_cast<const double*>(y), nullptr, nullptr,
                            1, L.N, part, dot, 0, 0, ticket, st);
            else   // kDotBlocks partials per right-hand side only
                launch_k(dots_kernel, dim3(kDotBlocks, nrhs), 256, 0, st, reinterpret_cast<const double*>(x),
                         reinterpret_cast<const double*>(y), (const double*)nullptr, (const double*)nullptr, 1, L.N,
                         part, dot, 0, 0, (unsigned*)nullptr, 0);
        }
    }
    return cudaSuccess;
}

template <typename T>
void launch_line_solve(const DevLevel<T>& L, int s, int mode, const T* g, const T* r, T* y, T* x, T alpha,
                       cudaStream_t st, int nrhs) {
    // levels with Def. 3.2 line blocks: the condensed block solve (set-up
    // guarantees the sizes it takes)
    if (L.blk[s] != nullptr) {
        launch_line_block<T>(L, s, mode, g, r, y, x, alpha, st, nrhs);
        return;
    }
    if (launch_line_warp<T>(L, s, mode, g, r, y, x, alpha, st, nrhs)) return;
    // long band-1 lines: the shared-memory kernel, one launch per right-hand side
    if (nrhs > 1) {
        for (int j = 0; j < nrhs; ++j) {
            const long long o = (long long)j * L.N;
            launch_line_solve<T>(L, s, mode, g ? g + o : nullptr, r ? r + o : nullptr, y ? y + o : nullptr, x + o,
                                 alpha, st, 1);
        }
        return;
    }
    LineArgs<T> A;
    A.n = L.n[s] - 2;
    if (A.n <= 0) return;
    int o1, o2;
    if (s == 0) { o1 = 1; o2 = 2; } else if (s == 1) { o1 = 0; o2 = 2; } else { o1 = 0; o2 = 1; }
    const long long strides[3] = {1, L.n[0], (long long)L.n[0] * L.n[1]};
    A.m1 = L.n[o1] - 2;
    const int m2 = L.dim == 3 ? L.n[o2] - 2 : 1;
    A.nlines = (long long)A.m1 * m2;
    if (A.nlines <= 0) return;
    A.stride = strides[s];
    A.st1 = strides[o1];
    A.st2 = L.dim == 3 ? strides[o2] : 0;
    if (L.dim == 2) A.st2 = 0;
    A.contiguous = s == 0;
    A.mode = mode;
    A.alpha = alpha;
    A.diag = L.diag;
    A.off = L.off[s];
    A.g = g;
    A.r = r;
    A.y = y;
    A.x = x;
    const size_t per_line = 4 * sizeof(T) * (size_t)A.n;
    long long W = (96 * 1024) / (long long)per_line;
    if (W > 32) W = 32;
    if (W < 1) W = 1;
    const long long wmin = A.contiguous ? 1 : (32 / (long long)sizeof(T));
    while (W > wmin && (A.nlines + W - 1) / W < 2 * 152) W /= 2;
    A.W = (int)W;
    const size_t smem = per_line * W;
    const long long blocks = (A.nlines + W - 1) / W;
    launch_k(line_kernel<T>, (unsigned)blocks, 256, smem, st, A);
}

template <typename T>
void launch_transfer(const DevBand<T>& M, int a, const int nin[3], const int nout[3], const T* in, const T* in2, T* out,
                     bool add, bool mask, cudaStream_t st, T* clear, int nrhs) {
    const long long total = (long long)nout[0] * nout[1] * nout[2];
    const int dim = nout[2] > 1 ? 3 : 2;
    const int3 ni = make_int3(nin[0], nin[1], nin[2]), no = make_int3(nout[0], nout[1], nout[2]);
    const int g = grid_for(total * nrhs);
    const int ad = add ? 1 : 0, mk = mask ? 1 : 0;
    if (M.width <= 4)
        launch_k(transfer_kernel<T, 4>, g, 256, 0, st, M, a, ni, no, in, in2, out, ad, mk, dim, clear, nrhs);
    else if (M.width <= 8)
        launch_k(transfer_kernel<T, 8>, g, 256, 0, st, M, a, ni, no, in, in2, out, ad, mk, dim, clear, nrhs);
    else if (M.width <= 16)
        launch_k(transfer_kernel<T, 16>, g, 256, 0, st, M, a, ni, no, in, in2, out, ad, mk, dim, clear, nrhs);
    else if (M.width <= 32)
        launch_k(transfer_kernel<T, 32>, g, 256, 0, st, M, a, ni, no, in, in2, out, ad, mk, dim, clear, nrhs);
    else launch_k(transfer_kernel<T, 0>, g, 256, 0, st, M, a, ni, no, in, in2, out, ad, mk, dim, clear, nrhs);
}

template <typename T>
bool launch_transfer2(const DevBand<T>& M0, const DevBand<T>& M1, const int nin[3], const int nout[3], const T* in,
                      const T* in2, T* out, bool add, bool mask, cudaStream_t st, T* clear, int nrhs) {
    constexpr int TY = 8;
    const size_t smem = sizeof(T) * (size_t)M1.span8 * (M0.span32 + 32);
    const int W = M0.width > M1.width ? M0.width : M1.width;
    if (M0.span32 <= 0 || M1.span8 <= 0 || smem > kMaxDynSmem || W > 32) return false;
    // the nrhs right-hand sides follow one another: nrhs x nout[2] planes of axis 2
    const dim3 grid((unsigned)((nout[0] + 31) / 32), (unsigned)((nout[1] + TY - 1) / TY), (unsigned)(nout[2] * nrhs));
    const int3 ni = make_int3(nin[0], nin[1], nin[2]), no = make_int3(nout[0], nout[1], nout[2]);
    const int ad = add ? 1 : 0, mk = mask ? 1 : 0;
    if (W <= 4) launch_k(transfer2_kernel<T, 4, TY>, grid, 256, smem, st, M0, M1, ni, no, in, in2, out, ad, mk, clear);
    else if (W <= 8) launch_k(transfer2_kernel<T, 8, TY>, grid, 256, smem, st, M0, M1, ni, no, in, in2, out, ad, mk, clear);
    else if (W <= 16) launch_k(transfer2_kernel<T, 16, TY>, grid, 256, smem, st, M0, M1, ni, no, in, in2, out, ad, mk, clear);
    else launch_k(transfer2_kernel<T, 32, TY>, grid, 256, smem, st, M0, M1, ni, no, in, in2, out, ad, mk, clear);
    return true;
}

// ---- work-list launchers ------------------------------------------------
// Tile grid, band-width bucket, tile height and shared memory of a fused
// transfer; false when the fused form does not apply (as launch_transfer2).
template <typename T>
bool transfer2_list_config(const DevBand<T>& M0, const DevBand<T>& M1, const int nout[3], int* gx, int* gy, int* wb,
                           int* ty, size_t* smem) {
    constexpr int TY = 8;
    *smem = sizeof(T) * (size_t)M1.span8 * (M0.span32 + 32);
    const int W = M0.width > M1.width ? M0.width : M1.width;
    if (M0.span32 <= 0 || M1.span8 <= 0 || *smem > kMaxDynSmem || W > 32) return false;
    *gx = (nout[0] + 31) / 32;
    *gy = (nout[1] + TY - 1) / TY;
    *ty = TY;
    *wb = W <= 4 ? 4 : W <= 8 ? 8 : W <= 16 ? 16 : 32;
    return true;
}

template <typename T>
bool launch_transfer2_list(int wb, int ty, const Transfer2Item<T>* items, const int* start, int nitems, int blocks,
                           size_t smem, bool add, bool mask, cudaStream_t st) {
    if (nitems < 1 || blocks < 1) return true;
    if (ty != 8) return false;
    const int ad = add ? 1 : 0, mk = mask ? 1 : 0;
    cudaError_t e;
    if (wb == 4) e = launch_k(transfer2_list_kernel<T, 4, 8>, blocks, 256, smem, st, items, start, nitems, ad, mk);
    else if (wb == 8) e = launch_k(transfer2_list_kernel<T, 8, 8>, blocks, 256, smem, st, items, start, nitems, ad, mk);
    else if (wb == 16)
        e = launch_k(transfer2_list_kernel<T, 16, 8>, blocks, 256, smem, st, items, start, nitems, ad, mk);
    else e = launch_k(transfer2_list_kernel<T, 32, 8>, blocks, 256, smem, st, items, start, nitems, ad, mk);
    return e == cudaSuccess;
}

template <typename T>
void launch_coarse_list(const CoarseItem<T>* items, const int* start, int nitems, int blocks, size_t smem,
                        cudaStream_t st) {
    if (nitems < 1 || blocks < 1) return;
    launch_k(coarse_list_kernel<T>, blocks, 256, smem, st, items, start, nitems);
}

template <typename T>
void launch_bcr_list(bool forward, int l, const BcrItem<T>* items, const int* start, int nitems, int blocks,
                     size_t smem, cudaStream_t st) {
    if (nitems < 1 || blocks < 1) return;
    launch_k(bcr_list_kernel<T>, blocks, 256, smem, st, items, start, nitems, l, forward ? 1 : 0);
}

void launch_fcg_list(int step, const FcgItem* items, int nitems, int flexible, int blocks, cudaStream_t st) {
    if (nitems < 1) return;
    launch_k(fcg_list_kernel, dim3(blocks, nitems), 256, 0, st, items, step, flexible);
}

template bool transfer2_list_config<float>(const DevBand<float>&, const DevBand<float>&, const int*, int*, int*, int*,
                                           int*, size_t*);
template bool transfer2_list_config<double>(const DevBand<double>&, const DevBand<double>&, const int*, int*, int*,
                                            int*, int*, size_t*);
template bool launch_transfer2_list<float>(int, int, const Transfer2Item<float>*, const int*, int, int, size_t, bool,
                                           bool, cudaStream_t);
template bool launch_transfer2_list<double>(int, int, const Transfer2Item<double>*, const int*, int, int, size_t, bool,
                                            bool, cudaStream_t);
template void launch_coarse_list<float>(const CoarseItem<float>*, const int*, int, int, size_t, cudaStream_t);
template void launch_coarse_list<double>(const CoarseItem<double>*, const int*, int, int, size_t, cudaStream_t);
template void launch_bcr_list<float>(bool, int, const BcrItem<float>*, const int*, int, int, size_t, cudaStream_t);
template void launch_bcr_list<double>(bool, int, const BcrItem<double>*, const int*, int, int, size_t, cudaStream_t);

template <typename T>
void launch_coarse(const DevCoarse<T>& C, long long N0, const T* r, T* e, T* w, cudaStream_t st, bool e_boundary_zero,
                   int nrhs) {
    // r, e, w: nrhs vectors of N0 values each (the right-hand side fastest
    // in every kernel's CTA order, so each block operator is read once)
    if (!e_boundary_zero) cudaMemsetAsync(e, 0, sizeof(T) * N0 * nrhs, st);
    const int k = C.cr_levels, m = C.m;
    const unsigned rows = (unsigned)((m + kBcrRows - 1) / kBcrRows);
    for (int l = 0; l < k; ++l) {
        const int a = C.nb >> l, nk = a / 2, ne = (a + 1) / 2;
        const unsigned gx = (unsigned)(l == 0 ? nk + ne : nk) * nrhs;
        launch_k(bcr_forward_kernel<T>, dim3(gx, rows), 256, 2 * sizeof(T) * (size_t)m, st, C.fh[l], l, C.nb, m,
                 C.ldm, C.index, r, w, nrhs, N0);
    }
    const size_t smem = sizeof(T) * (size_t)C.ld;
    long long blocks = (C.nr + 7) / 8;
    if (blocks > 2 * 152) blocks = 2 * 152;
    const T* src = k > 0 ? w : r;
    const long long* src_index = k > 0 ? nullptr : C.index;
    launch_k(coarse_kernel<T>, (unsigned)(blocks * nrhs), 256, smem, st, C.nr, C.ld, C.index, C.inv, src, src_index,
             m, 1 << k, e, nrhs, N0);
    for (int l = k - 1; l >= 0; --l) {
        const unsigned ne = (unsigned)(((C.nb >> l) + 1) / 2) * nrhs;
        launch_k(bcr_backward_kernel<T>, dim3(ne, rows), 256, 3 * sizeof(T) * (size_t)m, st, C.agk[l], l, C.nb, m,
                 C.ldm, C.index, (const T*)w, e, nrhs, N0);
    }
}

template <typename Ti, typename To>
void launch_cast(const Ti* in, To* out, long long n, cudaStream_t st) {
    launch_k(cast_kernel<Ti, To>, grid_for(n), 256, 0, st, in, out, n);
}

template <typename T>
void launch_zero_boundary(T* v, const int n[3], int dim, cudaStream_t st, int nrhs) {
    const long long total = (long long)n[0] * n[1] * n[2];
    launch_k(zero_boundary_kernel<T>, grid_for(total * nrhs), 256, 0, st, v, make_int3(n[0], n[1], n[2]), dim, nrhs);
}

void launch_dots(const double* a0, const double* b0, const double* a1, const double* b1, int ndots, long long n,
                 double* part, double* S, int slot0, int slot1, unsigned* ticket, cudaStream_t st, int nrhs) {
    launch_k(dots_kernel, dim3(kDotBlocks, nrhs), 256, 0, st, a0, b0, a1, b1, ndots, n, part, S, slot0, slot1, ticket,
             0);
}

void launch_fcg_update(double* x, double* r, const double* p, const double* q, long long n, const double* ppq,
                       int npq, const double* prz, int nrz, double* prr, double* S, unsigned* ticket, float* r32,
                       cudaStream_t st, int nrhs) {
    // nrz: the dots' CTA count, the same grid here (prr gets one partial per CTA)
    launch_k(fcg_update_kernel, dim3(nrz, nrhs), 256, 0, st, x, r, p, q, n, ppq, npq, prz, nrz, prr, S, ticket, r32);
}

void launch_dots_rz_zq(const double* r, double* z, const float* z32, double* q, long long n, double* prz, double* pzq,
                       cudaStream_t st, int nrhs) {
    launch_k(dots_rz_zq_kernel, dim3(fcg_blocks(n), nrhs), 256, 0, st, r, z, z32, q, n, prz, pzq);
}

void launch_fcg_direction(double* p, const double* z, long long n, const double* prz, const double* pzq, int nd,
                          const double* S, int flexible, cudaStream_t st, int nrhs) {
    launch_k(fcg_direction_kernel, dim3(nd, nrhs), 256, 0, st, p, z, n, prz, pzq, nd, S, flexible);
}

void launch_lift_rhs(const double* mass, const double* f, const double* y, double* f0, const int n[3], int dim,
                     cudaStream_t st, int nrhs) {
    const long long total = (long long)n[0] * n[1] * n[2];
    launch_k(lift_rhs_kernel, grid_for(total * nrhs), 256, 0, st, mass, f, y, f0, make_int3(n[0], n[1], n[2]), dim,
             nrhs);
}

void launch_boundary_only(const double* g, double* v, const int n[3], int dim, cudaStream_t st) {
    const long long total = (long long)n[0] * n[1] * n[2];
    launch_k(boundary_only_kernel, grid_for(total), 256, 0, st, g, v, make_int3(n[0], n[1], n[2]), dim);
}

void launch_multidot(const double* V, long long ld, int k1, const double* w, long long n, double* part, double* h,
                     unsigned* ticket, cudaStream_t st) {
    long long nb = (n + 255) / 256;
    if (nb > 64) nb = 64;
    launch_k(multidot_kernel, dim3((unsigned)nb, (unsigned)k1), 256, 0, st, V, ld, k1, w, n, part, h, ticket);
}

void launch_gs_update(double* w, const double* V, long long ld, int k1, const double* h, long long n, double sign,
                      cudaStream_t st) {
    launch_k(gs_update_kernel, grid_for(n), 256, 0, st, w, V, ld, k1, h, n, sign);
}

void launch_scale_by_norm(double* out, const double* in, const double* nrm2, long long n, cudaStream_t st) {
    launch_k(scale_by_norm_kernel, grid_for(n), 256, 0, st, out, in, nrm2, n);
}

void launch_solve_init(double* S, cudaGraphConditionalHandle h, double tol, int maxit, cudaStream_t st, int nrhs,
                       bool set_cond) {
    launch_k(solve_init_kernel, 1, 32, 0, st, S, h, tol, maxit, nrhs, set_cond ? 1 : 0);
}

void launch_solve_cond(double* S, cudaGraphConditionalHandle h, int maxit, cudaStream_t st, int nrhs,
                       bool set_cond) {
    launch_k(solve_cond_kernel, 1, 32, 0, st, S, h, maxit, nrhs, set_cond ? 1 : 0);
}

void launch_axpy(double* y, const double* x, double a, long long n, cudaStream_t st, int nrhs, bool x_shared) {
    launch_k(axpy_kernel, grid_for(n * nrhs), 256, 0, st, y, x, a, n, nrhs, x_shared ? 1 : 0);
}

bool pdl_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("GLLS_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

bool init_kernel_attributes() {
    const void* fns[] = {(const void*)apply_kernel<double, 2>, (const void*)apply_kernel<double, 3>,
                         (const void*)apply_kernel<float, 2>,  (const void*)apply_kernel<float, 3>,
                         (const void*)line_kernel<double>,     (const void*)line_kernel<float>,
                         (const void*)coarse_kernel<double>,   (const void*)coarse_kernel<float>,
                         (const void*)bcr_forward_kernel<double>, (const void*)bcr_forward_kernel<float>,
                         (const void*)bcr_backward_kernel<double>, (const void*)bcr_backward_kernel<float>,
                         (const void*)transfer2_kernel<double, 4, 8>, (const void*)transfer2_kernel<float, 4, 8>,
                         (const void*)transfer2_kernel<double, 8, 8>, (const void*)transfer2_kernel<float, 8, 8>,
                         (const void*)transfer2_kernel<double, 16, 8>, (const void*)transfer2_kernel<float, 16, 8>,
                         (const void*)transfer2_kernel<double, 32, 8>, (const void*)transfer2_kernel<float, 32, 8>,
                         (const void*)coarse_list_kernel<double>, (const void*)coarse_list_kernel<float>,
                         (const void*)bcr_list_kernel<double>, (const void*)bcr_list_kernel<float>,
                         (const void*)transfer2_list_kernel<double, 4, 8>, (const void*)transfer2_list_kernel<float, 4, 8>,
                         (const void*)transfer2_list_kernel<double, 8, 8>, (const void*)transfer2_list_kernel<float, 8, 8>,
                         (const void*)transfer2_list_kernel<double, 16, 8>,
                         (const void*)transfer2_list_kernel<float, 16, 8>,
                         (const void*)transfer2_list_kernel<double, 32, 8>,
                         (const void*)transfer2_list_kernel<float, 32, 8>};
    for (const void* f : fns)
        if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem) != cudaSuccess)
            return false;
    return init_line_warp_attributes() && init_line_block_attributes() && init_apply_col_attributes() &&
           init_apply_eo_attributes();
}

// explicit instantiations
template cudaError_t launch_apply<double>(const DevLevel<double>&, const double*, double*, bool, cudaStream_t, bool, double*,
                                   double*, unsigned*, int);
template cudaError_t launch_apply<float>(const DevLevel<float>&, const float*, float*, bool, cudaStream_t, bool, double*,
                                  double*, unsigned*, int);
template void launch_line_solve<double>(const DevLevel<double>&, int, int, const double*, const double*, double*,
                                        double*, double, cudaStream_t, int);
template void launch_line_solve<float>(const DevLevel<float>&, int, int, const float*, const float*, float*,
                                       float*, float, cudaStream_t, int);
template void launch_transfer<double>(const DevBand<double>&, int, const int*, const int*, const double*, const double*,
                                      double*, bool, bool, cudaStream_t, double*, int);
template void launch_transfer<float>(const DevBand<float>&, int, const int*, const int*, const float*, const float*,
                                     float*, bool, bool, cudaStream_t, float*, int);
template void launch_coarse<double>(const DevCoarse<double>&, long long, const double*, double*, double*, cudaStream_t,
                                    bool, int);
template void launch_coarse<float>(const DevCoarse<float>&, long long, const float*, float*, float*, cudaStream_t, bool,
                                   int);
template bool launch_transfer2<double>(const DevBand<double>&, const DevBand<double>&, const int*, const int*,
                                       const double*, const double*, double*, bool, bool, cudaStream_t, double*, int);
template bool launch_transfer2<float>(const DevBand<float>&, const DevBand<float>&, const int*, const int*,
                                      const float*, const float*, float*, bool, bool, cudaStream_t, float*, int);
template void launch_cast<double, float>(const double*, float*, long long, cudaStream_t);
template void launch_cast<float, double>(const float*, double*, long long, cudaStream_t);
template void launch_zero_boundary<double>(double*, const int*, int, cudaStream_t, int);
template void launch_zero_boundary<float>(float*, const int*, int, cudaStream_t, int);

}  // namespace glls
