// Stiffness apply y = A_l x (eq. discreteBilinear) specialised on the GLL
// order P, so that local index arithmetic and the sum-factorisation loops are
// resolved at compile time.  Per CTA: EPB elements; x gathered into shared
// memory, reference gradients by 1-D contractions with D, pointwise G, the
// transposed contractions, then element-interior nodes stored and shared
// nodes summed with atomics (direct stiffness summation).  32-bit indexing.
#include "device.cuh"
#include "reduce.cuh"

namespace glls {
namespace {

__device__ __forceinline__ bool on_boundary32(int I, int J, int K, const int n[3], int dim) {
    return I == 0 || I == n[0] - 1 || J == 0 || J == n[1] - 1 || (dim == 3 && (K == 0 || K == n[2] - 1));
}

// DOT: also sum_e x_e^T (A_e x_e) over all elements into *dot (last block).
// Each thread owns ITEMS local nodes (t = threadIdx.x + 256 * it); its
// geometry factors are loaded into registers before the x gather, so the two
// global-memory latencies overlap.
// sum_m a[m] b[m] and sum_m a[m] b[m * stride] over N terms with a (and, in
// the first form, b) contiguous and 16-byte aligned: float4 loads, the terms
// added in m order.
template <int N>
__device__ __forceinline__ float dot_cc(const float* a, const float* b) {
    const float4* a4 = reinterpret_cast<const float4*>(a);
    const float4* b4 = reinterpret_cast<const float4*>(b);
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < N / 4; ++q) {
        const float4 u = a4[q], v = b4[q];
        s += u.x * v.x;
        s += u.y * v.y;
        s += u.z * v.z;
        s += u.w * v.w;
    }
    return s;
}
template <int N, int STRIDE>
__device__ __forceinline__ float dot_cs(const float* a, const float* b) {
    const float4* a4 = reinterpret_cast<const float4*>(a);
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < N / 4; ++q) {
        const float4 u = a4[q];
        s += u.x * b[(4 * q) * STRIDE];
        s += u.y * b[(4 * q + 1) * STRIDE];
        s += u.z * b[(4 * q + 2) * STRIDE];
        s += u.w * b[(4 * q + 3) * STRIDE];
    }
    return s;
}

// Launch bounds (256, 1): at least one resident CTA per SM.  (Eight for 2-D
// FP32 would cap it at 32 registers; measured inside the solve that is
// 0.5-1 % slower than the 48 registers the compiler picks with one.)
// The CTA body: block `blk` of `nblk` (per right-hand side: the right-hand
// side fastest in the CTA order, see device.cuh).
template <typename T, int DIM, int P, bool DOT>
__device__ __forceinline__ void apply_p_body(const DevLevel<T>& L, const T* __restrict__ x, T* __restrict__ y,
                                             int mask, double* dot, double* part, unsigned* ticket, int nrhs, int blk,
                                             int nblk) {
    const int rhs = blk % nrhs, bx = blk / nrhs, nbx = nblk / nrhs;
    x += (long long)rhs * L.N;
    y += (long long)rhs * L.N;
    constexpr int N1 = P + 1;
    constexpr int NLOC = DIM == 2 ? N1 * N1 : N1 * N1 * N1;
    constexpr int EPB = NLOC >= 256 ? 1 : 256 / NLOC;
    constexpr int ITEMS = (EPB * NLOC + 255) / 256;
    constexpr int NC = DIM == 2 ? 3 : 6;
    // FP32 with N1 a multiple of 4: rows of D, D^T, x and w are 16-byte
    // aligned, so the contractions read them with float4 loads
    constexpr bool VEC = sizeof(T) == 4 && N1 % 4 == 0;
    __shared__ __align__(16) T sD[N1 * N1];
    __shared__ __align__(16) T sDT[VEC ? N1 * N1 : 1];
    __shared__ __align__(16) T sx[EPB * NLOC];
    __shared__ __align__(16) T sw[DIM * EPB * NLOC];
    __shared__ int sbase[EPB];   // global index of each element's first node
    __shared__ int sxyz[EPB];    // element coordinates packed 10:10:10 bits
    const int E = (int)L.E;
    const int n0 = L.n[0], n1 = L.n[1];
    const int EN = E * NLOC;
    const int e0 = bx * EPB;
    const int total = min(EPB, E - e0) * NLOC;
    if (threadIdx.x < EPB && e0 + (int)threadIdx.x < E) {
        const int e = e0 + threadIdx.x, ne0 = L.ne[0], ne1 = L.ne[1];
        const int ex = e % ne0, ey = (e / ne0) % ne1, ez = DIM == 3 ? e / (ne0 * ne1) : 0;
        sbase[threadIdx.x] = ((ez * P) * n1 + ey * P) * n0 + ex * P;
        sxyz[threadIdx.x] = ex | (ey << 10) | (ez << 20);
    }

    T gk[ITEMS][NC];
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const int t = threadIdx.x + 256 * it;
        if (t < total) {
            const int gq = e0 * NLOC + t;          // = (e0 + el) * NLOC + q
#pragma unroll
            for (int c = 0; c < NC; ++c) gk[it][c] = __ldg(L.G + c * EN + gq);
        }
    }
    for (int t = threadIdx.x; t < N1 * N1; t += 256) {
        sD[t] = L.D[t];
        if constexpr (VEC) sDT[t] = L.D[(t % N1) * N1 + t / N1];
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const int t = threadIdx.x + 256 * it;
        if (t < total) {
            const int el = t / NLOC, q = t - el * NLOC;
            const int i = q % N1, j = (q / N1) % N1, k = DIM == 3 ? q / (N1 * N1) : 0;
            sx[t] = x[sbase[el] + (k * n1 + j) * n0 + i];
        }
    }
    __syncthreads();

#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const int t = threadIdx.x + 256 * it;
        if (t >= total) break;
        const int el = t / NLOC, q = t - el * NLOC;
        const int i = q % N1, j = (q / N1) % N1, k = DIM == 3 ? q / (N1 * N1) : 0;
        const T* xe = sx + el * NLOC;
        T g0 = T(0), g1 = T(0), g2 = T(0);
        if constexpr (VEC) {
            g0 = dot_cc<N1>(sD + i * N1, xe + (k * N1 + j) * N1);
            g1 = dot_cs<N1, N1>(sD + j * N1, xe + k * N1 * N1 + i);
            if (DIM == 3) g2 = dot_cs<N1, N1 * N1>(sD + k * N1, xe + j * N1 + i);
        } else {
#pragma unroll
            for (int m = 0; m < N1; ++m) {
                g0 += sD[i * N1 + m] * xe[(k * N1 + j) * N1 + m];
                g1 += sD[j * N1 + m] * xe[(k * N1 + m) * N1 + i];
                if (DIM == 3) g2 += sD[k * N1 + m] * xe[(m * N1 + j) * N1 + i];
            }
        }
        const T* a = gk[it];
        if (DIM == 2) {
            sw[t] = a[0] * g0 + a[1] * g1;
            sw[EPB * NLOC + t] = a[1] * g0 + a[2] * g1;
        } else {
            sw[t] = a[0] * g0 + a[1] * g1 + a[2] * g2;
            sw[EPB * NLOC + t] = a[1] * g0 + a[3 % NC] * g1 + a[4 % NC] * g2;
            sw[2 * EPB * NLOC + t] = a[2] * g0 + a[4 % NC] * g1 + a[5 % NC] * g2;
        }
    }
    __syncthreads();

    double local = 0.0;
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const int t = threadIdx.x + 256 * it;
        if (t >= total) break;
        const int el = t / NLOC, q = t - el * NLOC;
        const int i = q % N1, j = (q / N1) % N1, k = DIM == 3 ? q / (N1 * N1) : 0;
        const T* w0 = sw + el * NLOC;
        const T* w1 = sw + EPB * NLOC + el * NLOC;
        T v = T(0);
        if constexpr (VEC) {
            v = dot_cc<N1>(sDT + i * N1, w0 + (k * N1 + j) * N1) + dot_cs<N1, N1>(sDT + j * N1, w1 + k * N1 * N1 + i);
            if (DIM == 3) v += dot_cs<N1, N1 * N1>(sDT + k * N1, sw + 2 * EPB * NLOC + el * NLOC + j * N1 + i);
        } else {
#pragma unroll
            for (int m = 0; m < N1; ++m) {
                v += sD[m * N1 + i] * w0[(k * N1 + j) * N1 + m];
                v += sD[m * N1 + j] * w1[(k * N1 + m) * N1 + i];
                if (DIM == 3) v += sD[m * N1 + k] * sw[2 * EPB * NLOC + el * NLOC + (m * N1 + j) * N1 + i];
            }
        }
        const int exyz = sxyz[el];
        const int I = (exyz & 1023) * P + i, J = ((exyz >> 10) & 1023) * P + j, K = (exyz >> 20) * P + k;
        const int g = sbase[el] + (k * n1 + j) * n0 + i;
        if (DOT) local += (double)sx[t] * (double)v;
        const bool inner = i > 0 && i < P && j > 0 && j < P && (DIM == 2 || (k > 0 && k < P));
        if (inner) {
            y[g] = v;
        } else {
            if (mask && on_boundary32(I, J, K, L.n, DIM)) continue;
            atomicAdd(&y[g], v);
        }
    }
    if (DOT) {
        // per-block partial of x.(A x); with a ticket the last block also sums
        // them into dot[0], without one the consumer sums the partials
        __shared__ double red[32];
        const double tsum = block_sum(local, red);
        if (threadIdx.x == 0) part[(long long)rhs * nbx + bx] = tsum;
        if (ticket && last_block(ticket)) {   // single right-hand side, single launch only
            finalize_partials(part, 1, nblk, dot, 0, 0, red);
            if (threadIdx.x == 0) *ticket = 0u;
        }
    }
}

template <typename T, int DIM, int P, bool DOT>
__global__ void __launch_bounds__(256, 1) apply_p_kernel(DevLevel<T> L, const T* __restrict__ x, T* __restrict__ y,
                                                         int mask, double* dot, double* part, unsigned* ticket,
                                                         int nrhs) {
    grid_dep_sync();
    apply_p_body<T, DIM, P, DOT>(L, x, y, mask, dot, part, ticket, nrhs, blockIdx.x, gridDim.x);
}

// Work-list form: item j (its own level, vectors and partials) owns the CTAs
// [start[j], start[j + 1]) of the launch.
template <typename T, int DIM, int P, bool DOT>
__global__ void __launch_bounds__(256, 1) apply_p_list_kernel(const ApplyItem<T>* __restrict__ items,
                                                              const int* __restrict__ start, int nitems, int mask) {
    grid_dep_sync();
    const int j = work_item(start, nitems, blockIdx.x);
    const ApplyItem<T>& it = items[j];
    if (it.done && *it.done != 0.0) return;
    apply_p_body<T, DIM, P, DOT>(it.L, it.x, it.y, mask, nullptr, it.part, nullptr, 1, blockIdx.x - start[j],
                                 start[j + 1] - start[j]);
}

// Number of CTAs (= dot partials) the specialised apply launches for L.
template <typename T, int DIM, int P>
int apply_blocks(const DevLevel<T>& L) {
    constexpr int N1 = P + 1;
    constexpr int NLOC = DIM == 2 ? N1 * N1 : N1 * N1 * N1;
    constexpr int EPB = NLOC >= 256 ? 1 : 256 / NLOC;
    return (int)((L.E + EPB - 1) / EPB);
}

template <typename T, int DIM, int P>
bool launch_p(const DevLevel<T>& L, const T* x, T* y, bool mask, double* dot, double* part, unsigned* ticket,
              cudaStream_t st, int nrhs) {
    constexpr int N1 = P + 1;
    constexpr int NLOC = DIM == 2 ? N1 * N1 : N1 * N1 * N1;
    constexpr int EPB = NLOC >= 256 ? 1 : 256 / NLOC;
    const long long blocks = (L.E + EPB - 1) / EPB * nrhs;
    if (blocks > 0x7fffffffLL) return false;
    if (dot) {
        launch_k(apply_p_kernel<T, DIM, P, true>, (unsigned)blocks, 256, 0, st, L, x, y, mask ? 1 : 0, dot, part,
                 ticket, nrhs);
    } else {
        launch_k(apply_p_kernel<T, DIM, P, false>, (unsigned)blocks, 256, 0, st, L, x, y, mask ? 1 : 0, nullptr,
                 nullptr, nullptr, nrhs);
    }
    return true;
}

template <typename T, int DIM, int P>
bool dispatch(int p, const DevLevel<T>& L, const T* x, T* y, bool mask, double* dot, double* part, unsigned* ticket,
              cudaStream_t st, int nrhs) {
    if constexpr (P == 0) {
        return false;
    } else {
        if (p == P) return launch_p<T, DIM, P>(L, x, y, mask, dot, part, ticket, st, nrhs);
        return dispatch<T, DIM, P - 1>(p, L, x, y, mask, dot, part, ticket, st, nrhs);
    }
}

template <typename T, int P>
bool launch_list_p(int p, const ApplyItem<T>* items, const int* start, int nitems, int blocks, bool mask, bool dot,
                   cudaStream_t st) {
    if constexpr (P == 0) {
        return false;
    } else {
        if (p != P) return launch_list_p<T, P - 1>(p, items, start, nitems, blocks, mask, dot, st);
        if (dot)
            launch_k(apply_p_list_kernel<T, 2, P, true>, (unsigned)blocks, 256, 0, st, items, start, nitems,
                     mask ? 1 : 0);
        else
            launch_k(apply_p_list_kernel<T, 2, P, false>, (unsigned)blocks, 256, 0, st, items, start, nitems,
                     mask ? 1 : 0);
        return true;
    }
}

}  // namespace

// CTAs of the 2-D work-list apply for a level of order p with E elements
// (one dot partial each).
int apply_list_blocks(int p, long long E) {
    const int nloc = (p + 1) * (p + 1);
    const int epb = nloc >= 256 ? 1 : 256 / nloc;
    return (int)((E + epb - 1) / epb);
}

// 2-D work-list apply (orders 1..16): every item's level has order p.
template <typename T>
bool launch_apply_list(int p, const ApplyItem<T>* items, const int* start, int nitems, int blocks, bool mask,
                       bool dot, cudaStream_t st) {
    if (nitems < 1 || blocks < 1) return true;
    return launch_list_p<T, 16>(p, items, start, nitems, blocks, mask, dot, st);
}
template bool launch_apply_list<float>(int, const ApplyItem<float>*, const int*, int, int, bool, bool, cudaStream_t);
template bool launch_apply_list<double>(int, const ApplyItem<double>*, const int*, int, int, bool, bool,
                                        cudaStream_t);

// Dot partials that launch_apply writes for L (one per CTA of the
// specialised kernel, else one per block of the separate dot launch).
template <typename T>
int apply_dot_partials(const DevLevel<T>& L) {
    bool fixed = L.N <= (1LL << 31) - 1 && L.E * L.nloc * (L.dim == 2 ? 3 : 6) <= (1LL << 31) - 1 && L.p >= 1 &&
                 L.p <= (L.dim == 2 ? 16 : 8);
    for (int a = 0; a < L.dim; ++a)
        if (L.ne[a] >= 1024) fixed = false;
    if (!fixed) return kDotBlocks;
    if (apply_eo_selected(L.dim, L.p, true)) return apply_eo_blocks(L.p, L.E);
    long long nloc = 1;
    for (int a = 0; a < L.dim; ++a) nloc *= L.p + 1;
    const long long epb = nloc >= 256 ? 1 : 256 / nloc;
    return (int)((L.E + epb - 1) / epb);
}
template int apply_dot_partials<double>(const DevLevel<double>&);

// Returns false when the order has no specialisation (the caller falls back).
template <typename T>
bool launch_apply_fixed(const DevLevel<T>& L, const T* x, T* y, bool mask, double* dot, double* part,
                        unsigned* ticket, cudaStream_t st, int nrhs) {
    if (L.N > (1LL << 31) - 1 || L.E * L.nloc * (L.dim == 2 ? 3 : 6) > (1LL << 31) - 1) return false;
    for (int a = 0; a < L.dim; ++a)
        if (L.ne[a] >= 1024) return false;   // element coordinates are packed in 10 bits
    // 3-D: the even-odd line kernel where it was measured fastest, then the
    // FP32 column kernel, else the node-per-thread kernel below
    if (launch_apply_eo<T>(L, x, y, mask, dot, part, ticket, st, nrhs)) return true;
    if constexpr (sizeof(T) == 4) {
        if (L.dim == 3 && !dot && launch_apply_col(L, x, y, mask, st, nrhs)) return true;
    }
    if (L.dim == 2) return dispatch<T, 2, 16>(L.p, L, x, y, mask, dot, part, ticket, st, nrhs);
    // 3-D FP32 is served by the even-odd and column kernels above at every
    // order up to 8; this kernel keeps 3-D FP64
    if constexpr (sizeof(T) == 8) return dispatch<T, 3, 8>(L.p, L, x, y, mask, dot, part, ticket, st, nrhs);
    return false;
}

template bool launch_apply_fixed<float>(const DevLevel<float>&, const float*, float*, bool, double*, double*,
                                        unsigned*, cudaStream_t, int);
template bool launch_apply_fixed<double>(const DevLevel<double>&, const double*, double*, bool, double*, double*,
                                         unsigned*, cudaStream_t, int);

}  // namespace glls
