// 3-D stiffness apply y = A_l x (eq. discreteBilinear) with one thread per
// element grid line and the 1-D derivative sweeps in even-odd form.
//
// The GLL nodes are symmetric about 0, so the differentiation matrix is
// centro-antisymmetric: D[N-1-i][N-1-m] = -D[i][m] (N = p + 1), and so is
// D^T.  With u_e[m] = u[m] + u[N-1-m], u_o[m] = u[m] - u[N-1-m] (m < N/2),
//   A_i = sum_m E[i][m] u_e[m] (+ D[i][h] u[h], N odd, h = N/2),
//   B_i = sum_m O[i][m] u_o[m],   E, O = (D[i][m] +- D[i][N-1-m]) / 2,
// a line's derivative is (Du)[i] = A_i + B_i, (Du)[N-1-i] = B_i - A_i, and
// for N odd (Du)[h] = sum_m D[h][m] u_o[m]: N^2/2 multiply-adds and 2N adds
// per line instead of N^2 multiply-adds.  The coefficients are kernel
// parameters read with compile-time indices (constant-bank operands, no
// registers, no loads).  One thread owning a whole line is what lets the
// pairs (i, N-1-i) share A_i and B_i.
//
// Per element (N^2 threads), thread (a, b) owns the t-line (i, j) = (a, b)
// in registers (global reads of x and G, the t sweeps and the scatter, all
// coalesced along i), and the r-line (j, k) = (a, b) and the s-line
// (i, k) = (a, b) through shared memory.  Element-interior nodes are stored,
// shared nodes summed with atomics (direct stiffness summation), Dirichlet
// rows skipped when mask is set.  DOT: per-block partials of
// sum_e x_e^T (A_e x_e) as in the node-per-thread kernels.
#include "device.cuh"
#include "reduce.cuh"
#include "setup.h"

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

namespace glls {

namespace {

// Elements per CTA of the even-odd kernel: at most 256 threads, and no more
// elements than keep about eight CTAs per SM on the level (152 SMs).
int eo_epb(int p, long long E) {
    const long long most = 256 / ((p + 1) * (p + 1));
    const long long fill = E / (152 * 8);
    return (int)std::max(1LL, std::min(most, fill));
}

// One N x N matrix M in even-odd form (H = N / 2).
template <typename T, int N>
struct EoMat {
    static constexpr int H = N / 2;
    T e[H * H];   // (M[i][m] + M[i][N-1-m]) / 2, i, m < H
    T o[H * H];   // (M[i][m] - M[i][N-1-m]) / 2
    T c[H];       // M[i][h], N odd
    T r[H];       // M[h][m], N odd
};
template <typename T, int N>
struct EoParams {
    EoMat<T, N> f;   // D
    EoMat<T, N> t;   // D^T
};

// out = M u for one line, even-odd form
template <typename T, int N>
__device__ __forceinline__ void eo_line(const EoMat<T, N>& M, const T (&u)[N], T (&out)[N]) {
    constexpr int H = N / 2;
    constexpr bool ODD = (N & 1) != 0;
    T ue[H], uo[H];
#pragma unroll
    for (int m = 0; m < H; ++m) {
        ue[m] = u[m] + u[N - 1 - m];
        uo[m] = u[m] - u[N - 1 - m];
    }
#pragma unroll
    for (int i = 0; i < H; ++i) {
        T a = ODD ? M.c[i] * u[H] : T(0), b = T(0);
#pragma unroll
        for (int m = 0; m < H; ++m) {
            a += M.e[i * H + m] * ue[m];
            b += M.o[i * H + m] * uo[m];
        }
        out[i] = a + b;
        out[N - 1 - i] = b - a;
    }
    if constexpr (ODD) {
        T s = T(0);
#pragma unroll
        for (int m = 0; m < H; ++m) s += M.r[m] * uo[m];
        out[H] = s;
    }
}

// Shared-memory strides (in elements of T): row RS, plane PS, element ES,
// chosen so that the row, column and node accesses of a warp spread over the
// banks (at most a two-way conflict).
template <typename T, int N>
struct EoShape {
    static constexpr bool F64 = sizeof(T) == 8;
    static constexpr int NP = N * N, NLOC = NP * N;
    static constexpr int EPB = 256 / NP;                     // most elements per CTA (256 threads)
    static constexpr int RS = N == 8 ? 9 : N == 7 ? (F64 ? 7 : 9) : N == 6 ? (F64 ? 9 : 6) : N == 9 ? 9 : N;
    static constexpr int PS = N == 2 ? 5 : N == 3 ? 9 : N == 4 ? 19 : N == 5 ? 25 : N == 6 ? (F64 ? 54 : 37)
                            : N == 7 ? (F64 ? 52 : 71) : N == 8 ? 72 : (F64 ? 89 : 81);
    static constexpr int ES = N == 2 ? 12 : N == 3 ? 27 : N == 4 ? (F64 ? 76 : 80) : N == 5 ? 125
                            : N == 6 ? (F64 ? 324 : 228) : N == 7 ? (F64 ? 369 : 497) : N == 8 ? 576 : (F64 ? 801 : 729);
    static constexpr int NBUF = 3;                           // x, and two work buffers
};

__device__ __forceinline__ bool on_bd(int I, int J, int K, const int n[3]) {
    return I == 0 || I == n[0] - 1 || J == 0 || J == n[1] - 1 || K == 0 || K == n[2] - 1;
}

// epb elements per CTA (at most EoShape::EPB), chosen at launch so that
// small levels still spread over many CTAs per SM.  Two resident CTAs per SM
// bound the registers (at most 128 per thread).
template <typename T, int P, bool DOT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2)
    apply_eo3_kernel(DevLevel<T> L, const __grid_constant__ EoParams<T, P + 1> M, const T* __restrict__ x,
                     T* __restrict__ y, int mask, double* dot, double* part, unsigned* ticket, int epb, int nrhs) {
    using S = EoShape<T, P + 1>;
    constexpr int N = P + 1, NP = S::NP, NLOC = S::NLOC, RS = S::RS, PS = S::PS, ES = S::ES;
    extern __shared__ __align__(16) unsigned char eo_smem3[];
    T* sX = reinterpret_cast<T*>(eo_smem3);
    T* sU = sX + epb * ES;
    T* sV = sU + epb * ES;
    grid_dep_sync();
    // right-hand side fastest in the CTA order (see device.cuh)
    const int rhs = blockIdx.x % nrhs, bx = blockIdx.x / nrhs, nbx = gridDim.x / nrhs;
    x += (long long)rhs * L.N;
    y += (long long)rhs * L.N;
    const int E = (int)L.E, n0 = L.n[0], n1 = L.n[1];
    const int nplane = n0 * n1;
    const int tid = threadIdx.x;
    const int el = tid / NP, c = tid - el * NP, a = c % N, b = c / N;
    const int e = bx * epb + el;
    const bool act = el < epb && e < E;
    const int elo = act ? el : 0;
    T* X = sX + elo * ES;
    T* U = sU + elo * ES;
    T* V = sV + elo * ES;
    int base = 0, I = 0, J = 0, K0 = 0;
    T xc[N], ut[N];
    if (act) {
        const int ne0 = L.ne[0], ne1 = L.ne[1];
        const int ex = e % ne0, ey = (e / ne0) % ne1, ez = e / (ne0 * ne1);
        I = ex * P + a;
        J = ey * P + b;
        K0 = ez * P;
        base = (K0 * n1 + J) * n0 + I;
#pragma unroll
        for (int k = 0; k < N; ++k) xc[k] = x[base + k * nplane];
#pragma unroll
        for (int k = 0; k < N; ++k) X[k * PS + b * RS + a] = xc[k];
        eo_line<T, N>(M.f, xc, ut);
    }
    __syncthreads();
    if (act) {
        // r-line (j, k) = (a, b) of x into U, s-line (i, k) = (a, b) into V
        T u[N], v[N];
#pragma unroll
        for (int m = 0; m < N; ++m) u[m] = X[b * PS + a * RS + m];
        eo_line<T, N>(M.f, u, v);
#pragma unroll
        for (int m = 0; m < N; ++m) U[b * PS + a * RS + m] = v[m];
#pragma unroll
        for (int m = 0; m < N; ++m) u[m] = X[b * PS + m * RS + a];
        eo_line<T, N>(M.f, u, v);
#pragma unroll
        for (int m = 0; m < N; ++m) V[b * PS + m * RS + a] = v[m];
    }
    __syncthreads();
    T yt[N];
    if (act) {
        // node (a, b, k): w = G grad x; w_r, w_s over the node's own U, V slots,
        // w_t along the t-line in registers, then D^T along it
        const int EN = E * NLOC;
        const T* G = L.G + e * NLOC + c;
        T wt[N];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const T g0 = __ldg(G + k * NP), g1 = __ldg(G + EN + k * NP), g2 = __ldg(G + 2 * EN + k * NP);
            const T g3 = __ldg(G + 3 * EN + k * NP), g4 = __ldg(G + 4 * EN + k * NP);
            const T g5 = __ldg(G + 5 * EN + k * NP);
            const int s = k * PS + b * RS + a;
            const T dr = U[s], ds = V[s], dt = ut[k];
            U[s] = g0 * dr + g1 * ds + g2 * dt;
            V[s] = g1 * dr + g3 * ds + g4 * dt;
            wt[k] = g2 * dr + g4 * ds + g5 * dt;
        }
        eo_line<T, N>(M.t, wt, yt);
    }
    __syncthreads();
    if (act) {
        // D^T along the r-line (j, k) = (a, b) of w_r and the s-line (i, k) = (a, b) of w_s, in place
        T u[N], v[N];
#pragma unroll
        for (int m = 0; m < N; ++m) u[m] = U[b * PS + a * RS + m];
        eo_line<T, N>(M.t, u, v);
#pragma unroll
        for (int m = 0; m < N; ++m) U[b * PS + a * RS + m] = v[m];
#pragma unroll
        for (int m = 0; m < N; ++m) u[m] = V[b * PS + m * RS + a];
        eo_line<T, N>(M.t, u, v);
#pragma unroll
        for (int m = 0; m < N; ++m) V[b * PS + m * RS + a] = v[m];
    }
    __syncthreads();
    double local = 0.0;
    if (act) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const int s = k * PS + b * RS + a;
            const T v = yt[k] + U[s] + V[s];
            if (DOT) local += (double)xc[k] * (double)v;
            const int g = base + k * nplane;
            if (a > 0 && a < P && b > 0 && b < P && k > 0 && k < P) {
                y[g] = v;
            } else {
                if (mask && on_bd(I, J, K0 + k, L.n)) continue;
                atomicAdd(&y[g], v);
            }
        }
    }
    if (DOT) {
        __shared__ double red[32];
        const double tsum = block_sum(local, red);
        if (tid == 0) part[(long long)rhs * nbx + bx] = tsum;
        if (ticket && last_block(ticket)) {   // single right-hand side only
            finalize_partials(part, 1, gridDim.x, dot, 0, 0, red);
            if (tid == 0) *ticket = 0u;
        }
    }
}

// Even-odd coefficients of D and D^T of order p in T, built once per order
template <typename T>
const std::vector<T>& eo_table(int p) {
    static std::once_flag once;
    static std::vector<T> tab[9];
    std::call_once(once, [] {
        for (int q = 1; q <= 8; ++q) {
            const int n = q + 1, h = n / 2;
            const std::vector<double> D = derivative_matrix(q);
            std::vector<T>& v = tab[q];
            for (int tr = 0; tr < 2; ++tr) {
                auto Mv = [&](int i, int m) { return tr ? D[m * n + i] : D[i * n + m]; };
                for (int i = 0; i < h; ++i)
                    for (int m = 0; m < h; ++m) v.push_back((T)(0.5 * (Mv(i, m) + Mv(i, n - 1 - m))));
                for (int i = 0; i < h; ++i)
                    for (int m = 0; m < h; ++m) v.push_back((T)(0.5 * (Mv(i, m) - Mv(i, n - 1 - m))));
                for (int i = 0; i < h; ++i) v.push_back((T)Mv(i, h));
                for (int m = 0; m < h; ++m) v.push_back((T)Mv(h, m));
            }
        }
    });
    return tab[p];
}

template <typename T, int N>
EoParams<T, N> eo_params() {
    static_assert(sizeof(EoParams<T, N>) == sizeof(T) * 2 * (2 * (N / 2) * (N / 2) + 2 * (N / 2)), "packed");
    EoParams<T, N> M;
    const std::vector<T>& v = eo_table<T>(N - 1);
    std::memcpy(&M, v.data(), sizeof(M));
    return M;
}

template <typename T, int P>
bool launch_eo(const DevLevel<T>& L, const T* x, T* y, bool mask, double* dot, double* part, unsigned* ticket,
               cudaStream_t st, int nrhs) {
    using S = EoShape<T, P + 1>;
    const EoParams<T, P + 1> M = eo_params<T, P + 1>();
    const int epb = eo_epb(P, L.E);
    const long long nb = (L.E + epb - 1) / epb * nrhs;
    if (nb > 0x7fffffffLL) return false;
    const int blocks = (int)nb;
    const int threads = (epb * S::NP + 31) / 32 * 32;
    const size_t smem = sizeof(T) * S::NBUF * epb * S::ES;
    if (dot) launch_k(apply_eo3_kernel<T, P, true>, blocks, threads, smem, st, L, M, x, y, mask ? 1 : 0, dot, part,
                      ticket, epb, nrhs);
    else launch_k(apply_eo3_kernel<T, P, false>, blocks, threads, smem, st, L, M, x, y, mask ? 1 : 0,
                  (double*)nullptr, (double*)nullptr, (unsigned*)nullptr, epb, nrhs);
    return true;
}

template <typename T, int P>
bool set_eo_attr() {
    using S = EoShape<T, P + 1>;
    const int smem = (int)(sizeof(T) * S::NBUF * S::EPB * S::ES);
    return cudaFuncSetAttribute((const void*)apply_eo3_kernel<T, P, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess &&
           cudaFuncSetAttribute((const void*)apply_eo3_kernel<T, P, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess;
}

}  // namespace

// Orders measured faster with this kernel than with the node-per-thread and
// column kernels on 16^3-element levels (graph replay and L2-cold launches):
// FP32 p >= 4 (p = 7: 15.1 against 16.4 and 24.4 us), FP64 p = 6, 7 (p = 7:
// 193 against 218 us).  FP64 elsewhere: the 2N adds per line and the lower
// thread count cost more than the saved multiply-adds.
bool apply_eo_selected(int dim, int p, bool f64) {
    if (dim != 3) return false;
    return f64 ? (p == 6 || p == 7) : (p >= 4 && p <= 8);
}

// Number of CTAs (= dot partials) of the even-odd kernel for L.
int apply_eo_blocks(int p, long long E) {
    const int epb = eo_epb(p, E);
    return (int)((E + epb - 1) / epb);
}

template <typename T>
bool launch_apply_eo(const DevLevel<T>& L, const T* x, T* y, bool mask, double* dot, double* part,
                     unsigned* ticket, cudaStream_t st, int nrhs) {
    if (!apply_eo_selected(L.dim, L.p, sizeof(T) == 8)) return false;
    if constexpr (sizeof(T) == 8) {
        switch (L.p) {
            case 6: return launch_eo<T, 6>(L, x, y, mask, dot, part, ticket, st, nrhs);
            default: return launch_eo<T, 7>(L, x, y, mask, dot, part, ticket, st, nrhs);
        }
    } else {
        switch (L.p) {
            case 4: return launch_eo<T, 4>(L, x, y, mask, dot, part, ticket, st, nrhs);
            case 5: return launch_eo<T, 5>(L, x, y, mask, dot, part, ticket, st, nrhs);
            case 6: return launch_eo<T, 6>(L, x, y, mask, dot, part, ticket, st, nrhs);
            case 7: return launch_eo<T, 7>(L, x, y, mask, dot, part, ticket, st, nrhs);
            default: return launch_eo<T, 8>(L, x, y, mask, dot, part, ticket, st, nrhs);
        }
    }
}
template bool launch_apply_eo<float>(const DevLevel<float>&, const float*, float*, bool, double*, double*,
                                     unsigned*, cudaStream_t, int);
template bool launch_apply_eo<double>(const DevLevel<double>&, const double*, double*, bool, double*, double*,
                                      unsigned*, cudaStream_t, int);

bool init_apply_eo_attributes() {
    return set_eo_attr<float, 4>() && set_eo_attr<float, 5>() && set_eo_attr<float, 6>() && set_eo_attr<float, 7>() &&
           set_eo_attr<float, 8>() && set_eo_attr<double, 6>() && set_eo_attr<double, 7>();
}

}  // namespace glls
