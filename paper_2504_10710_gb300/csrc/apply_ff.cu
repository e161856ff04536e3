// The outer iteration's 2-D apply q = A_L p with the per-CTA partial sums of
// p.(A p), computed in float-float arithmetic (ff.cuh) instead of FP64: the
// same sum factorisation as apply_p_kernel (1-D contractions with D, the
// pointwise geometric factors G, the transposed contractions; eq.
// discreteBilinear), every product and sum on FP32 pairs.  GB300 issues FP32
// fused multiply-adds at 64 times its FP64 rate, so about 12 FP32 operations
// per FP64 multiply-add still leave the kernel faster than the FP64 one, which
// is FP64-pipe bound (measured 1.8 times in 2-D at p = 8, 2.7 times in 3-D at
// p = 7, where the even-odd sweeps below also apply); the result carries about 48 bits
// (relative rounding near 2^-44 per contraction), which moves the point at
// which the flexible-CG recurrence residual and the true residual part to
// about 1e-13 relative, below the solver tolerances it is used with.
// p is read and q written as FP64 (the outer Krylov vectors); G is the FP32
// level's factors (the FP64 factors rounded to nearest) plus their FP32
// rounding remainders, D is split from the FP64 matrix per CTA; element-
// interior nodes are stored, shared nodes summed with FP64 atomics, the dot
// partial accumulated in FP64 from the FP64 values.
//
// 3-D: the same product with one thread per element grid line and the 1-D
// sweeps in even-odd form (the centro-antisymmetry of the GLL
// differentiation matrix, D[N-1-i][N-1-m] = -D[i][m], halves the multiply-
// adds of a line: with u_e[m] = u[m] + u[N-1-m] and u_o[m] = u[m] - u[N-1-m],
// (Du)[i] = a_i + b_i and (Du)[N-1-i] = b_i - a_i for a_i, b_i the products of
// u_e, u_o with the even and odd halves of D), the coefficients as kernel
// parameters, the three line directions of an element through shared memory.
#include "device.cuh"
#include "ff.cuh"
#include "setup.h"

#include <algorithm>
#include <mutex>
#include <vector>

namespace glls {
namespace {

// Block sum of one FP64 value per thread (blockDim.x <= 256, a multiple of
// 32) with few FP64 adds: the values go through shared memory, lane l of
// warp 0 adds values l, l + 32, ... in that order, then warp 0's shuffle
// tree.  A shuffle tree over every warp would cost each thread five FP64
// adds, which on GB300's FP64 pipe is a visible share of these kernels.
__device__ __forceinline__ double block_sum_lean(double v, double* sv) {
    sv[threadIdx.x] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        for (int i = threadIdx.x; i < (int)blockDim.x; i += 32) s += sv[i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;   // valid in thread 0
}

template <int P>
__device__ __forceinline__ void apply_ff_body(const DevLevel<double>& L, const double* __restrict__ x,
                                              double* __restrict__ y, int mask, double* part, int nrhs, int blk,
                                              int nblk) {
    const int rhs = blk % nrhs, bx = blk / nrhs, nbx = nblk / nrhs;
    x += (long long)rhs * L.N;
    y += (long long)rhs * L.N;
    constexpr int N1 = P + 1;
    constexpr int NLOC = N1 * N1;
    constexpr int EPB = NLOC >= 256 ? 1 : 256 / NLOC;
    constexpr int ITEMS = (EPB * NLOC + 255) / 256;
    __shared__ ffloat sD[N1 * N1];
    __shared__ ffloat sx[EPB * NLOC];
    __shared__ ffloat sw[2 * EPB * NLOC];
    __shared__ int sbase[EPB];   // global index of each element's first node
    __shared__ int sxy[EPB];     // element coordinates packed 16:16 bits
    const int E = (int)L.E;
    const int n0 = L.n[0];
    const int EN = E * NLOC;
    const int e0 = bx * EPB;
    const int total = min(EPB, E - e0) * NLOC;
    if (threadIdx.x < EPB && e0 + (int)threadIdx.x < E) {
        const int e = e0 + threadIdx.x, ne0 = L.ne[0];
        const int ex = e % ne0, ey = e / ne0;
        sbase[threadIdx.x] = ey * P * n0 + ex * P;
        sxy[threadIdx.x] = ex | (ey << 16);
    }
    ffloat gk[ITEMS][3];
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const int t = threadIdx.x + 256 * it;
        if (t < total) {
            const int gq = e0 * NLOC + t;
#pragma unroll
            for (int c = 0; c < 3; ++c) gk[it][c] = {__ldg(L.Ghi + c * EN + gq), __ldg(L.Glo + c * EN + gq)};
        }
    }
    for (int t = threadIdx.x; t < N1 * N1; t += 256) sD[t] = ff_from_double(L.D[t]);
    __syncthreads();
    double xd[ITEMS];
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const int t = threadIdx.x + 256 * it;
        xd[it] = 0.0;
        if (t < total) {
            const int el = t / NLOC, q = t - el * NLOC;
            const int i = q % N1, j = q / N1;
            xd[it] = x[sbase[el] + j * n0 + i];
            sx[t] = ff_from_double(xd[it]);
        }
    }
    __syncthreads();

#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const int t = threadIdx.x + 256 * it;
        if (t >= total) break;
        const int el = t / NLOC, q = t - el * NLOC;
        const int i = q % N1, j = q / N1;
        const ffloat* xe = sx + el * NLOC;
        ffloat g0 = {0.f, 0.f}, g1 = {0.f, 0.f};
#pragma unroll
        for (int m = 0; m < N1; ++m) {
            ff_mac(g0, sD[i * N1 + m], xe[j * N1 + m]);
            ff_mac(g1, sD[j * N1 + m], xe[m * N1 + i]);
        }
        g0 = ff_norm(g0);
        g1 = ff_norm(g1);
        const ffloat* a = gk[it];
        ffloat w0 = {0.f, 0.f}, w1 = {0.f, 0.f};
        ff_mac(w0, a[0], g0);
        ff_mac(w0, a[1], g1);
        ff_mac(w1, a[1], g0);
        ff_mac(w1, a[2], g1);
        sw[t] = ff_norm(w0);
        sw[EPB * NLOC + t] = ff_norm(w1);
    }
    __syncthreads();

    double local = 0.0;
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const int t = threadIdx.x + 256 * it;
        if (t >= total) break;
        const int el = t / NLOC, q = t - el * NLOC;
        const int i = q % N1, j = q / N1;
        const ffloat* w0 = sw + el * NLOC;
        const ffloat* w1 = sw + EPB * NLOC + el * NLOC;
        ffloat v = {0.f, 0.f};
#pragma unroll
        for (int m = 0; m < N1; ++m) {
            ff_mac(v, sD[m * N1 + i], w0[j * N1 + m]);
            ff_mac(v, sD[m * N1 + j], w1[m * N1 + i]);
        }
        const double vd = ff_to_double(ff_norm(v));
        local += xd[it] * vd;
        const int exy = sxy[el];
        const int I = (exy & 0xffff) * P + i, J = (exy >> 16) * P + j;
        const int g = sbase[el] + j * n0 + i;
        const bool inner = i > 0 && i < P && j > 0 && j < P;
        if (inner) {
            y[g] = vd;
        } else {
            if (mask && (I == 0 || I == n0 - 1 || J == 0 || J == L.n[1] - 1)) continue;
            atomicAdd(&y[g], vd);
        }
    }
    __shared__ double sv[256];
    const double tsum = block_sum_lean(local, sv);
    if (threadIdx.x == 0) part[(long long)rhs * nbx + bx] = tsum;
}

template <int P>
__global__ void __launch_bounds__(256, 1) apply_ff_kernel(DevLevel<double> L, const double* __restrict__ x,
                                                          double* __restrict__ y, int mask, double* part, int nrhs) {
    grid_dep_sync();
    apply_ff_body<P>(L, x, y, mask, part, nrhs, blockIdx.x, gridDim.x);
}

// Work-list form: item j owns the CTAs [start[j], start[j + 1]).
template <int P>
__global__ void __launch_bounds__(256, 1) apply_ff_list_kernel(const ApplyItem<double>* __restrict__ items,
                                                               const int* __restrict__ start, int nitems, int mask) {
    grid_dep_sync();
    const int j = work_item(start, nitems, blockIdx.x);
    const ApplyItem<double>& it = items[j];
    if (it.done && *it.done != 0.0) return;
    apply_ff_body<P>(it.L, it.x, it.y, mask, it.part, 1, blockIdx.x - start[j], start[j + 1] - start[j]);
}

template <int P>
bool launch_ff(int p, const DevLevel<double>& L, const double* x, double* y, bool mask, double* part,
               cudaStream_t st, int nrhs) {
    if constexpr (P < 2) {
        return false;
    } else {
        if (p != P) return launch_ff<P - 1>(p, L, x, y, mask, part, st, nrhs);
        constexpr int NLOC = (P + 1) * (P + 1);
        constexpr int EPB = NLOC >= 256 ? 1 : 256 / NLOC;
        const long long blocks = (L.E + EPB - 1) / EPB * nrhs;
        if (blocks > 0x7fffffffLL) return false;
        return launch_k(apply_ff_kernel<P>, (unsigned)blocks, 256, 0, st, L, x, y, mask ? 1 : 0, part, nrhs) ==
               cudaSuccess;
    }
}

template <int P>
bool launch_ff_list(int p, const ApplyItem<double>* items, const int* start, int nitems, int blocks, bool mask,
                    cudaStream_t st) {
    if constexpr (P < 2) {
        return false;
    } else {
        if (p != P) return launch_ff_list<P - 1>(p, items, start, nitems, blocks, mask, st);
        return launch_k(apply_ff_list_kernel<P>, (unsigned)blocks, 256, 0, st, items, start, nitems,
                        mask ? 1 : 0) == cudaSuccess;
    }
}

// ---- 3-D, even-odd line sweeps ---------------------------------------------

// Elements per CTA: at most 192 threads (three CTAs per SM at 96 registers
// a thread; with two CTAs of 256 threads the kernel ran at 128 registers and
// 18 % warp occupancy), and no more elements than keep about eight CTAs per
// SM on the level (152 SMs).
constexpr int kEoFfThreads = 192;
int eo_ff_epb(int p, long long E) {
    const long long most = kEoFfThreads / ((p + 1) * (p + 1));
    const long long fill = E / (152 * 8);
    return (int)std::max(1LL, std::min(most, fill));
}

// D (f) and D^T (t) in even-odd form, float-float (H = N / 2)
template <int N>
struct EoMatFF {
    static constexpr int H = N / 2;
    ffloat e[H * H];   // (M[i][m] + M[i][N-1-m]) / 2, i, m < H
    ffloat o[H * H];   // (M[i][m] - M[i][N-1-m]) / 2
    ffloat c[H];       // M[i][h], N odd
    ffloat r[H];       // M[h][m], N odd
};
template <int N>
struct EoParamsFF {
    EoMatFF<N> f, t;
};

template <int N>
__device__ __forceinline__ void eo_line_ff(const EoMatFF<N>& M, const ffloat (&u)[N], ffloat (&out)[N]) {
    constexpr int H = N / 2;
    constexpr bool ODD = (N & 1) != 0;
    ffloat ue[H], uo[H];
#pragma unroll
    for (int m = 0; m < H; ++m) {
        ue[m] = ff_add(u[m], u[N - 1 - m]);
        uo[m] = ff_sub(u[m], u[N - 1 - m]);
    }
#pragma unroll
    for (int i = 0; i < H; ++i) {
        ffloat a = {0.f, 0.f}, b = {0.f, 0.f};
        if constexpr (ODD) ff_mac(a, M.c[i], u[H]);
#pragma unroll
        for (int m = 0; m < H; ++m) {
            ff_mac(a, M.e[i * H + m], ue[m]);
            ff_mac(b, M.o[i * H + m], uo[m]);
        }
        a = ff_norm(a);
        b = ff_norm(b);
        out[i] = ff_add(a, b);
        out[N - 1 - i] = ff_sub(b, a);
    }
    if constexpr (ODD) {
        ffloat sum = {0.f, 0.f};
#pragma unroll
        for (int m = 0; m < H; ++m) ff_mac(sum, M.r[m], uo[m]);
        out[H] = ff_norm(sum);
    }
}

// Shared-memory strides for 8-byte values (row RS, plane PS, element ES),
// spread over the banks as for the FP64 even-odd kernel.
template <int N>
struct EoShapeFF {
    static constexpr int NP = N * N, NLOC = NP * N;
    static constexpr int EPB = kEoFfThreads / NP;
    static constexpr int RS = N == 8 ? 9 : N == 7 ? 7 : N == 6 ? 9 : N;
    static constexpr int PS = N == 3 ? 9 : N == 4 ? 19 : N == 5 ? 25 : N == 6 ? 54 : N == 7 ? 52 : N == 8 ? 72 : 89;
    static constexpr int ES = N == 3 ? 27 : N == 4 ? 76 : N == 5 ? 125 : N == 6 ? 324 : N == 7 ? 369 : N == 8 ? 576 : 801;
};

// Thread (a, b) of an element owns the t-line (i, j) = (a, b) in registers
// and the r-line (j, k) = (a, b) and s-line (i, k) = (a, b) through shared
// memory (X: x, U, V: the r and s work buffers).
template <int P>
__global__ void __launch_bounds__(kEoFfThreads, 3)
    apply_eo3_ff_kernel(DevLevel<double> L, const __grid_constant__ EoParamsFF<P + 1> M, const double* __restrict__ x,
                        double* __restrict__ y, int mask, double* part, int epb, int nrhs) {
    using S = EoShapeFF<P + 1>;
    constexpr int N = P + 1, NP = S::NP, NLOC = S::NLOC, RS = S::RS, PS = S::PS, ES = S::ES;
    extern __shared__ __align__(16) unsigned char eo_ff_smem[];
    ffloat* sX = reinterpret_cast<ffloat*>(eo_ff_smem);
    ffloat* sU = sX + epb * ES;
    ffloat* sV = sU + epb * ES;
    grid_dep_sync();
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
    ffloat* X = sX + elo * ES;
    ffloat* U = sU + elo * ES;
    ffloat* V = sV + elo * ES;
    int base = 0, I = 0, J = 0, K0 = 0;
    ffloat xc[N], ut[N];
    if (act) {
        const int ne0 = L.ne[0], ne1 = L.ne[1];
        const int ex = e % ne0, ey = (e / ne0) % ne1, ez = e / (ne0 * ne1);
        I = ex * P + a;
        J = ey * P + b;
        K0 = ez * P;
        base = (K0 * n1 + J) * n0 + I;
#pragma unroll
        for (int k = 0; k < N; ++k) xc[k] = ff_from_double(x[base + k * nplane]);
#pragma unroll
        for (int k = 0; k < N; ++k) X[k * PS + b * RS + a] = xc[k];
        eo_line_ff<N>(M.f, xc, ut);
    }
    __syncthreads();
    if (act) {
        ffloat u[N], v[N];
#pragma unroll
        for (int m = 0; m < N; ++m) u[m] = X[b * PS + a * RS + m];
        eo_line_ff<N>(M.f, u, v);
#pragma unroll
        for (int m = 0; m < N; ++m) U[b * PS + a * RS + m] = v[m];
#pragma unroll
        for (int m = 0; m < N; ++m) u[m] = X[b * PS + m * RS + a];
        eo_line_ff<N>(M.f, u, v);
#pragma unroll
        for (int m = 0; m < N; ++m) V[b * PS + m * RS + a] = v[m];
    }
    __syncthreads();
    ffloat yt[N];
    if (act) {
        // node (a, b, k): w = G grad x over the node's U, V slots and the t-line
        const int EN = E * NLOC;
        const int gi = e * NLOC + c;
        ffloat wt[N];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            ffloat g[6];
#pragma unroll
            for (int q = 0; q < 6; ++q)
                g[q] = {__ldg(L.Ghi + q * EN + gi + k * NP), __ldg(L.Glo + q * EN + gi + k * NP)};
            const int s = k * PS + b * RS + a;
            const ffloat dr = U[s], ds = V[s], dt = ut[k];
            ffloat wr = {0.f, 0.f}, ws = {0.f, 0.f}, w3 = {0.f, 0.f};
            ff_mac(wr, g[0], dr);
            ff_mac(wr, g[1], ds);
            ff_mac(wr, g[2], dt);
            ff_mac(ws, g[1], dr);
            ff_mac(ws, g[3], ds);
            ff_mac(ws, g[4], dt);
            ff_mac(w3, g[2], dr);
            ff_mac(w3, g[4], ds);
            ff_mac(w3, g[5], dt);
            U[s] = ff_norm(wr);
            V[s] = ff_norm(ws);
            wt[k] = ff_norm(w3);
        }
        eo_line_ff<N>(M.t, wt, yt);
    }
    __syncthreads();
    if (act) {
        ffloat u[N], v[N];
#pragma unroll
        for (int m = 0; m < N; ++m) u[m] = U[b * PS + a * RS + m];
        eo_line_ff<N>(M.t, u, v);
#pragma unroll
        for (int m = 0; m < N; ++m) U[b * PS + a * RS + m] = v[m];
#pragma unroll
        for (int m = 0; m < N; ++m) u[m] = V[b * PS + m * RS + a];
        eo_line_ff<N>(M.t, u, v);
#pragma unroll
        for (int m = 0; m < N; ++m) V[b * PS + m * RS + a] = v[m];
    }
    __syncthreads();
    double local = 0.0;
    if (act) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const int s = k * PS + b * RS + a;
            const double v = ff_to_double(ff_add(ff_add(yt[k], U[s]), V[s]));
            const int g = base + k * nplane;
            local += x[g] * v;
            if (a > 0 && a < P && b > 0 && b < P && k > 0 && k < P) {
                y[g] = v;
            } else {
                const int K = K0 + k;
                if (mask && (I == 0 || I == n0 - 1 || J == 0 || J == n1 - 1 || K == 0 || K == L.n[2] - 1)) continue;
                atomicAdd(&y[g], v);
            }
        }
    }
    __shared__ double sv[kEoFfThreads];
    const double tsum = block_sum_lean(local, sv);
    if (tid == 0) part[(long long)rhs * nbx + bx] = tsum;
}

// Even-odd tables of D and D^T of order P, split into float-float
template <int N>
EoParamsFF<N> eo_ff_params() {
    static std::once_flag once;
    static EoParamsFF<N> M;
    std::call_once(once, [] {
        constexpr int H = N / 2;
        const std::vector<double> D = derivative_matrix(N - 1);
        auto split = [](double v) {
            const float hi = (float)v;
            return ffloat{hi, (float)(v - (double)hi)};
        };
        for (int tr = 0; tr < 2; ++tr) {
            EoMatFF<N>& T = tr ? M.t : M.f;
            auto Mv = [&](int i, int m) { return tr ? D[m * N + i] : D[i * N + m]; };
            for (int i = 0; i < H; ++i)
                for (int m = 0; m < H; ++m) {
                    T.e[i * H + m] = split(0.5 * (Mv(i, m) + Mv(i, N - 1 - m)));
                    T.o[i * H + m] = split(0.5 * (Mv(i, m) - Mv(i, N - 1 - m)));
                }
            for (int i = 0; i < H; ++i) T.c[i] = split(Mv(i, H));
            for (int m = 0; m < H; ++m) T.r[m] = split(Mv(H, m));
        }
    });
    return M;
}

template <int P>
bool launch_eo_ff_p(int p, const DevLevel<double>& L, const double* x, double* y, bool mask, double* part,
                    cudaStream_t st, int nrhs) {
    if constexpr (P < 2) {
        return false;
    } else {
        if (p != P) return launch_eo_ff_p<P - 1>(p, L, x, y, mask, part, st, nrhs);
        using S = EoShapeFF<P + 1>;
        static std::once_flag attr_once;
        static bool attr_ok = false;
        std::call_once(attr_once, [] {
            attr_ok = cudaFuncSetAttribute((const void*)apply_eo3_ff_kernel<P>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(sizeof(ffloat) * 3 * S::EPB * S::ES)) == cudaSuccess;
        });
        if (!attr_ok) return false;
        const EoParamsFF<P + 1> M = eo_ff_params<P + 1>();
        const int epb = eo_ff_epb(P, L.E);
        const long long nb = (L.E + epb - 1) / epb * nrhs;
        if (nb > 0x7fffffffLL) return false;
        const int threads = (epb * S::NP + 31) / 32 * 32;
        const size_t smem = sizeof(ffloat) * 3 * epb * S::ES;
        return launch_k(apply_eo3_ff_kernel<P>, (unsigned)nb, threads, smem, st, L, M, x, y, mask ? 1 : 0, part,
                        epb, nrhs) == cudaSuccess;
    }
}

}  // namespace

bool apply_ff_supported(const DevLevel<double>& L) {
    if (!L.Ghi || !L.Glo || L.colored || L.p < 2) return false;
    if (L.dim == 2) {
        if (L.p > 16 || L.ne[0] >= 0x10000 || L.ne[1] >= 0x10000) return false;
    } else {
        if (L.p > 8) return false;
    }
    return L.N <= (1LL << 31) - 1 && L.E * L.nloc * (L.dim == 2 ? 3 : 6) <= (1LL << 31) - 1 &&
           (long long)apply_ff_partials(L) <= (1LL << 24);
}

int apply_ff_partials(const DevLevel<double>& L) {
    if (L.dim == 3) {
        const int epb = eo_ff_epb(L.p, L.E);
        return (int)((L.E + epb - 1) / epb);
    }
    const long long nloc = (long long)(L.p + 1) * (L.p + 1);
    const long long epb = nloc >= 256 ? 1 : 256 / nloc;
    return (int)((L.E + epb - 1) / epb);
}

bool launch_apply_ff(const DevLevel<double>& L, const double* x, double* y, bool mask, double* part,
                     cudaStream_t st, int nrhs) {
    if (!apply_ff_supported(L)) return false;
    if (L.dim == 3) return launch_eo_ff_p<8>(L.p, L, x, y, mask, part, st, nrhs);
    return launch_ff<16>(L.p, L, x, y, mask, part, st, nrhs);
}

bool launch_apply_ff_list(int p, const ApplyItem<double>* items, const int* start, int nitems, int blocks, bool mask,
                          cudaStream_t st) {
    if (nitems < 1 || blocks < 1) return true;
    return launch_ff_list<16>(p, items, start, nitems, blocks, mask, st);
}

}  // namespace glls
