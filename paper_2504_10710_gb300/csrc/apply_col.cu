// 3-D FP32 stiffness apply y = A_l x (eq. discreteBilinear) for p <= 3 with
// one thread per (i, j) column of an element: the thread holds the column's N1 = p + 1
// values along the third axis in registers, so the t-contractions (forward
// D and transposed D^T) run on registers with D read as compile-time-indexed
// kernel parameters (constant-bank operands, no load instructions).  The r-
// and s-contractions read rows of the element's planes from shared memory:
// rows of the natural layout for r, rows of a per-plane transposed copy for
// s (float4 rows when N1 is a multiple of 4).  Each thread keeps the rows
// D[i][.], D[j][.], D[.][i] and D[.][j] it needs in registers.  The
// geometric factors are read once per node, coalesced along i.  Element-
// interior nodes are stored, shared nodes summed with atomics (direct
// stiffness summation), Dirichlet rows skipped when mask is set.
#include "device.cuh"
#include "setup.h"

#include <mutex>
#include <vector>

namespace glls {
namespace {

template <int N1>
struct DParam {
    float d[N1 * N1];   // D row-major, D[a][b] = d[a * N1 + b]
};

template <int P>
struct ColShape {
    static constexpr int N1 = P + 1, NP = N1 * N1, NLOC = NP * N1;
    static constexpr int EPB = 256 / NP;   // elements per CTA
    static constexpr bool VEC = N1 % 4 == 0;
    // row stride of the transposed planes and padding of the element blocks,
    // chosen so that every warp's row reads and column stores hit distinct
    // banks (one wavefront per instruction)
    static constexpr int RS = N1 == 4 ? 8 : N1;
    static constexpr int PAD = N1 == 2 ? 4 : N1 == 3 ? 14 : 16;
    static constexpr int SA = NLOC + PAD;                                  // natural element block
    static constexpr int SB = VEC ? NP * RS + (N1 == 4 ? 4 : 0) : SA;      // transposed element block
    static constexpr int PB = VEC ? N1 * RS : NP;                          // plane stride of the s-buffers
    static constexpr int MINB = 4;   // resident CTAs per SM the registers must allow (64 registers)
};

// sum_m a[m] row[m], m in order; row 16-byte aligned when VEC
template <int N1, bool VEC>
__device__ __forceinline__ float rowdot(const float (&a)[N1], const float* row) {
    float s = 0.f;
    if constexpr (VEC) {
        const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
        for (int q = 0; q < N1 / 4; ++q) {
            const float4 v = r4[q];
            s += a[4 * q] * v.x;
            s += a[4 * q + 1] * v.y;
            s += a[4 * q + 2] * v.z;
            s += a[4 * q + 3] * v.w;
        }
    } else {
#pragma unroll
        for (int m = 0; m < N1; ++m) s += a[m] * row[m];
    }
    return s;
}

// sum_m a[m] col[m * stride], m in order
template <int N1, int STRIDE>
__device__ __forceinline__ float coldot(const float (&a)[N1], const float* col) {
    float s = 0.f;
#pragma unroll
    for (int m = 0; m < N1; ++m) s += a[m] * col[m * STRIDE];
    return s;
}

template <int P>
__global__ void __launch_bounds__(256, ColShape<P>::MINB) apply_col_kernel(DevLevel<float> L, DParam<P + 1> Dk,
                                                           const float* __restrict__ x, float* __restrict__ y,
                                                           int mask, int nrhs) {
    grid_dep_sync();
    // right-hand side fastest in the CTA order (see device.cuh)
    const int rhs = blockIdx.x % nrhs, cta = blockIdx.x / nrhs;
    x += (long long)rhs * L.N;
    y += (long long)rhs * L.N;
    using S = ColShape<P>;
    constexpr int N1 = S::N1, NP = S::NP, NLOC = S::NLOC, EPB = S::EPB;
    constexpr bool VEC = S::VEC;
    constexpr int SA = S::SA, SB = S::SB, PB = S::PB, RS = S::RS;
    __shared__ __align__(16) float sx[EPB * SA];            // x, natural layout [k][j][i]
    __shared__ __align__(16) float sxt[VEC ? EPB * SB : 4];  // x, transposed planes [k][i][j]
    __shared__ __align__(16) float swr[EPB * SA];           // w_r, natural
    __shared__ __align__(16) float sws[EPB * SB];           // w_s, transposed planes (natural when !VEC)

    const int E = (int)L.E, n0 = L.n[0], n1 = L.n[1];
    const int nplane = n0 * n1;
    const int tid = threadIdx.x;
    const int el = tid / NP, c = tid - el * NP, i = c % N1, j = c / N1;
    const int e = cta * EPB + el;
    const bool act = el < EPB && e < E;
    int base = 0, I = 0, J = 0, K0 = 0;
    if (act) {
        const int ne0 = L.ne[0], ne1 = L.ne[1];
        const int ex = e % ne0, ey = (e / ne0) % ne1, ez = e / (ne0 * ne1);
        I = ex * P + i;
        J = ey * P + j;
        K0 = ez * P;
        base = (K0 * n1 + J) * n0 + I;
    }
    // column of x, and the D rows and columns this thread contracts with
    float xc[N1], Dr[N1], Ds[N1];
#pragma unroll
    for (int k = 0; k < N1; ++k) xc[k] = act ? __ldg(x + base + k * nplane) : 0.f;
#pragma unroll
    for (int m = 0; m < N1; ++m) {
        Dr[m] = __ldg(L.D + i * N1 + m);
        Ds[m] = __ldg(L.D + j * N1 + m);
    }
    const int elo = act ? el : 0;
    float* ax = sx + elo * SA;
    float* bx = sxt + (VEC ? elo * SB : 0);
    float* cw = swr + elo * SA;
    float* dw = sws + elo * SB;
    if (act) {
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            ax[k * NP + j * N1 + i] = xc[k];
            if constexpr (VEC) bx[k * PB + i * RS + j] = xc[k];
        }
    }
    __syncthreads();

    // reference gradient, geometric factors, w = G grad x
    float wt[N1];
    if (act) {
        const int EN = E * NLOC;
        const float* Gq = L.G + e * NLOC + c;
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            const float g0 = __ldg(Gq + k * NP), g1 = __ldg(Gq + EN + k * NP), g2 = __ldg(Gq + 2 * EN + k * NP);
            const float g3 = __ldg(Gq + 3 * EN + k * NP), g4 = __ldg(Gq + 4 * EN + k * NP);
            const float g5 = __ldg(Gq + 5 * EN + k * NP);
            const float ur = rowdot<N1, VEC>(Dr, ax + k * NP + j * N1);
            float us;
            if constexpr (VEC) us = rowdot<N1, true>(Ds, bx + k * PB + i * RS);
            else us = coldot<N1, N1>(Ds, ax + k * NP + i);
            float ut = 0.f;
#pragma unroll
            for (int m = 0; m < N1; ++m) ut += Dk.d[k * N1 + m] * xc[m];
            cw[k * NP + j * N1 + i] = g0 * ur + g1 * us + g2 * ut;
            const float ws = g1 * ur + g3 * us + g4 * ut;
            if constexpr (VEC) dw[k * PB + i * RS + j] = ws;
            else dw[k * NP + j * N1 + i] = ws;
            wt[k] = g2 * ur + g4 * us + g5 * ut;
        }
    }
    __syncthreads();

    // transposed contractions and direct stiffness summation (the D^T rows
    // are loaded here so that their registers are not live in the first pass)
    float DTr[N1], DTs[N1];
#pragma unroll
    for (int m = 0; m < N1; ++m) {
        DTr[m] = __ldg(L.D + m * N1 + i);
        DTs[m] = __ldg(L.D + m * N1 + j);
    }
    if (act) {
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            float v = rowdot<N1, VEC>(DTr, cw + k * NP + j * N1);
            if constexpr (VEC) v += rowdot<N1, true>(DTs, dw + k * PB + i * RS);
            else v += coldot<N1, N1>(DTs, dw + k * NP + i);
            float vt = 0.f;
#pragma unroll
            for (int m = 0; m < N1; ++m) vt += Dk.d[m * N1 + k] * wt[m];
            v += vt;
            const int g = base + k * nplane;
            const bool inner = i > 0 && i < P && j > 0 && j < P && k > 0 && k < P;
            if (inner) {
                y[g] = v;
            } else {
                const int K = K0 + k;
                const bool bd = I == 0 || I == n0 - 1 || J == 0 || J == n1 - 1 || K == 0 || K == L.n[2] - 1;
                if (!(mask && bd)) atomicAdd(&y[g], v);
            }
        }
    }
}

// D of order p in FP32 (the values the levels upload), built once per order
const float* d_table(int p) {
    static std::once_flag once;
    static std::vector<float> tab[4];
    std::call_once(once, [] {
        for (int q = 1; q <= 3; ++q) {
            const std::vector<double> D = derivative_matrix(q);
            tab[q].resize(D.size());
            for (size_t t = 0; t < D.size(); ++t) tab[q][t] = (float)D[t];
        }
    });
    return tab[p].data();
}

template <int P>
bool launch_col(const DevLevel<float>& L, const float* x, float* y, bool mask, cudaStream_t st, int nrhs) {
    DParam<P + 1> Dk;
    const float* d = d_table(P);
    for (int t = 0; t < (P + 1) * (P + 1); ++t) Dk.d[t] = d[t];
    constexpr int EPB = ColShape<P>::EPB;
    const long long nb = (L.E + EPB - 1) / EPB * nrhs;
    if (nb > 0x7fffffffLL) return false;
    launch_k(apply_col_kernel<P>, (unsigned)nb, 256, 0, st, L, Dk, x, y, mask ? 1 : 0, nrhs);
    return true;
}

template <int P>
bool prefer_shared() {
    return cudaFuncSetAttribute((const void*)apply_col_kernel<P>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared) == cudaSuccess;
}

}  // namespace

// Shared-memory carveout for the column apply (p <= 3: up to 27 KB per CTA).
bool init_apply_col_attributes() { return prefer_shared<1>() && prefer_shared<2>() && prefer_shared<3>(); }

bool launch_apply_col(const DevLevel<float>& L, const float* x, float* y, bool mask, cudaStream_t st, int nrhs) {
    if (L.dim != 3 || L.p < 1 || L.p > 3) return false;
    switch (L.p) {
        case 1: return launch_col<1>(L, x, y, mask, st, nrhs);
        case 2: return launch_col<2>(L, x, y, mask, st, nrhs);
        default: return launch_col<3>(L, x, y, mask, st, nrhs);
    }
}

}  // namespace glls
