// Cyclic reduction of one tridiagonal system per warp, in registers.
//
// Each lane holds a contiguous chunk of C unknowns (unknown k = C lane + j).
// The odd-even order of Algorithm 1 / Thm. 3.8 / Cor. 3.9 is kept: at level h
// the odd multiples of h are eliminated into the even ones with the Prop. 3.7
// coefficients
//   a' = a - l u_{i-h}/a_{i-h} - u l_{i+h}/a_{i+h},  l' = -l l_{i-h}/a_{i-h},
//   u' = -u u_{i+h}/a_{i+h},  g' = g - l g_{i-h}/a_{i-h} - u g_{i+h}/a_{i+h},
// and the back substitution restores x_i = (g_i - l_i x_{i-h} - u_i x_{i+h})/a_i.
// Each eliminated unknown's pivot is inverted once (1/a_i, reused by both
// neighbours and by the back substitution).  Levels h < C run inside a lane
// (one shuffle brings the next lane's neighbour), levels h >= C across lanes
// with shuffles at distance h / C.  Unknowns past the end of the system are
// decoupled identity rows (a = 1, l = u = g = 0), which leaves every real
// unknown's arithmetic unchanged.  All 32 lanes must take part.
#pragma once
#include <cuda_runtime.h>

namespace glls {

constexpr unsigned kFullMask = 0xffffffffu;

// 1 / a: in FP32 the hardware approximate reciprocal (one instruction on
// the reduction's critical path, at most 1 ulp from the rounded quotient;
// pivots are never subnormal), in FP64 a division.
__device__ __forceinline__ float recip(float a) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ double recip(double a) { return 1.0 / a; }

// Solves the warp's system; on return g holds the solution (a, l, u are
// overwritten).
template <typename T, int C>
__device__ __forceinline__ void warp_cr_solve(T (&a)[C], T (&l)[C], T (&u)[C], T (&g)[C], int lane) {
    // ---- forward reduction inside the lane: h = 1, 2, ..., C/2
#pragma unroll
    for (int h = 1; h < C; h *= 2) {
        // the odd points of this level are eliminated: keep 1/a from here on
#pragma unroll
        for (int j = h - 1; j < C; j += 2 * h) a[j] = recip(a[j]);
        // the next lane's first odd point, premultiplied by its 1/a
        T lr = __shfl_down_sync(kFullMask, a[h - 1] * l[h - 1], 1);
        T ur = __shfl_down_sync(kFullMask, a[h - 1] * u[h - 1], 1);
        T gr = __shfl_down_sync(kFullMask, a[h - 1] * g[h - 1], 1);
        if (lane == 31) { lr = T(0); ur = T(0); gr = T(0); }
#pragma unroll
        for (int j = 2 * h - 1; j < C; j += 2 * h) {
            const int jl = j - h, jr = j + h;
            const int jr0 = jr < C ? jr : 0;
            // right odd point's couplings times its reciprocal
            const T lR = jr < C ? a[jr0] * l[jr0] : lr;
            const T uR = jr < C ? a[jr0] * u[jr0] : ur;
            const T gR = jr < C ? a[jr0] * g[jr0] : gr;
            const T al = -l[j] * a[jl];
            const T mu = -u[j];
            a[j] = a[j] + al * u[jl] + mu * lR;
            g[j] = g[j] + al * g[jl] + mu * gR;
            l[j] = al * l[jl];
            u[j] = mu * uR;
        }
    }
    // ---- forward reduction across lanes on each lane's top unknown (position C (lane+1))
    T At = a[C - 1], Lt = l[C - 1], Ut = u[C - 1], Gt = g[C - 1];
#pragma unroll
    for (int d = 1; d < 32; d *= 2) {
        // a lane eliminated at this level sends its couplings premultiplied
        // by its reciprocal pivot: 3 values each way instead of 4
        const bool odd = ((lane + 1) & (2 * d - 1)) == d;
        if (odd) At = recip(At);
        const T pl = At * Lt, pu = At * Ut, pg = At * Gt;
        const T lL = __shfl_up_sync(kFullMask, pl, d), uL = __shfl_up_sync(kFullMask, pu, d);
        const T gL = __shfl_up_sync(kFullMask, pg, d);
        T lR = __shfl_down_sync(kFullMask, pl, d), uR = __shfl_down_sync(kFullMask, pu, d);
        T gR = __shfl_down_sync(kFullMask, pg, d);
        if (lane + d > 31) { lR = T(0); uR = T(0); gR = T(0); }
        if (((lane + 1) & (2 * d - 1)) == 0) {
            const T ml = -Lt, mu = -Ut;
            At = At + ml * uL + mu * lR;
            Gt = Gt + ml * gL + mu * gR;
            Lt = ml * lL;
            Ut = mu * uR;
        }
    }
    // ---- top equation (position 32 C) and back substitution across lanes
    T X = lane == 31 ? Gt * recip(At) : T(0);
#pragma unroll
    for (int d = 16; d >= 1; d /= 2) {
        T xl = __shfl_up_sync(kFullMask, X, d);
        T xr = __shfl_down_sync(kFullMask, X, d);
        if (lane - d < 0) xl = T(0);
        if (lane + d > 31) xr = T(0);
        if (((lane + 1) & (2 * d - 1)) == d) X = (Gt - Lt * xl - Ut * xr) * At;
    }
    // ---- back substitution inside the lane
    g[C - 1] = X;
    T xprev = __shfl_up_sync(kFullMask, X, 1);
    if (lane == 0) xprev = T(0);
#pragma unroll
    for (int h = C / 2; h >= 1; h /= 2) {
#pragma unroll
        for (int j = h - 1; j < C; j += 2 * h) {
            const T xl = j - h >= 0 ? g[j - h >= 0 ? j - h : 0] : xprev;
            const T xr = g[j + h < C ? j + h : C - 1];
            g[j] = (g[j] - l[j] * xl - u[j] * xr) * a[j];
        }
    }
}

}  // namespace glls
