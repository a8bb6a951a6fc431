// Device building blocks of the Krylov loop: complex arithmetic, block-row
// products, CTA column sums and the bounded grid barrier.
#pragma once

#include "fe_internal.cuh"

namespace fe {

template <typename T>
struct CplxT;
template <>
struct CplxT<float> {
    using type = float2;
};
template <>
struct CplxT<double> {
    using type = double2;
};

__device__ __forceinline__ float2 mk(float r, float i) { return make_float2(r, i); }
__device__ __forceinline__ double2 mk(double r, double i) { return make_double2(r, i); }

// Loads: matrix data never changes inside a launch (read-only path); vectors
// written by other CTAs earlier in the same launch bypass L1 (.cg).
template <typename C>
__device__ __forceinline__ C ld_ro(const C* p) {
    return __ldg(p);
}
template <typename C>
__device__ __forceinline__ C ld_cg(const C* p) {
    return __ldcg(p);
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Warp-per-row product of one block row with a single vector (R = 1): lanes
// walk the row's 9*(s1-s0) complex entries in order, so every load of the
// matrix is a coalesced 32-entry stretch; each lane accumulates into the
// output component alpha of its entry, then a butterfly leaves the three
// row results in every lane.
template <typename C, bool kCoherentX>
__device__ __forceinline__ void row_product_r1(const C* __restrict__ val, const int* __restrict__ col, int s0, int s1,
                                               const C* x, int lane, C& y0, C& y1, C& y2) {
    using Tr = decltype(C{}.x);
    Tr a0r = 0, a0i = 0, a1r = 0, a1i = 0, a2r = 0, a2i = 0;
    int slot = s0 + lane / 9;
    int w = lane % 9;
    const int end = s1 * 9;
#pragma unroll 4
    for (int e = s0 * 9 + lane; e < end; e += 32) {
        const C v = ld_ro(val + e);
        const int c = __ldg(col + slot);
        const int al = w / 3;
        const int be = w - 3 * al;
        const C xv = kCoherentX ? ld_cg(x + 3 * c + be) : ld_ro(x + 3 * c + be);
        const Tr pr = v.x * xv.x - v.y * xv.y;
        const Tr pi = v.x * xv.y + v.y * xv.x;
        if (al == 0) {
            a0r += pr;
            a0i += pi;
        } else if (al == 1) {
            a1r += pr;
            a1i += pi;
        } else {
            a2r += pr;
            a2i += pi;
        }
        w += 5;  // 32 = 3*9 + 5
        slot += 3;
        if (w >= 9) {
            w -= 9;
            slot += 1;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a0r += __shfl_xor_sync(0xffffffffu, a0r, o);
        a0i += __shfl_xor_sync(0xffffffffu, a0i, o);
        a1r += __shfl_xor_sync(0xffffffffu, a1r, o);
        a1i += __shfl_xor_sync(0xffffffffu, a1i, o);
        a2r += __shfl_xor_sync(0xffffffffu, a2r, o);
        a2i += __shfl_xor_sync(0xffffffffu, a2i, o);
    }
    y0 = mk(a0r, a0i);
    y1 = mk(a1r, a1i);
    y2 = mk(a2r, a2i);
}

// Product of one block row with column c of a multi-vector X [n_dof][ldx]:
// one lane per (row, column).
template <typename C, bool kCoherentX>
__device__ __forceinline__ void row_product_col(const C* __restrict__ val, const int* __restrict__ col, int s0, int s1,
                                                const C* x, int ldx, int c, C& y0, C& y1, C& y2) {
    using Tr = decltype(C{}.x);
    Tr a[6] = {0, 0, 0, 0, 0, 0};
    for (int s = s0; s < s1; ++s) {
        const int cb = __ldg(col + s);
        C xv[3];
#pragma unroll
        for (int be = 0; be < 3; ++be)
            xv[be] = kCoherentX ? ld_cg(x + (size_t)(3 * cb + be) * ldx + c) : ld_ro(x + (size_t)(3 * cb + be) * ldx + c);
#pragma unroll
        for (int al = 0; al < 3; ++al)
#pragma unroll
            for (int be = 0; be < 3; ++be) {
                const C v = ld_ro(val + (size_t)s * 9 + 3 * al + be);
                a[2 * al] += v.x * xv[be].x - v.y * xv[be].y;
                a[2 * al + 1] += v.x * xv[be].y + v.y * xv[be].x;
            }
    }
    y0 = mk(a[0], a[1]);
    y1 = mk(a[2], a[3]);
    y2 = mk(a[4], a[5]);
}

}  // namespace fe
