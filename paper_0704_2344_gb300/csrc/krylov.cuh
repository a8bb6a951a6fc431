// Device building blocks of the Krylov loop: complex arithmetic, block-row
// products, CTA column sums and the bounded grid barrier.
#pragma once

#include <type_traits>

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

// Regular-row class stencils are used by the complex64 products only (the
// argument is the real or the complex inner type).
// Tag of the double-float inner precision: a complex value as FP32 pairs in
// one float4 (re_hi, im_hi, re_lo, im_lo) with hi = RN32(v), lo = RN32(v - hi).
struct DFloat {};
template <>
struct CplxT<DFloat> {
    using type = float4;
};

template <typename T>
constexpr bool kClassPath = std::is_same<T, float>::value || std::is_same<T, float2>::value ||
                            std::is_same<T, DFloat>::value || std::is_same<T, float4>::value;

// (sh, sl) += a * x for FP32 pairs a = (ah, al), x = (xh, xl).  The rounding
// error of ah*xh is exact with one FMA and collects the cross terms ah*xl and
// al*xh (al*xl, about 2^-48 relative, is dropped); the rounded product joins
// sh by Knuth's TwoSum, whose error term is exact as well (error-free
// transformations, Knuth, TAOCP vol. 2, 4.2.2; Ogita, Rump and Oishi, 2005).
// The _rn intrinsics keep the compiler from contracting or reordering them.
__device__ __forceinline__ void df_mac(float& sh, float& sl, float ah, float al, float xh, float xl) {
    const float p = __fmul_rn(ah, xh);
    float e = __fmaf_rn(ah, xh, -p);
    e = __fmaf_rn(ah, xl, e);
    e = __fmaf_rn(al, xh, e);
    const float t = __fadd_rn(sh, p);
    const float v = __fsub_rn(t, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, v)), __fsub_rn(p, v));
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(err, e));
}

// acc = (re_hi, re_lo, im_hi, im_lo) += m * x for complex FP32 pairs.
__device__ __forceinline__ void dfc_mac(float (&acc)[4], const float4& m, const float4& x) {
    df_mac(acc[0], acc[1], m.x, m.z, x.x, x.z);
    df_mac(acc[0], acc[1], -m.y, -m.w, x.y, x.w);
    df_mac(acc[2], acc[3], m.x, m.z, x.y, x.w);
    df_mac(acc[2], acc[3], m.y, m.w, x.x, x.z);
}

__device__ __forceinline__ float4 df_result(const float (&acc)[4]) { return make_float4(acc[0], acc[2], acc[1], acc[3]); }

// acc (4 floats as above) += m * x through a pointer.
__device__ __forceinline__ void dfc_mac4(float* acc, const float4& m, const float4& x) {
    df_mac(acc[0], acc[1], m.x, m.z, x.x, x.z);
    df_mac(acc[0], acc[1], -m.y, -m.w, x.y, x.w);
    df_mac(acc[2], acc[3], m.x, m.z, x.y, x.w);
    df_mac(acc[2], acc[3], m.y, m.w, x.x, x.z);
}

// (h, l) += (h2, l2): TwoSum of the high parts, the error and both low parts
// into l.
__device__ __forceinline__ void df_add(float& h, float& l, float h2, float l2) {
    const float t = __fadd_rn(h, h2);
    const float v = __fsub_rn(t, h);
    const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(t, v)), __fsub_rn(h2, v));
    h = t;
    l = __fadd_rn(l, __fadd_rn(l2, e));
}

// Canonical pair of h + l (TwoSum: h = RN(h + l), l = the exact remainder).
__device__ __forceinline__ void df_norm(float& h, float& l) {
    const float t = __fadd_rn(h, l);
    const float v = __fsub_rn(t, h);
    l = __fadd_rn(__fsub_rn(h, __fsub_rn(t, v)), __fsub_rn(l, v));
    h = t;
}

// ---- FP32-pair scalar arithmetic, for the per-column recurrence scalars of
// the FP32-pair solve.  On GB300 one dependent FP64 operation of a thread
// takes about 64 cycles and one FP32 operation about 5, so a chain of a few
// dozen FP64 operations that every CTA repeats after each grid reduction costs
// more than its FP32-pair equivalent.  A real pair is a float2 (h, l) with
// value h + l; a complex pair is a float4 (re_h, im_h, re_l, im_l) as in the
// vectors, or a DZ of two real pairs.
__device__ __forceinline__ float2 dd_fast_two_sum(float a, float b) {  // needs |a| >= |b| or a = 0 (Dekker)
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ float2 dd_two_sum(float a, float b) {  // Knuth's TwoSum
    const float s = __fadd_rn(a, b);
    const float v = __fsub_rn(s, a);
    return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v)));
}

// a + b, accurate under cancellation too: the two high parts and the two low
// parts by TwoSum, then two renormalisations (the accurate pair addition of
// Joldes, Muller and Popescu, ACM TOMS 2017, Algorithm 6)
__device__ __forceinline__ float2 dd_add(float2 a, float2 b) {
    const float2 s = dd_two_sum(a.x, b.x);
    const float2 t = dd_two_sum(a.y, b.y);
    const float2 u = dd_fast_two_sum(s.x, __fadd_rn(s.y, t.x));
    return dd_fast_two_sum(u.x, __fadd_rn(u.y, t.y));
}

__device__ __forceinline__ float2 dd_neg(float2 a) { return make_float2(-a.x, -a.y); }

// a b: the exact error of a.h b.h from one FMA, the cross terms added to it
// (a.l b.l, about 2^-48 relative, dropped)
__device__ __forceinline__ float2 dd_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    return dd_fast_two_sum(p, e);
}

// a / b: a first FP32 quotient, the remainder a - q1 b in pair arithmetic,
// and its quotient as the correction (Dekker, Numer. Math. 1971)
__device__ __forceinline__ float2 dd_div(float2 a, float2 b) {
    const float q1 = __fdiv_rn(a.x, b.x);
    const float2 r = dd_add(a, dd_neg(dd_mul(make_float2(q1, 0.f), b)));
    return dd_fast_two_sum(q1, __fdiv_rn(r.x, b.x));
}

struct DZ {
    float2 re, im;
};

__device__ __forceinline__ DZ dz_of(const float4& v) { return {make_float2(v.x, v.z), make_float2(v.y, v.w)}; }
__device__ __forceinline__ float4 dz_f4(const DZ& a) { return make_float4(a.re.x, a.im.x, a.re.y, a.im.y); }
__device__ __forceinline__ DZ dz_add(const DZ& a, const DZ& b) { return {dd_add(a.re, b.re), dd_add(a.im, b.im)}; }
__device__ __forceinline__ DZ dz_sub(const DZ& a, const DZ& b) {
    return {dd_add(a.re, dd_neg(b.re)), dd_add(a.im, dd_neg(b.im))};
}
__device__ __forceinline__ DZ dz_mul(const DZ& a, const DZ& b) {
    return {dd_add(dd_mul(a.re, b.re), dd_neg(dd_mul(a.im, b.im))), dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re))};
}

// a / b by Smith's method (Comm. ACM 1962): no square of b is formed, so the
// FP32 exponent range holds whenever a, b and the quotient do.
__device__ __forceinline__ DZ dz_div(const DZ& a, const DZ& b) {
    const float2 one = make_float2(1.f, 0.f);
    if (fabsf(b.re.x) >= fabsf(b.im.x)) {
        const float2 t = dd_div(b.im, b.re);
        const float2 inv = dd_div(one, dd_add(b.re, dd_mul(b.im, t)));
        return {dd_mul(dd_add(a.re, dd_mul(a.im, t)), inv), dd_mul(dd_add(a.im, dd_neg(dd_mul(a.re, t))), inv)};
    }
    const float2 t = dd_div(b.re, b.im);
    const float2 inv = dd_div(one, dd_add(dd_mul(b.re, t), b.im));
    return {dd_mul(dd_add(dd_mul(a.re, t), a.im), inv), dd_mul(dd_add(dd_mul(a.im, t), dd_neg(a.re)), inv)};
}

// a finite, nonzero complex pair (its high parts decide)
__device__ __forceinline__ bool dz_usable(const DZ& a) {
    const float m = fabsf(a.re.x) + fabsf(a.im.x);
    return m > 0.f && m <= 3.0e38f;
}

// Accumulator -> stored complex FP32 pair, renormalised.
__device__ __forceinline__ float4 df_result_norm(float (&acc)[4]) {
    df_norm(acc[0], acc[1]);
    df_norm(acc[2], acc[3]);
    return make_float4(acc[0], acc[2], acc[1], acc[3]);
}

// y + a * x for complex FP32 pairs.
__device__ __forceinline__ float4 dfc_axpy(const float4& y, const float4& a, const float4& x) {
    float acc[4] = {y.x, y.z, y.y, y.w};
    dfc_mac(acc, a, x);
    return df_result_norm(acc);
}

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

}  // namespace fe

namespace fe {

// ---------------------------------------------------------------------------
// Bulk (TMA) copies global -> shared completed on an mbarrier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* mbar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(mbar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of the mbarrier; gives up after timeout_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mbar, unsigned parity, unsigned long long timeout_ns) {
    if (mbar_try_wait(mbar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (!mbar_try_wait(mbar, parity)) {
        if (globaltimer_ns() - t0 > timeout_ns) return false;
    }
    return true;
}

// Orders this thread's earlier generic-proxy accesses (and those it has
// acquired from other threads) before its later async-proxy (bulk copy)
// accesses, for global and shared memory.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

// FP64 reciprocal (CUDA's round-to-nearest intrinsic).
__device__ __forceinline__ double rcp64(double x) { return __drcp_rn(x); }

// Row product for column c of a multi-vector (ldx columns), one lane per
// (row, column).  The next block's column index is loaded while the current
// block is multiplied, so each block costs one memory round trip.
template <typename C, bool kShared>
__device__ __forceinline__ void row_product_colx(const C* __restrict__ val, int64_t stride, const int* __restrict__ col,
                                                 int s0, int s1, const C* xs, int xoff, int ldx, int c, C& y0, C& y1,
                                                 C& y2) {
  if constexpr (std::is_same<C, float4>::value) {
    float a[3][4] = {};
    int cb = s1 > s0 ? __ldg(col + s0) : 0;
    for (int s = s0; s < s1; ++s) {
        const int cb_next = __ldg(col + min(s + 1, s1 - 1));
        float4 xv[3];
#pragma unroll
        for (int be = 0; be < 3; ++be) {
            const int xi = (3 * cb + be) * ldx + c - xoff;
            xv[be] = kShared ? xs[xi] : ld_cg(xs + xi);
        }
#pragma unroll
        for (int al = 0; al < 3; ++al)
#pragma unroll
            for (int be = 0; be < 3; ++be) dfc_mac(a[al], ld_ro(val + (3 * al + be) * stride + s), xv[be]);
        cb = cb_next;
    }
    y0 = df_result(a[0]);
    y1 = df_result(a[1]);
    y2 = df_result(a[2]);
  } else {
    using Tr = decltype(C{}.x);
    Tr a[6] = {0, 0, 0, 0, 0, 0};
    int cb = s1 > s0 ? __ldg(col + s0) : 0;
    for (int s = s0; s < s1; ++s) {
        const int cb_next = __ldg(col + min(s + 1, s1 - 1));
        C xv[3];
#pragma unroll
        for (int be = 0; be < 3; ++be) {
            const int xi = (3 * cb + be) * ldx + c - xoff;
            xv[be] = kShared ? xs[xi] : ld_cg(xs + xi);
        }
#pragma unroll
        for (int al = 0; al < 3; ++al)
#pragma unroll
            for (int be = 0; be < 3; ++be) {
                const C v = ld_ro(val + (3 * al + be) * stride + s);
                a[2 * al] += v.x * xv[be].x - v.y * xv[be].y;
                a[2 * al + 1] += v.x * xv[be].y + v.y * xv[be].x;
            }
        cb = cb_next;
    }
    y0 = mk(a[0], a[1]);
    y1 = mk(a[2], a[3]);
    y2 = mk(a[4], a[5]);
  }
}

}  // namespace fe

namespace fe {

// Component alpha of a block row times a single vector: one thread per
// (row, alpha) walks the row's blocks; per block it reads the column index,
// the three entries (alpha, 0..2) from their planes and the three vector
// entries at the column.  No cross-lane reduction is needed.  `xs` is
// indexed by vector entry minus `xoff`.  cols[s - s0] is the block's column
// (node) index, or with kElem the index in `xs` of the column's first vector
// entry (a column map resolved once per launch).
template <typename C, bool kShared, bool kElem = false>
__device__ __forceinline__ C row_component(const C* __restrict__ val, int64_t stride, const int* cols, int s0, int s1,
                                           int al, const C* xs, int xoff) {
  if constexpr (std::is_same<C, float4>::value) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const float4* v0 = val + (3 * al) * stride;
    const float4* v1 = v0 + stride;
    const float4* v2 = v1 + stride;
    for (int s = s0; s < s1; ++s) {
        const int xa = (kElem ? cols[s - s0] : 3 * cols[s - s0]) - xoff;
        const float4 m0 = ld_ro(v0 + s), m1 = ld_ro(v1 + s), m2 = ld_ro(v2 + s);
        const float4 x0 = kShared ? xs[xa] : ld_cg(xs + xa), x1 = kShared ? xs[xa + 1] : ld_cg(xs + xa + 1),
                     x2 = kShared ? xs[xa + 2] : ld_cg(xs + xa + 2);
        dfc_mac(acc, m0, x0);
        dfc_mac(acc, m1, x1);
        dfc_mac(acc, m2, x2);
    }
    return df_result(acc);
  } else {
    using Tr = decltype(C{}.x);
    Tr ar = 0, ai = 0, br = 0, bi = 0;
    const C* v0 = val + (3 * al) * stride;
    const C* v1 = v0 + stride;
    const C* v2 = v1 + stride;
    int s = s0;
    for (; s + 1 < s1; s += 2) {  // two blocks per step, two accumulator pairs
        const int xa = (kElem ? cols[s - s0] : 3 * cols[s - s0]) - xoff,
                  xb = (kElem ? cols[s + 1 - s0] : 3 * cols[s + 1 - s0]) - xoff;
        const C ma0 = ld_ro(v0 + s), ma1 = ld_ro(v1 + s), ma2 = ld_ro(v2 + s);
        const C mb0 = ld_ro(v0 + s + 1), mb1 = ld_ro(v1 + s + 1), mb2 = ld_ro(v2 + s + 1);
        const C xa0 = kShared ? xs[xa] : ld_cg(xs + xa), xa1 = kShared ? xs[xa + 1] : ld_cg(xs + xa + 1),
                xa2 = kShared ? xs[xa + 2] : ld_cg(xs + xa + 2);
        const C xb0 = kShared ? xs[xb] : ld_cg(xs + xb), xb1 = kShared ? xs[xb + 1] : ld_cg(xs + xb + 1),
                xb2 = kShared ? xs[xb + 2] : ld_cg(xs + xb + 2);
        ar += ma0.x * xa0.x - ma0.y * xa0.y + ma1.x * xa1.x - ma1.y * xa1.y + ma2.x * xa2.x - ma2.y * xa2.y;
        ai += ma0.x * xa0.y + ma0.y * xa0.x + ma1.x * xa1.y + ma1.y * xa1.x + ma2.x * xa2.y + ma2.y * xa2.x;
        br += mb0.x * xb0.x - mb0.y * xb0.y + mb1.x * xb1.x - mb1.y * xb1.y + mb2.x * xb2.x - mb2.y * xb2.y;
        bi += mb0.x * xb0.y + mb0.y * xb0.x + mb1.x * xb1.y + mb1.y * xb1.x + mb2.x * xb2.y + mb2.y * xb2.x;
    }
    if (s < s1) {
        const int xa = (kElem ? cols[s - s0] : 3 * cols[s - s0]) - xoff;
        const C m0 = ld_ro(v0 + s), m1 = ld_ro(v1 + s), m2 = ld_ro(v2 + s);
        const C x0 = kShared ? xs[xa] : ld_cg(xs + xa), x1 = kShared ? xs[xa + 1] : ld_cg(xs + xa + 1),
                x2 = kShared ? xs[xa + 2] : ld_cg(xs + xa + 2);
        ar += m0.x * x0.x - m0.y * x0.y + m1.x * x1.x - m1.y * x1.y + m2.x * x2.x - m2.y * x2.y;
        ai += m0.x * x0.y + m0.y * x0.x + m1.x * x1.y + m1.y * x1.x + m2.x * x2.y + m2.y * x2.x;
    }
    return mk(ar + br, ai + bi);
  }
}

// Row product for column c of a multi-vector from the class stencil of a
// regular row (27 blocks, column indices read from global memory): a real
// diagonal stencil (kind 2) needs one vector entry and one real multiply-add
// per block and component; general blocks (kind 1) a full 3x3 product.
template <typename C, bool kShared>
__device__ __forceinline__ void row_product_colx_class(const StencilSet* __restrict__ S, int cls, int kind,
                                                       const int* __restrict__ col, int s0, const C* xs, int xoff,
                                                       int ldx, int c, C& y0, C& y1, C& y2) {
  if constexpr (std::is_same<C, float4>::value) {
    float a[3][4] = {};
    if (kind == 2) {
#pragma unroll 3
        for (int kk = 0; kk < 27; ++kk) {
            const int xb = 3 * __ldg(col + s0 + kk) * ldx + c - xoff;
#pragma unroll
            for (int al = 0; al < 3; ++al) {
                const float4 xv = kShared ? xs[xb + al * ldx] : ld_cg(xs + xb + al * ldx);
                const float2 dk = __ldg(&S->dvaldf[cls][al][kk]);
                df_mac(a[al][0], a[al][1], dk.x, dk.y, xv.x, xv.z);
                df_mac(a[al][2], a[al][3], dk.x, dk.y, xv.y, xv.w);
            }
        }
    } else {
        for (int kk = 0; kk < 27; ++kk) {
            const int xb = 3 * __ldg(col + s0 + kk) * ldx + c - xoff;
            float4 xv[3];
#pragma unroll
            for (int be = 0; be < 3; ++be) xv[be] = kShared ? xs[xb + be * ldx] : ld_cg(xs + xb + be * ldx);
#pragma unroll
            for (int al = 0; al < 3; ++al)
#pragma unroll
                for (int be = 0; be < 3; ++be) dfc_mac(a[al], ld_ro(&S->sdf[cls][al][kk][be]), xv[be]);
        }
    }
    y0 = df_result(a[0]);
    y1 = df_result(a[1]);
    y2 = df_result(a[2]);
  } else {
    using Tr = decltype(C{}.x);
    constexpr bool kF32 = sizeof(C) == 8;
    Tr a[6] = {0, 0, 0, 0, 0, 0};
    if (kind == 2) {
#pragma unroll 3
        for (int kk = 0; kk < 27; ++kk) {
            const int xb = 3 * __ldg(col + s0 + kk) * ldx + c - xoff;
#pragma unroll
            for (int al = 0; al < 3; ++al) {
                const C xv = kShared ? xs[xb + al * ldx] : ld_cg(xs + xb + al * ldx);
                const Tr dk = kF32 ? (Tr)__ldg(&S->dval32[cls][al][kk]) : (Tr)__ldg(&S->dval[cls][al][kk]);
                a[2 * al] += dk * xv.x;
                a[2 * al + 1] += dk * xv.y;
            }
        }
    } else {
        const C* st = kF32 ? (const C*)S->s32[cls][0][0] : (const C*)S->s64[cls][0][0];
        for (int kk = 0; kk < 27; ++kk) {
            const int xb = 3 * __ldg(col + s0 + kk) * ldx + c - xoff;
            C xv[3];
#pragma unroll
            for (int be = 0; be < 3; ++be) xv[be] = kShared ? xs[xb + be * ldx] : ld_cg(xs + xb + be * ldx);
#pragma unroll
            for (int al = 0; al < 3; ++al)
#pragma unroll
                for (int be = 0; be < 3; ++be) {
                    const C v = ld_ro(st + (al * 27 + kk) * 3 + be);
                    a[2 * al] += v.x * xv[be].x - v.y * xv[be].y;
                    a[2 * al + 1] += v.x * xv[be].y + v.y * xv[be].x;
                }
        }
    }
    y0 = mk(a[0], a[1]);
    y1 = mk(a[2], a[3]);
    y2 = mk(a[4], a[5]);
  }
}

// Copies the column indices of the warp's rows [rb, re) into shared memory
// (one coalesced pass); returns the first block index sb of the range.
__device__ __forceinline__ int stage_cols(const int* __restrict__ rp, const int* __restrict__ col, int rb, int re,
                                          int* cols, int lane) {
    const int sb = __ldg(rp + rb), se = __ldg(rp + re);
    for (int j = lane; j < se - sb; j += 32) cols[j] = __ldg(col + sb + j);
    __syncwarp();
    return sb;
}

// Component alpha of a regular row (all 27 blocks present) from the class
// stencil: a real diagonal stencil (kind 2) needs one vector entry and one
// real multiply-add per block; general blocks (kind 1) a full 3x3 product.
template <typename C, bool kShared, bool kElem = false>
__device__ __forceinline__ C row_component_class(const StencilSet* __restrict__ S, int cls, int kind, const int* cols,
                                                 int al, const C* xs, int xoff) {
  if constexpr (std::is_same<C, float4>::value) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    if (kind == 2) {
        const float2* d = S->dvaldf[cls][al];
#pragma unroll 9
        for (int kk = 0; kk < 27; ++kk) {
            const int xi = (kElem ? cols[kk] : 3 * cols[kk]) + al - xoff;
            const float4 xv = kShared ? xs[xi] : ld_cg(xs + xi);
            const float2 dk = __ldg(d + kk);
            df_mac(acc[0], acc[1], dk.x, dk.y, xv.x, xv.z);
            df_mac(acc[2], acc[3], dk.x, dk.y, xv.y, xv.w);
        }
    } else {
        const float4* sp = S->sdf[cls][al][0];
#pragma unroll 3
        for (int kk = 0; kk < 27; ++kk) {
            const int xi = (kElem ? cols[kk] : 3 * cols[kk]) - xoff;
#pragma unroll
            for (int be = 0; be < 3; ++be) dfc_mac(acc, ld_ro(sp + 3 * kk + be), kShared ? xs[xi + be] : ld_cg(xs + xi + be));
        }
    }
    return df_result(acc);
  } else {
    using Tr = decltype(C{}.x);
    constexpr bool kF32 = sizeof(C) == 8;
    Tr ar = 0, ai = 0;
    if (kind == 2) {
        const Tr* d = kF32 ? (const Tr*)S->dval32[cls][al] : (const Tr*)S->dval[cls][al];
#pragma unroll 9
        for (int kk = 0; kk < 27; ++kk) {
            const int xi = (kElem ? cols[kk] : 3 * cols[kk]) + al - xoff;
            const C xv = kShared ? xs[xi] : ld_cg(xs + xi);
            const Tr dk = __ldg(d + kk);
            ar += dk * xv.x;
            ai += dk * xv.y;
        }
    } else {
        const C* s = kF32 ? (const C*)S->s32[cls][al][0] : (const C*)S->s64[cls][al][0];
#pragma unroll 3
        for (int kk = 0; kk < 27; ++kk) {
            const int xi = (kElem ? cols[kk] : 3 * cols[kk]) - xoff;
#pragma unroll
            for (int be = 0; be < 3; ++be) {
                const C m = ld_ro(s + 3 * kk + be);
                const C xv = kShared ? xs[xi + be] : ld_cg(xs + xi + be);
                ar += m.x * xv.x - m.y * xv.y;
                ai += m.x * xv.y + m.y * xv.x;
            }
        }
    }
    return mk(ar, ai);
  }
}

}  // namespace fe
