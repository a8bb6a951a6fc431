// Standalone sparse products y = A x (fe_spmv): the Krylov loop's product
// (Section 3.1.5.1) as its own entry point, for one or several vectors.
#include "krylov.cuh"

#include <algorithm>
#include <cstdint>
#include <type_traits>

namespace fe {

template <typename C>
__global__ void __launch_bounds__(256) k_spmv_cols(const C* __restrict__ val, int64_t stride,
                                                   const int* __restrict__ col, const int* __restrict__ rp,
                                                   const C* __restrict__ x, C* __restrict__ y, int n_rows, int nrhs) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_rows * nrhs) return;
    const int row = (int)(t / nrhs), c = (int)(t - (int64_t)row * nrhs);
    C v[3];
    row_product_colx<C, false>(val, stride, col, __ldg(rp + row), __ldg(rp + row + 1), x, 0, nrhs, c, v[0], v[1],
                               v[2]);
#pragma unroll
    for (int al = 0; al < 3; ++al) y[(size_t)(3 * row + al) * nrhs + c] = v[al];
}

// y = A x for R = 1, 2, 4, ..., 32 columns: one warp per block row, its lanes
// split into 32/R block groups x R columns.  A block's nine entries are read
// once per warp (the R lanes of a group read the same address), the R values
// of one vector entry are contiguous, and the groups' partial sums meet in a
// shuffle reduction (FP32 pairs: error-free pair additions).
template <typename C, int R>
__global__ void __launch_bounds__(256) k_spmv_warp(const C* __restrict__ val, int64_t stride,
                                                   const int* __restrict__ col, const int* __restrict__ rp,
                                                   const C* __restrict__ x, C* __restrict__ y, int n_rows) {
    const int lane = threadIdx.x & 31;
    constexpr int G = 32 / R;
    const int c = lane % R, g = lane / R;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n_rows; row += nw) {
        const int s0 = __ldg(rp + row), s1 = __ldg(rp + row + 1);
        // the nine entries of a block load before its (dependent) vector entries;
        // the next column index loads one step ahead
        int cb = s0 + g < s1 ? __ldg(col + s0 + g) : 0;
        if constexpr (std::is_same<C, float4>::value) {
            float a[3][4] = {};
            for (int s = s0 + g; s < s1; s += G) {
                const int cb_next = s + G < s1 ? __ldg(col + s + G) : 0;
                float4 m[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) m[q] = __ldg(val + q * stride + s);
                const int xb = 3 * cb * R + c;
                float4 xv[3];
#pragma unroll
                for (int be = 0; be < 3; ++be) xv[be] = __ldg(x + xb + be * R);
#pragma unroll
                for (int al = 0; al < 3; ++al)
#pragma unroll
                    for (int be = 0; be < 3; ++be) dfc_mac(a[al], m[3 * al + be], xv[be]);
                cb = cb_next;
            }
#pragma unroll
            for (int o = 16; o >= R; o >>= 1)
#pragma unroll
                for (int al = 0; al < 3; ++al)
#pragma unroll
                    for (int q = 0; q < 4; q += 2) {
                        const float h2 = __shfl_xor_sync(0xffffffffu, a[al][q], o);
                        const float l2 = __shfl_xor_sync(0xffffffffu, a[al][q + 1], o);
                        df_add(a[al][q], a[al][q + 1], h2, l2);
                    }
            if (g == 0)
#pragma unroll
                for (int al = 0; al < 3; ++al) y[(size_t)(3 * row + al) * R + c] = df_result_norm(a[al]);
        } else {
            using Tr = decltype(C{}.x);
            Tr a[6] = {0, 0, 0, 0, 0, 0};
            for (int s = s0 + g; s < s1; s += G) {
                const int cb_next = s + G < s1 ? __ldg(col + s + G) : 0;
                C m[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) m[q] = __ldg(val + q * stride + s);
                const int xb = 3 * cb * R + c;
                C xv[3];
#pragma unroll
                for (int be = 0; be < 3; ++be) xv[be] = __ldg(x + xb + be * R);
#pragma unroll
                for (int al = 0; al < 3; ++al)
#pragma unroll
                    for (int be = 0; be < 3; ++be) {
                        a[2 * al] += m[3 * al + be].x * xv[be].x - m[3 * al + be].y * xv[be].y;
                        a[2 * al + 1] += m[3 * al + be].x * xv[be].y + m[3 * al + be].y * xv[be].x;
                    }
                cb = cb_next;
            }
#pragma unroll
            for (int o = 16; o >= R; o >>= 1)
#pragma unroll
                for (int k = 0; k < 6; ++k) a[k] += __shfl_xor_sync(0xffffffffu, a[k], o);
            if (g == 0)
#pragma unroll
                for (int al = 0; al < 3; ++al) y[(size_t)(3 * row + al) * R + c] = mk(a[2 * al], a[2 * al + 1]);
        }
    }
}

// y = A x for R = 8, 16 or 32 columns: a warp takes G = 32/R consecutive
// block rows, one group of R lanes (one lane per column) per row.  The warp
// first copies the nine entries and the column index of every block of its
// G rows into shared memory with coalesced loads (lane l takes block l, l +
// 32, ...: the blocks of consecutive rows are consecutive in each plane), so
// that the whole group of rows is in flight at once; then each group walks
// its row from shared memory (the R lanes read the same entry) and multiplies
// by the R contiguous vector values of each block's column.  No reduction
// across lanes is needed.
constexpr int kSpmmWarps = 4;

template <typename C, int R>
__global__ void __launch_bounds__(32 * kSpmmWarps) k_spmm_rows(const C* __restrict__ val, int64_t stride,
                                                               const int* __restrict__ col,
                                                               const int* __restrict__ rp, const C* __restrict__ x,
                                                               C* __restrict__ y, int n_rows) {
    constexpr int G = 32 / R;
    constexpr int kMax = 27 * G;
    __shared__ C s_val[kSpmmWarps][9][kMax];
    __shared__ int s_col[kSpmmWarps][kMax];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = lane % R, g = lane / R;
    const int n_groups = (n_rows + G - 1) / G;
    const int nw = gridDim.x * kSpmmWarps;
    C(*sv)[kMax] = s_val[warp];
    int* sc = s_col[warp];
    for (int grp = blockIdx.x * kSpmmWarps + warp; grp < n_groups; grp += nw) {
        const int r0 = grp * G, r1 = min(r0 + G, n_rows);
        const int b0 = __ldg(rp + r0), nb = __ldg(rp + r1) - b0;
        if (nb > kMax) {  // not a voxel pattern (at most 27 blocks per row): read the blocks directly
            const int row = r0 + g;
            if (row < r1) {
                C v[3];
                row_product_colx<C, false>(val, stride, col, __ldg(rp + row), __ldg(rp + row + 1), x, 0, R, c, v[0],
                                           v[1], v[2]);
#pragma unroll
                for (int al = 0; al < 3; ++al) y[(size_t)(3 * row + al) * R + c] = v[al];
            }
            continue;
        }
        for (int k = lane; k < nb; k += 32) {
            sc[k] = __ldg(col + b0 + k);
#pragma unroll
            for (int q = 0; q < 9; ++q) sv[q][k] = __ldg(val + q * stride + b0 + k);
        }
        __syncwarp();
        const int row = r0 + g;
        if (row < r1) {
            const int k0 = __ldg(rp + row) - b0, k1 = __ldg(rp + row + 1) - b0;
            if constexpr (std::is_same<C, float4>::value) {
                float a[3][4] = {};
                for (int k = k0; k < k1; ++k) {
                    const int xb = 3 * sc[k] * R + c;
                    const float4 x0 = __ldg(x + xb), x1 = __ldg(x + xb + R), x2 = __ldg(x + xb + 2 * R);
#pragma unroll
                    for (int al = 0; al < 3; ++al) {
                        dfc_mac(a[al], sv[3 * al][k], x0);
                        dfc_mac(a[al], sv[3 * al + 1][k], x1);
                        dfc_mac(a[al], sv[3 * al + 2][k], x2);
                    }
                }
#pragma unroll
                for (int al = 0; al < 3; ++al) y[(size_t)(3 * row + al) * R + c] = df_result_norm(a[al]);
            } else {
                using Tr = decltype(C{}.x);
                Tr a[6] = {0, 0, 0, 0, 0, 0};
                for (int k = k0; k < k1; ++k) {
                    const int xb = 3 * sc[k] * R + c;
                    const C xv[3] = {__ldg(x + xb), __ldg(x + xb + R), __ldg(x + xb + 2 * R)};
#pragma unroll
                    for (int al = 0; al < 3; ++al)
#pragma unroll
                        for (int be = 0; be < 3; ++be) {
                            const C m = sv[3 * al + be][k];
                            a[2 * al] += m.x * xv[be].x - m.y * xv[be].y;
                            a[2 * al + 1] += m.x * xv[be].y + m.y * xv[be].x;
                        }
                }
#pragma unroll
                for (int al = 0; al < 3; ++al) y[(size_t)(3 * row + al) * R + c] = mk(a[2 * al], a[2 * al + 1]);
            }
        }
        __syncwarp();
    }
}

// y = A x for R = 8, 16 or 32 complex64 columns, with several columns per
// lane: CPL adjacent columns per lane, L = R / CPL lanes per row and G = 32 /
// L rows per warp.  As in k_spmm_rows the warp first stages its rows' blocks
// (nine planes and the column indices) in shared memory with coalesced
// loads; each entry read from shared memory then serves CPL columns, and a
// lane reads its CPL vector values of a block row with 16-byte loads.  PF
// loads the next block's vector values one step ahead.
template <int CPL>
struct SpmmX;
template <>
struct SpmmX<2> {
    float4 v[1];
};
template <>
struct SpmmX<4> {
    float4 v[2];
};

template <int R, int CPL>
__device__ __forceinline__ void spmm_load_x(const float2* __restrict__ x, int cb, int c0, SpmmX<CPL> (&d)[3]) {
#pragma unroll
    for (int be = 0; be < 3; ++be) {
        const float4* p = (const float4*)(x + (size_t)(3 * cb + be) * R + c0);
#pragma unroll
        for (int v = 0; v < CPL / 2; ++v) d[be].v[v] = __ldg(p + v);
    }
}

template <int R, int CPL, int W, bool PF>
__global__ void __launch_bounds__(32 * W) k_spmm_cpl(const float2* __restrict__ val, int64_t stride,
                                                     const int* __restrict__ col, const int* __restrict__ rp,
                                                     const float2* __restrict__ x, float2* __restrict__ y,
                                                     int n_rows) {
    constexpr int L = R / CPL, G = 32 / L, kMax = 27 * G;
    __shared__ float2 s_val[W][9][kMax];
    __shared__ int s_col[W][kMax];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c0 = (lane % L) * CPL, g = lane / L;
    const int n_groups = (n_rows + G - 1) / G;
    float2(*sv)[kMax] = s_val[warp];
    int* sc = s_col[warp];
    for (int grp = blockIdx.x * W + warp; grp < n_groups; grp += gridDim.x * W) {
        const int r0 = grp * G, r1 = min(r0 + G, n_rows);
        const int b0 = __ldg(rp + r0), nb = __ldg(rp + r1) - b0;
        const int row = r0 + g;
        float a[3][CPL][2] = {};
        if (nb > kMax) {  // not a voxel pattern (at most 27 blocks per row): read the blocks directly
            if (row < r1)
#pragma unroll
                for (int j = 0; j < CPL; ++j) {
                    float2 v[3];
                    row_product_colx<float2, false>(val, stride, col, __ldg(rp + row), __ldg(rp + row + 1), x, 0, R,
                                                    c0 + j, v[0], v[1], v[2]);
#pragma unroll
                    for (int al = 0; al < 3; ++al) {
                        a[al][j][0] = v[al].x;
                        a[al][j][1] = v[al].y;
                    }
                }
        } else {
            for (int k = lane; k < nb; k += 32) {
                sc[k] = __ldg(col + b0 + k);
#pragma unroll
                for (int q = 0; q < 9; ++q) sv[q][k] = __ldg(val + q * stride + b0 + k);
            }
            __syncwarp();
            if (row < r1) {
                const int k0 = __ldg(rp + row) - b0, k1 = __ldg(rp + row + 1) - b0;
                SpmmX<CPL> xn[3];
                if (PF && k0 < k1) spmm_load_x<R, CPL>(x, sc[k0], c0, xn);
                for (int k = k0; k < k1; ++k) {
                    SpmmX<CPL> xv[3];
                    if (PF) {
#pragma unroll
                        for (int be = 0; be < 3; ++be) xv[be] = xn[be];
                        if (k + 1 < k1) spmm_load_x<R, CPL>(x, sc[k + 1], c0, xn);
                    } else {
                        spmm_load_x<R, CPL>(x, sc[k], c0, xv);
                    }
#pragma unroll
                    for (int al = 0; al < 3; ++al)
#pragma unroll
                        for (int be = 0; be < 3; ++be) {
                            const float2 m = sv[3 * al + be][k];
#pragma unroll
                            for (int v = 0; v < CPL / 2; ++v) {
                                const float4 q = xv[be].v[v];
                                a[al][2 * v][0] += m.x * q.x - m.y * q.y;
                                a[al][2 * v][1] += m.x * q.y + m.y * q.x;
                                a[al][2 * v + 1][0] += m.x * q.z - m.y * q.w;
                                a[al][2 * v + 1][1] += m.x * q.w + m.y * q.z;
                            }
                        }
                }
            }
            __syncwarp();
        }
        if (row < r1)
#pragma unroll
            for (int al = 0; al < 3; ++al) {
                float4* p = (float4*)(y + (size_t)(3 * row + al) * R + c0);
#pragma unroll
                for (int v = 0; v < CPL / 2; ++v)
                    p[v] = make_float4(a[al][2 * v][0], a[al][2 * v][1], a[al][2 * v + 1][0], a[al][2 * v + 1][1]);
            }
    }
}

// Columns per lane, warps per CTA and prefetch for each width, chosen by
// timing every combination on a 27-point pattern of 81^3 nodes (14.0 M
// blocks) on GB300: R = 8 2 / 2 / on, R = 16 4 / 2 / off, R = 32 2 / 8 / off.
template <int R, int CPL, int W, bool PF>
static void launch_spmm_cpl_t(cudaStream_t st, int sms, const float2* val, int64_t stride, const int* col,
                              const int* rp, const float2* x, float2* y, int n_rows) {
    constexpr int G = 32 / (R / CPL);
    int per_sm = 0;  // resident CTAs per SM (a host query, no device work)
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmm_cpl<R, CPL, W, PF>, 32 * W, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int64_t groups = ((int64_t)n_rows + G - 1) / G;
    const unsigned blocks =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * per_sm, (groups + W - 1) / W));
    k_spmm_cpl<R, CPL, W, PF><<<blocks, 32 * W, 0, st>>>(val, stride, col, rp, x, y, n_rows);
}

static void launch_spmm_cpl(int R, cudaStream_t st, int sms, const float2* val, int64_t stride, const int* col,
                            const int* rp, const float2* x, float2* y, int n_rows) {
    switch (R) {
        case 8: launch_spmm_cpl_t<8, 2, 2, true>(st, sms, val, stride, col, rp, x, y, n_rows); break;
        case 16: launch_spmm_cpl_t<16, 4, 2, false>(st, sms, val, stride, col, rp, x, y, n_rows); break;
        default: launch_spmm_cpl_t<32, 2, 8, false>(st, sms, val, stride, col, rp, x, y, n_rows); break;
    }
}

template <typename C>
static void launch_spmm_rows(int R, cudaStream_t st, int sms, const C* val, int64_t stride, const int* col,
                             const int* rp, const C* x, C* y, int n_rows) {
    const int G = 32 / R;
    const int64_t groups = ((int64_t)n_rows + G - 1) / G;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 16,
                                                                            (groups + kSpmmWarps - 1) / kSpmmWarps));
    switch (R) {
        case 8: k_spmm_rows<C, 8><<<blocks, 32 * kSpmmWarps, 0, st>>>(val, stride, col, rp, x, y, n_rows); break;
        case 16: k_spmm_rows<C, 16><<<blocks, 32 * kSpmmWarps, 0, st>>>(val, stride, col, rp, x, y, n_rows); break;
        default: k_spmm_rows<C, 32><<<blocks, 32 * kSpmmWarps, 0, st>>>(val, stride, col, rp, x, y, n_rows); break;
    }
}

template <typename C>
static void launch_spmv_warp(int R, unsigned blocks, cudaStream_t st, const C* val, int64_t stride, const int* col,
                             const int* rp, const C* x, C* y, int n_rows) {
    switch (R) {
        case 1: k_spmv_warp<C, 1><<<blocks, 256, 0, st>>>(val, stride, col, rp, x, y, n_rows); break;
        case 2: k_spmv_warp<C, 2><<<blocks, 256, 0, st>>>(val, stride, col, rp, x, y, n_rows); break;
        case 4: k_spmv_warp<C, 4><<<blocks, 256, 0, st>>>(val, stride, col, rp, x, y, n_rows); break;
        case 8: k_spmv_warp<C, 8><<<blocks, 256, 0, st>>>(val, stride, col, rp, x, y, n_rows); break;
        case 16: k_spmv_warp<C, 16><<<blocks, 256, 0, st>>>(val, stride, col, rp, x, y, n_rows); break;
        default: k_spmv_warp<C, 32><<<blocks, 256, 0, st>>>(val, stride, col, rp, x, y, n_rows); break;
    }
}

}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_spmv(fe_ctx* ctx, const fe_system* s, int32_t precision, int32_t nrhs, const void* x, void* y) {
    if (!ctx || !s || !x || !y || nrhs < 1) {
        set_error("fe_spmv: NULL argument or nrhs < 1");
        return FE_ERR_INVALID_ARG;
    }
    const fe_mesh* m = s->mesh;
    cudaStream_t st = ctx->stream;
    const int* rp = (const int*)m->row_ptr.ptr;
    const int* col = (const int*)m->col_idx.ptr;
    const bool pow2 = nrhs <= 32 && (nrhs & (nrhs - 1)) == 0;
    const unsigned warp_blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)ctx->num_sms * 8,
                                                                                  ((int64_t)m->n_act + 7) / 8));
    const int64_t n_items = (int64_t)m->n_act * nrhs;
    const unsigned col_blocks = (unsigned)((n_items + 255) / 256);
    if (precision == FE_PREC_FP64) {
        if (pow2 && nrhs >= 8)
            launch_spmm_rows<double2>(nrhs, st, ctx->num_sms, (const double2*)s->val64.ptr, s->stride, col, rp,
                                  (const double2*)x, (double2*)y, m->n_act);
        else if (pow2)
            launch_spmv_warp<double2>(nrhs, warp_blocks, st, (const double2*)s->val64.ptr, s->stride, col, rp,
                                  (const double2*)x, (double2*)y, m->n_act);
        else
            k_spmv_cols<double2><<<col_blocks, 256, 0, st>>>((const double2*)s->val64.ptr, s->stride, col, rp,
                                                             (const double2*)x, (double2*)y, m->n_act, nrhs);
    } else if (precision == FE_PREC_MIXED) {
        if (!s->val32.ptr) {
            set_error("fe_spmv: no complex64 copy (system assembled in FP64)");
            return FE_ERR_INVALID_ARG;
        }
        const bool aligned16 = (((uintptr_t)x | (uintptr_t)y) & 15) == 0;  // the lanes' 16-byte vector accesses
        if (pow2 && nrhs >= 8 && aligned16)
            launch_spmm_cpl(nrhs, st, ctx->num_sms, (const float2*)s->val32.ptr, s->stride, col, rp,
                            (const float2*)x, (float2*)y, m->n_act);
        else if (pow2 && nrhs >= 8)
            launch_spmm_rows<float2>(nrhs, st, ctx->num_sms, (const float2*)s->val32.ptr, s->stride, col, rp,
                                  (const float2*)x, (float2*)y, m->n_act);
        else if (pow2)
            launch_spmv_warp<float2>(nrhs, warp_blocks, st, (const float2*)s->val32.ptr, s->stride, col, rp,
                                  (const float2*)x, (float2*)y, m->n_act);
        else
            k_spmv_cols<float2><<<col_blocks, 256, 0, st>>>((const float2*)s->val32.ptr, s->stride, col, rp,
                                                            (const float2*)x, (float2*)y, m->n_act, nrhs);
    } else if (precision == FE_PREC_DF) {
        if (!s->valdf.ptr) {
            set_error("fe_spmv: no FP32-pair copy (system not assembled with FE_PREC_DF)");
            return FE_ERR_INVALID_ARG;
        }
        if (pow2 && nrhs >= 8)
            launch_spmm_rows<float4>(nrhs, st, ctx->num_sms, (const float4*)s->valdf.ptr, s->stride, col, rp,
                                  (const float4*)x, (float4*)y, m->n_act);
        else if (pow2)
            launch_spmv_warp<float4>(nrhs, warp_blocks, st, (const float4*)s->valdf.ptr, s->stride, col, rp,
                                  (const float4*)x, (float4*)y, m->n_act);
        else
            k_spmv_cols<float4><<<col_blocks, 256, 0, st>>>((const float4*)s->valdf.ptr, s->stride, col, rp,
                                                            (const float4*)x, (float4*)y, m->n_act, nrhs);
    } else {
        set_error("fe_spmv: bad precision");
        return FE_ERR_INVALID_ARG;
    }
    FE_LAUNCHED();
    return FE_OK;
}

}  // extern "C"
