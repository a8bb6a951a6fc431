// Block incomplete Cholesky preconditioner (BICP), Section 3.1.5.3.
//
// The node rows are split into S contiguous bands, one per CTA of the
// persistent solve (band b: floor(b n / S) <= I < floor((b + 1) n / S), the
// rows a CTA updates).  Each band's diagonal block of A gets an incomplete
// Cholesky factor on its own lower node-block pattern (Eq. 5, with the terms
// that couple different bands dropped), unconjugated since A is complex
// symmetric: L L^T = A on every stored block (I, J), J <= I, of the band.
// On full 3x3 blocks the scalar column-by-column algorithm of Eq. 5 and the
// block form used here give the same factor (an incomplete Cholesky factor
// is unique on its pattern): off-diagonal blocks are full, diagonal blocks
// are lower triangular 3x3 Cholesky factors.
//
//   L_IJ = (A_IJ - sum_{K < J} L_IK L_JK^T) L_JJ^{-T}          J < I
//   L_II L_II^T = A_II - sum_{K < I} L_IK L_IK^T               (3x3 Cholesky)
//
// Setup runs on the device: one thread per band walks its rows in order
// (the factor is sequential within a band, and is built once per system).
// The same pass sorts each band's nodes by level for the substitutions of
// Eq. 6: the level of a node is one more than the highest level of its lower
// neighbours in the band, so the nodes of one level do not couple and each
// level is one parallel step of the forward (or, in reverse, back)
// substitution inside the solve kernel.
#include "fe_internal.cuh"

#include <algorithm>
#include <vector>

namespace fe {
namespace {

__device__ __forceinline__ double2 c_mul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 c_sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 c_div(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
// Principal square root (Re >= 0; the sign of Im follows Im z), from
// sqrt(a + ib) = t + i b / (2t) with t = sqrt((|z| + a) / 2) for a >= 0, and
// the mirrored form for a < 0 (no cancellation in either branch).
__device__ __forceinline__ double2 c_sqrt(double2 z) {
    const double m = hypot(z.x, z.y);
    if (m == 0.0) return make_double2(0.0, 0.0);
    if (z.x >= 0.0) {
        const double t = sqrt(0.5 * (m + z.x));
        return make_double2(t, z.y / (2.0 * t));
    }
    const double t = sqrt(0.5 * (m - z.x));
    return make_double2(fabs(z.y) / (2.0 * t), copysign(t, z.y));
}
__device__ __forceinline__ bool c_usable(double2 v) {
    const double m = fabs(v.x) + fabs(v.y);
    return m > 0.0 && m < 1e300;
}

__device__ __forceinline__ void band_of(int b, int n, int S, int& i0, int& i1) {
    i0 = (int)((int64_t)b * n / S);
    i1 = (int)((int64_t)(b + 1) * n / S);
}

// tpos[p] = slot of block (J, I) for the block p = (I, J) (the pattern is
// structurally symmetric).
__global__ void k_bicp_tpos(int n, const int* __restrict__ rp, const int* __restrict__ col, int* __restrict__ tpos,
                            int* __restrict__ status) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= n) return;
    for (int p = rp[I]; p < rp[I + 1]; ++p) {
        const int J = col[p];
        int t = -1;
        for (int q = rp[J]; q < rp[J + 1]; ++q)
            if (col[q] == I) t = q;
        tpos[p] = t;
        if (t < 0) atomicOr(status, kDevBadIndex);
    }
}

// Levels and the level-sorted node table of each band: (node, first slot of
// the row inside the band, diagonal slot, end of the row's slots inside the
// band), so the substitutions reach a row's band blocks without searching.
__global__ void k_bicp_levels(int n, int S, const int* __restrict__ rp, const int* __restrict__ col,
                              int* __restrict__ lvl, int4* __restrict__ tab, int* __restrict__ lev,
                              int* __restrict__ nlev) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= S) return;
    int i0, i1;
    band_of(b, n, S, i0, i1);
    int top = -1;
    for (int I = i0; I < i1; ++I) {
        int l = 0;
        for (int p = rp[I]; p < rp[I + 1]; ++p) {
            const int J = col[p];
            if (J >= I) break;
            if (J >= i0) l = max(l, lvl[J] + 1);
        }
        lvl[I] = l;
        top = max(top, l);
    }
    const int nl = top + 1;
    int* off = lev + i0 + b;  // nl + 1 <= (i1 - i0) + 1 entries
    for (int l = 0; l <= nl; ++l) off[l] = 0;
    for (int I = i0; I < i1; ++I) off[lvl[I] + 1] += 1;
    for (int l = 1; l <= nl; ++l) off[l] += off[l - 1];
    for (int I = i0; I < i1; ++I) {
        int lo = rp[I + 1], dg = -1, hi = rp[I + 1];
        for (int p = rp[I + 1] - 1; p >= rp[I]; --p) {
            const int J = col[p];
            if (J >= i1) hi = p;
            if (J >= i0) lo = p;
            if (J == I) dg = p;
        }
        tab[i0 + off[lvl[I]]++] = make_int4(I, lo, dg, hi);  // off[l] ends at the start of level l + 1
    }
    for (int l = nl; l >= 1; --l) off[l] = off[l - 1];
    off[0] = 0;
    nlev[b] = nl;
}

// The factor of each band, row by row (the block form of Eq. 5).
__global__ void k_bicp_factor(int n, int S, const int* __restrict__ rp, const int* __restrict__ col,
                              const double2* __restrict__ val64, int64_t stride, double2* L, double2* Linv,
                              int* __restrict__ status) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= S) return;
    int i0, i1;
    band_of(b, n, S, i0, i1);
    for (int I = i0; I < i1; ++I) {
        const int p0 = rp[I], p1 = rp[I + 1];
        for (int p = p0; p < p1; ++p) {
            const int J = col[p];
            if (J < i0) continue;
            if (J > I) break;
            double2 Sb[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) Sb[q] = val64[q * stride + p];
            // minus sum over the common lower neighbours K (i0 <= K < J) of rows I and J
            int q = p0, r = rp[J];
            const int rend = rp[J + 1];
            while (q < p && r < rend) {
                const int kq = col[q], kr = col[r];
                if (kr >= J) break;
                if (kq < kr) {
                    ++q;
                } else if (kr < kq) {
                    ++r;
                } else {
                    if (kq >= i0) {
                        const double2* Lq = L + (size_t)q * 9;
                        const double2* Lr = L + (size_t)r * 9;
#pragma unroll
                        for (int al = 0; al < 3; ++al)
#pragma unroll
                            for (int be = 0; be < 3; ++be) {
                                double2 acc = Sb[3 * al + be];
#pragma unroll
                                for (int ga = 0; ga < 3; ++ga) acc = c_sub(acc, c_mul(Lq[3 * al + ga], Lr[3 * be + ga]));
                                Sb[3 * al + be] = acc;
                            }
                    }
                    ++q;
                    ++r;
                }
            }
            double2* out = L + (size_t)p * 9;
            if (J < I) {
                // L_IJ = S L_JJ^{-T}: (al, be) = sum_{ga <= be} S[al][ga] Linv_J[be][ga]
                const double2* M = Linv + (size_t)J * 9;
#pragma unroll
                for (int al = 0; al < 3; ++al)
#pragma unroll
                    for (int be = 0; be < 3; ++be) {
                        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
                        for (int ga = 0; ga <= be; ++ga) {
                            const double2 t = c_mul(Sb[3 * al + ga], M[3 * be + ga]);
                            acc.x += t.x;
                            acc.y += t.y;
                        }
                        out[3 * al + be] = acc;
                    }
            } else {
                // 3x3 unconjugated Cholesky of S (lower entries), then its inverse
                const double2 l00 = c_sqrt(Sb[0]);
                if (!c_usable(l00)) {
                    atomicOr(status, kDevSingular);
                    return;
                }
                const double2 l10 = c_div(Sb[3], l00), l20 = c_div(Sb[6], l00);
                const double2 l11 = c_sqrt(c_sub(Sb[4], c_mul(l10, l10)));
                if (!c_usable(l11)) {
                    atomicOr(status, kDevSingular);
                    return;
                }
                const double2 l21 = c_div(c_sub(Sb[7], c_mul(l20, l10)), l11);
                const double2 l22 = c_sqrt(c_sub(c_sub(Sb[8], c_mul(l20, l20)), c_mul(l21, l21)));
                if (!c_usable(l22)) {
                    atomicOr(status, kDevSingular);
                    return;
                }
                const double2 z = make_double2(0.0, 0.0), one = make_double2(1.0, 0.0);
                out[0] = l00; out[1] = z;   out[2] = z;
                out[3] = l10; out[4] = l11; out[5] = z;
                out[6] = l20; out[7] = l21; out[8] = l22;
                // inverse of the lower triangular factor
                const double2 m00 = c_div(one, l00), m11 = c_div(one, l11), m22 = c_div(one, l22);
                const double2 m10 = c_mul(make_double2(-m11.x, -m11.y), c_mul(l10, m00));
                const double2 m21 = c_mul(make_double2(-m22.x, -m22.y), c_mul(l21, m11));
                const double2 s20 = c_mul(l20, m00), s21 = c_mul(l21, m10);
                const double2 m20 = c_mul(make_double2(-m22.x, -m22.y), make_double2(s20.x + s21.x, s20.y + s21.y));
                double2* M = Linv + (size_t)I * 9;
                M[0] = m00; M[1] = z;   M[2] = z;
                M[3] = m10; M[4] = m11; M[5] = z;
                M[6] = m20; M[7] = m21; M[8] = m22;
            }
        }
    }
}

unsigned blocks_of(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace
}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_system_factor_bicp(fe_ctx* ctx, fe_system* s, int32_t n_sub) {
    if (!ctx || !s) {
        set_error("fe_system_factor_bicp: NULL argument");
        return FE_ERR_INVALID_ARG;
    }
    const fe_mesh* m = s->mesh;
    if (!s->val64.ptr || m->n_act < 1 || s->variant == FE_VARIANT_L) {
        set_error("fe_system_factor_bicp: needs a symmetric variant (S or P) with rows");
        return FE_ERR_INVALID_ARG;
    }
    const int n = m->n_act;
    const int S = n_sub == 0 ? std::min(ctx->num_sms, n) : n_sub;
    if (S < 1 || S > n) {
        set_error("fe_system_factor_bicp: %d bands for %d node rows", (int)n_sub, n);
        return FE_ERR_INVALID_ARG;
    }
    FE_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    for (DevBuf* b : {&s->bicp_l, &s->bicp_linv, &s->bicp_tpos, &s->bicp_tab, &s->bicp_lev, &s->bicp_nlev})
        dev_free(st, *b);
    s->bicp_n_sub = 0;
    DevBuf lvl, status;
    auto fail = [&](fe_status e) {
        for (DevBuf* b : {&s->bicp_l, &s->bicp_linv, &s->bicp_tpos, &s->bicp_tab, &s->bicp_lev, &s->bicp_nlev, &lvl,
                          &status})
            dev_free(st, *b);
        return e;
    };
    fe_status e;
    const size_t nb = (size_t)m->nnzb;
    if ((e = dev_alloc(st, s->bicp_l, nb * 9 * sizeof(double2))) != FE_OK) return fail(e);
    if ((e = dev_alloc(st, s->bicp_linv, (size_t)n * 9 * sizeof(double2))) != FE_OK) return fail(e);
    if ((e = dev_alloc(st, s->bicp_tpos, nb * sizeof(int))) != FE_OK) return fail(e);
    if ((e = dev_alloc(st, s->bicp_tab, (size_t)n * sizeof(int4))) != FE_OK) return fail(e);
    if ((e = dev_alloc(st, s->bicp_lev, ((size_t)n + S) * sizeof(int))) != FE_OK) return fail(e);
    if ((e = dev_alloc(st, s->bicp_nlev, (size_t)S * sizeof(int))) != FE_OK) return fail(e);
    if ((e = dev_alloc(st, lvl, (size_t)n * sizeof(int))) != FE_OK) return fail(e);
    if ((e = dev_alloc(st, status, sizeof(int))) != FE_OK) return fail(e);
    const int* rp = (const int*)m->row_ptr.ptr;
    const int* col = (const int*)m->col_idx.ptr;
    if (cudaMemsetAsync(s->bicp_l.ptr, 0, s->bicp_l.bytes, st) != cudaSuccess ||
        cudaMemsetAsync(s->bicp_linv.ptr, 0, s->bicp_linv.bytes, st) != cudaSuccess ||
        cudaMemsetAsync(status.ptr, 0, sizeof(int), st) != cudaSuccess) {
        set_error("fe_system_factor_bicp: memset failed");
        return fail(FE_ERR_CUDA);
    }
    k_bicp_tpos<<<blocks_of(n, 128), 128, 0, st>>>(n, rp, col, (int*)s->bicp_tpos.ptr, (int*)status.ptr);
    count_launches(1);
    k_bicp_levels<<<blocks_of(S, 32), 32, 0, st>>>(n, S, rp, col, (int*)lvl.ptr, (int4*)s->bicp_tab.ptr,
                                                   (int*)s->bicp_lev.ptr, (int*)s->bicp_nlev.ptr);
    count_launches(1);
    k_bicp_factor<<<blocks_of(S, 32), 32, 0, st>>>(n, S, rp, col, (const double2*)s->val64.ptr, s->stride,
                                                   (double2*)s->bicp_l.ptr, (double2*)s->bicp_linv.ptr,
                                                   (int*)status.ptr);
    count_launches(1);
    int hs = 0;
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&hs, status.ptr, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) {
        set_error("fe_system_factor_bicp: %s", cudaGetErrorString(ce));
        return fail(FE_ERR_CUDA);
    }
    if (hs & kDevBadIndex) {
        set_error("fe_system_factor_bicp: the block pattern is not structurally symmetric");
        return fail(FE_ERR_CUDA);
    }
    if (hs & kDevSingular) {
        set_error("fe_system_factor_bicp: a pivot of the incomplete factor is zero or not finite");
        return fail(FE_ERR_BREAKDOWN);
    }
    dev_free(st, lvl);
    dev_free(st, status);
    s->bicp_n_sub = S;
    return FE_OK;
}

fe_status fe_system_export_bicp(fe_ctx* ctx, const fe_system* s, void* l_c128, int32_t* n_sub) {
    if (!ctx || !s) {
        set_error("fe_system_export_bicp: NULL argument");
        return FE_ERR_INVALID_ARG;
    }
    if (s->bicp_n_sub < 1) {
        set_error("fe_system_export_bicp: no factor (call fe_system_factor_bicp first)");
        return FE_ERR_INVALID_ARG;
    }
    if (n_sub) *n_sub = s->bicp_n_sub;
    if (l_c128) {
        FE_CUDA(cudaMemcpyAsync(l_c128, s->bicp_l.ptr, s->bicp_l.bytes, cudaMemcpyDeviceToHost, ctx->stream));
        FE_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    return FE_OK;
}

}  // extern "C"
