// Device code of the persistent solve and its launch templates, shared by
// the host logic (solve.cu) and by one translation unit per product
// arithmetic (solve_fp64.cu, solve_mixed.cu, solve_df.cu) that instantiates
// the kernels, so that the three compile in parallel.
#pragma once

#include "krylov.cuh"

#include <algorithm>
#include <cstdlib>
#include <new>
#include <type_traits>
#include <vector>

namespace fe {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxNV = 11;    // reduced values per column and barrier
constexpr int kTraceIters = 64;
constexpr int kRowsPerWarpR1 = 10;   // R = 1 products: one thread per (row, component), 10 rows per warp
constexpr int kColsPerWarp = 272;    // >= 10 rows x 27 blocks
constexpr int kTracePhases = 8;

struct SyncState {
    unsigned count;
    unsigned gen;
    int err;
    int pad;
};

// Krylov storage.  The solution x, the recurrences (r, u, p, s) and all inner
// products are FP64; the sparse product of the Krylov loop runs in the
// matrix precision TM (complex64 in the mixed mode) on TM copies uM, pM of u
// and p.  FP64 recurrences and an FP64 block-Jacobi application keep the
// loop converging (with complex64 recurrences it stalls on these indefinite
// systems); the complex64 product halves the matrix bytes and runs on the
// FP32 pipes.  The FP64 true residual replaces the recursive one whenever the
// latter has dropped by `reliable` since the last replacement (reliable
// updates), so the Krylov directions are kept across refinements.
struct SolveParams {
    int n_rows, n_cta;
    const int* rp;
    const int* col;
    const double2* val64;
    const void* valM;       // matrix in the inner precision
    int64_t stride;         // plane stride of the block values
    const double2* dinv64;  // block-Jacobi inverse, applied in FP64
    const float4* dinvdf;   // its FP32 pairs (FE_PREC_DF: Krylov vectors are FP32 pairs)
    const signed char* row_class;  // regular-row class per row (-1: explicit blocks)
    const StencilSet* stencil;     // class stencils
    const int* cost_prefix;        // per-row product cost prefix [n_rows + 1] (product phases split by cost)
    int64_t cost_total;            // cost_prefix[n_rows] (host copy, sizes the halo buffer)
    int cost_min, cost_max;        // bounds of one row's cost (host only: halo sizing)
    const double2* b;
    double2* x;
    double2* r;
    double2* u;
    double2* p;
    double2* s;
    void* uM;  // u in the inner precision (aliases u when TM = double)
    void* pM;  // p in the inner precision (aliases p when TM = double)
    void* w;   // w = A uM in the inner precision
    SyncState* sync;
    double* partial;
    double* result;
    double tol, reliable;
    int restart;  // 1: a true-residual pass restarts the directions (p = s = 0); 0: keeps them
    int max_pass;  // iterations after which a restarting pass is replaced anyway (0: no cap)
    int max_iter, max_outer, use_x0;
    int halo;       // bound on |column rank - row rank|
    int stage;      // stage the CTA's uM halo in shared memory (1) or gather from L2 (0)
    int64_t halo_bytes;  // dynamic shared memory left for the halo (a CTA whose halo is larger gathers)
    int red_bytes;  // dynamic shared memory used by the column sums
    int col_bytes;  // dynamic shared memory for the per-warp column-index staging (R = 1)
    int* rep_status;
    int* rep_iters;
    int* rep_outer;
    double* rep_rel;
    unsigned long long* trace;  // optional [n_cta][kTraceIters][kTracePhases] timestamps
    unsigned long long timeout_ns;
    unsigned spin_ns;           // back-off between polls of the barrier generation
    // block incomplete Cholesky factor, one band per CTA (FP64 solves; null:
    // block Jacobi)
    const double2* bicp_l;      // [nnzb * 9] L_IJ by block slot, row-major 3x3
    const double2* bicp_linv;   // [n_rows * 9] L_II^{-1}
    const int* bicp_tpos;       // [nnzb] slot of the transposed block
    const int4* bicp_tab;       // [n_rows] band nodes by level: (node, first band slot, diagonal slot, band end)
    const int* bicp_lev;        // band b's level offsets at [first row + b, ...]
    const int* bicp_nlev;       // [n_cta] levels per band
};

// ---------------------------------------------------------------------------
// Grid barrier with fused reduction.  Every CTA writes NV partial values and
// arrives on a counter; the last arrival sums the partials of all CTAs in CTA
// order (lane-strided, then a fixed butterfly), publishes the NV results and
// bumps the generation.  One thread per CTA fences: the CTA barrier before
// it makes the whole CTA's writes part of its release (fences are
// cumulative).  Waits are bounded by P.timeout_ns; on expiry the CTA records
// kDevTimeout and every CTA leaves at its next barrier.
// ---------------------------------------------------------------------------
template <int NV>
__device__ __noinline__ bool grid_reduce(const SolveParams& P, int cta, const double* s_in, double* s_out) {
    __shared__ int s_last, s_ok;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int v = threadIdx.x; v < NV; v += kThreads) P.partial[(size_t)cta * NV + v] = s_in[v];
    __syncthreads();
    volatile unsigned* vgen = &P.sync->gen;
    volatile int* verr = &P.sync->err;
    if (threadIdx.x == 0) {
        const unsigned g = *vgen;
        __threadfence();
        const unsigned old = atomicAdd(&P.sync->count, 1u);
        s_ok = 1;
        s_last = old == (unsigned)P.n_cta - 1u;
        if (!s_last) {
            const unsigned long long t0 = globaltimer_ns();
            while (*vgen == g) {
                if (*verr) {
                    s_ok = 0;
                    break;
                }
                if (globaltimer_ns() - t0 > P.timeout_ns) {
                    atomicCAS(&P.sync->err, 0, kDevTimeout);
                    s_ok = 0;
                    break;
                }
                if (P.spin_ns) __nanosleep(P.spin_ns);
            }
        }
        __threadfence();
    }
    __syncthreads();
    if (s_last) {
        for (int v = warp; v < NV; v += kWarps) {
            double acc = 0.0;
            for (int c = lane; c < P.n_cta; c += 32) acc += __ldcg(P.partial + (size_t)c * NV + v);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) P.result[v] = acc;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicExch(&P.sync->count, 0u);
            __threadfence();
            atomicAdd(&P.sync->gen, 1u);
        }
    }
    if (threadIdx.x == 0 && *verr) s_ok = 0;
    for (int v = threadIdx.x; v < NV; v += kThreads) s_out[v] = __ldcg(P.result + v);
    __syncthreads();
    return s_ok != 0;
}

// Sum over the CTA of per-thread values, per column (thread t holds column
// t % R): a fixed butterfly inside each warp, then one warp per (value,
// column) adds the warp totals with a fixed butterfly.
template <int R, int NV>
__device__ __forceinline__ void cta_colsum(const double (&v)[NV], double* s_red, double* s_in) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double w = v[k];
#pragma unroll
        for (int o = 16; o >= R; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (lane < R) s_red[(k * kWarps + warp) * R + lane] = w;
    }
    __syncthreads();
    for (int i = warp; i < NV * R; i += kWarps) {
        const int k = i / R, c = i % R;
        double acc = s_red[(k * kWarps + lane) * R + c];  // kWarps == 32
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) s_in[i] = acc;
    }
    __syncthreads();
}

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C>
__device__ __forceinline__ C cfma(C a, C b, C c) {  // a * b + c
    return mk(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 to_c64(double2 a) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double2 to_c128(float2 a) { return make_double2(a.x, a.y); }
__device__ __forceinline__ double2 to_c128(double2 a) { return a; }
__device__ __forceinline__ double2 to_c128(float4 a) {  // FP32 pair -> FP64
    return make_double2((double)a.x + (double)a.z, (double)a.y + (double)a.w);
}
template <typename C>
__device__ __forceinline__ C from_c128(double2 a);
template <>
__device__ __forceinline__ float2 from_c128<float2>(double2 a) {
    return to_c64(a);
}
template <>
__device__ __forceinline__ double2 from_c128<double2>(double2 a) {
    return a;
}
template <>
__device__ __forceinline__ float4 from_c128<float4>(double2 a) {  // FP64 -> FP32 pair
    const float rh = __double2float_rn(a.x), ih = __double2float_rn(a.y);
    return make_float4(rh, ih, __double2float_rn(a.x - (double)rh), __double2float_rn(a.y - (double)ih));
}

// z = Dinv r for one node and column (3x3 complex block times 3-vector) in
// the inner precision C.
template <typename C>
__device__ __forceinline__ void apply_dinv(const C* __restrict__ dinv, int node, const C (&r)[3], C (&z)[3]) {
    C m[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) m[q] = ld_ro(dinv + (size_t)node * 9 + q);
#pragma unroll
    for (int al = 0; al < 3; ++al) {
        C acc = mk(decltype(C{}.x)(0), decltype(C{}.x)(0));
#pragma unroll
        for (int be = 0; be < 3; ++be) {
            acc.x += m[3 * al + be].x * r[be].x - m[3 * al + be].y * r[be].y;
            acc.y += m[3 * al + be].x * r[be].y + m[3 * al + be].y * r[be].x;
        }
        z[al] = acc;
    }
}

// Copies vector entries [3*h0*R, 3*h1*R) of v into the CTA's shared halo
// buffer with one bulk (TMA) copy; sets `shift` so that smem[i + shift]
// holds v[i].  Returns false when the bounded wait expired.
template <typename C, int R>
__device__ __forceinline__ bool stage_halo(const SolveParams& P, const C* v, int r0, int r1, char* halo_buf,
                                           uint64_t* mbar, unsigned& phase, int& shift) {
    const int h0 = max(0, r0 - P.halo), h1 = min(P.n_rows, r1 + P.halo);
    const size_t b0 = (size_t)3 * h0 * R * sizeof(C), b1 = (size_t)3 * h1 * R * sizeof(C);
    const size_t a0 = b0 & ~(size_t)15, a1 = (b1 + 15) & ~(size_t)15;
    if (threadIdx.x == 0) {
        fence_proxy_async();
        mbar_expect_tx(mbar, (unsigned)(a1 - a0));
        bulk_g2s(halo_buf, (const char*)v + a0, (unsigned)(a1 - a0), mbar);
    }
    // one decision for the whole CTA (no thread may leave while others wait at a barrier)
    const bool ok = __syncthreads_and(mbar_wait_bounded(mbar, phase & 1u, P.timeout_ns)) != 0;
    if (!ok) {
        atomicCAS(&P.sync->err, 0, kDevTimeout);
        // let the copy land before the CTA leaves (its shared memory is the destination)
        mbar_wait_bounded(mbar, phase & 1u, P.timeout_ns > 2000000000ull ? P.timeout_ns : 2000000000ull);
    }
    phase += 1;
    shift = (int)((b0 - a0) / sizeof(C)) - 3 * h0 * R;
    return ok;
}

// One Krylov product phase over the CTA's rows: w = A uM and, for columns
// whose s must be refreshed after a residual replacement, s = A pM; with the
// per-column FP64 partial dots
//   acc[0..1] = r^T u, acc[2..3] = u^T w, acc[4] = |r|^2,
//   acc[5..6] = u^T s, acc[7..8] = p^T w, acc[9..10] = p^T s (refresh only).
// NV = 5 (no column refreshes) or 11: the refresh accumulators exist only in
// the NV = 11 instance, which runs after a replacement.
template <typename TM, int R, bool kStaged, int NV>
__device__ __forceinline__ bool product_phase(const SolveParams& P, const typename CplxT<TM>::type* xs, int xshift,
                                              int r0, int r1, const int* s_refresh, bool any_refresh, int* s_cols,
                                              double (&acc)[NV]) {
    constexpr bool kRefresh = NV == 11;
    // FP32-pair vectors: dots accumulate as FP32 pairs, facc[2k] + facc[2k+1]
    // is acc[k] (converted to FP64 once, at the end of the phase)
    constexpr bool kDFV = std::is_same<TM, DFloat>::value && (R > 1);
    float facc[kDFV ? 2 * NV : 1] = {};
    bool ok = true;
    using C = typename CplxT<TM>::type;
    const C* valM = (const C*)P.valM;
    const C* uM = (const C*)P.uM;
    const C* pM = (const C*)P.pM;
    C* w = (C*)P.w;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto dots = [&](size_t o, const C& wy, bool refresh, const C& sy) {
      if constexpr (kDFV) {
        const float4 rv = ld_cg((const float4*)P.r + o), uv = ld_cg((const float4*)P.u + o);
        dfc_mac4(facc + 0, rv, uv);
        dfc_mac4(facc + 4, uv, wy);
        df_mac(facc[8], facc[9], rv.x, rv.z, rv.x, rv.z);
        df_mac(facc[8], facc[9], rv.y, rv.w, rv.y, rv.w);
        if constexpr (kRefresh) {
          if (refresh) {
            const float4 pv = ld_cg((const float4*)P.p + o);
            dfc_mac4(facc + 10 % (2 * NV), uv, sy);
            dfc_mac4(facc + 14 % (2 * NV), pv, wy);
            dfc_mac4(facc + 18 % (2 * NV), pv, sy);
            ((float4*)P.s)[o] = sy;
          }
        }
      } else {
        const double2 rv = __ldcg(P.r + o), uv = __ldcg(P.u + o), wd = to_c128(wy);
        acc[0] += rv.x * uv.x - rv.y * uv.y;
        acc[1] += rv.x * uv.y + rv.y * uv.x;
        acc[2] += uv.x * wd.x - uv.y * wd.y;
        acc[3] += uv.x * wd.y + uv.y * wd.x;
        acc[4] += rv.x * rv.x + rv.y * rv.y;
        if constexpr (kRefresh) {
          if (refresh) {
            const double2 pv = __ldcg(P.p + o), sd = to_c128(sy);
            acc[5 % NV] += uv.x * sd.x - uv.y * sd.y;
            acc[6 % NV] += uv.x * sd.y + uv.y * sd.x;
            acc[7 % NV] += pv.x * wd.x - pv.y * wd.y;
            acc[8 % NV] += pv.x * wd.y + pv.y * wd.x;
            acc[9 % NV] += pv.x * sd.x - pv.y * sd.y;
            acc[10 % NV] += pv.x * sd.y + pv.y * sd.x;
            P.s[o] = sd;
          }
        }
      }
    };
    if (R == 1) {
        // one thread per (row, component): ten rows per warp, their column
        // indices staged in shared memory first
        int* cols = s_cols + warp * kColsPerWarp;
        const bool refresh = kRefresh && s_refresh[0] != 0;
        const int al = lane % 3;
        for (int rb = r0 + warp * kRowsPerWarpR1; rb < r1; rb += kWarps * kRowsPerWarpR1) {
            const int re = min(rb + kRowsPerWarpR1, r1);
            const int sb = stage_cols(P.rp, P.col, rb, re, cols, lane);
            const int row = rb + lane / 3;
            if (lane < 30 && row < re) {
                const int s0 = __ldg(P.rp + row), s1 = __ldg(P.rp + row + 1);
                const int* rc = cols + (s0 - sb);
                // class stencils only in the complex64 kernels (keeps the FP64 kernel's registers)
                const int cls = (kClassPath<C> && P.row_class) ? __ldg(P.row_class + row) : -1;
                const int kind = cls >= 0 ? __ldg(&P.stencil->kind[cls]) : 0;
                const C y = kind ? row_component_class<C, kStaged>(P.stencil, cls, kind, rc, al, kStaged ? xs : uM,
                                                                   kStaged ? -xshift : 0)
                                 : row_component<C, kStaged>(valM, P.stride, rc, s0, s1, al, kStaged ? xs : uM,
                                                             kStaged ? -xshift : 0);
                const size_t o = (size_t)3 * row + al;
                w[o] = y;
                C sy = y;
                if (refresh)
                    sy = kind ? row_component_class<C, false>(P.stencil, cls, kind, rc, al, pM, 0)
                              : row_component<C, false>(valM, P.stride, rc, s0, s1, al, pM, 0);
                dots(o, y, refresh, sy);
            }
            __syncwarp();
        }
    } else {
        constexpr int kRowsPerWarp = 32 / R;
        const int c = lane % R;
        const bool refresh = kRefresh && s_refresh[c] != 0;
        for (int row = r0 + warp * kRowsPerWarp + lane / R; row < r1; row += kWarps * kRowsPerWarp) {
            const int s0 = __ldg(P.rp + row), s1 = __ldg(P.rp + row + 1);
            const int cls = (kClassPath<C> && P.row_class) ? __ldg(P.row_class + row) : -1;
            const int kind = cls >= 0 ? __ldg(&P.stencil->kind[cls]) : 0;
            C y[3], sy[3];
            if (kind)
                row_product_colx_class<C, kStaged>(P.stencil, cls, kind, P.col, s0, kStaged ? xs : uM,
                                                   kStaged ? -xshift : 0, R, c, y[0], y[1], y[2]);
            else
                row_product_colx<C, kStaged>(valM, P.stride, P.col, s0, s1, kStaged ? xs : uM, kStaged ? -xshift : 0,
                                             R, c, y[0], y[1], y[2]);
            if (refresh) {
                if (kind)
                    row_product_colx_class<C, false>(P.stencil, cls, kind, P.col, s0, pM, 0, R, c, sy[0], sy[1], sy[2]);
                else
                    row_product_colx<C, false>(valM, P.stride, P.col, s0, s1, pM, 0, R, c, sy[0], sy[1], sy[2]);
            }
#pragma unroll
            for (int al = 0; al < 3; ++al) {
                const size_t o = (size_t)(3 * row + al) * R + c;
                w[o] = y[al];
                dots(o, y[al], refresh, refresh ? sy[al] : y[al]);
            }
        }
    }
    if constexpr (kDFV) {
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += (double)facc[2 * k] + (double)facc[2 * k + 1];
    }
    (void)any_refresh;
    return ok;
}

// Diagnostics (FE_TRACE=1): every CTA stamps the end of each phase of its
// first kTraceIters iterations, [cta][iteration][phase]; after those stamps
// come kTraceStats values per CTA describing its product rows.
constexpr int kTraceStats = 8;
#define FE_TRACE_MARK(k)                                                                        \
    do {                                                                                        \
        if (P.trace && tid == 0 && trace_it < kTraceIters)                                      \
            P.trace[((size_t)cta * kTraceIters + trace_it) * kTracePhases + (k)] = globaltimer_ns(); \
    } while (0)

// z = (L L^T)^{-1} r over the CTA's band of rows (block incomplete Cholesky,
// Section 3.1.5.3; Eq. 6): the forward substitution
//     y_I = L_II^{-1} (r_I - sum_{J < I in the band} L_IJ y_J)
// level by level, then the back substitution
//     z_I = L_II^{-T} (y_I - sum_{J > I in the band} L_JI^T z_J)
// in reverse level order, in place in z.  Nodes of one level do not couple;
// a CTA barrier separates the levels.  One half-warp per (node, column):
// lane k takes the k-th band block on its side of the diagonal (at most 13
// on each side of a 27-point row; the node table gives the slot ranges, and
// the back substitution finds L_JI at the transposed slot, where the forward
// pass has just read it), so a node's block loads are issued together, and a
// fixed butterfly sums the lanes.  Only the columns with s_mask[c] != 0
// are written.  r and z are written earlier in this kernel, so they are read
// through the coherent path.
__device__ __forceinline__ double2 half_warp_csum(double2 v) {
#pragma unroll
    for (int m = 8; m >= 1; m >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, m);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, m);
    }
    return v;
}

// t = L v (kTrans = false) or L^T v (true) for one 3x3 block
template <bool kTrans>
__device__ __forceinline__ void block_times(const double2* __restrict__ L, double2 v0, double2 v1, double2 v2,
                                            double2& t0, double2& t1, double2& t2) {
    const double2 zero = make_double2(0.0, 0.0);
    constexpr int a = kTrans ? 3 : 1, b = kTrans ? 1 : 3;  // strides along v and along t
    t0 = cfma(__ldg(L + 2 * a), v2, cfma(__ldg(L + a), v1, cfma(__ldg(L + 0), v0, zero)));
    t1 = cfma(__ldg(L + b + 2 * a), v2, cfma(__ldg(L + b + a), v1, cfma(__ldg(L + b), v0, zero)));
    t2 = cfma(__ldg(L + 2 * b + 2 * a), v2, cfma(__ldg(L + 2 * b + a), v1, cfma(__ldg(L + 2 * b), v0, zero)));
}

template <int R>
__device__ __noinline__ void bicp_apply(const SolveParams& P, const int cta, const int r0, const double2* rv,
                                        double2* z, const int* s_mask) {
    constexpr int kItems = kThreads / 16;  // (node, column) items per pass
    const int sub = threadIdx.x & 15, item = threadIdx.x >> 4;
    const int nlev = __ldg(P.bicp_nlev + cta);
    const int* off = P.bicp_lev + r0 + cta;
    const int4* tab = P.bicp_tab + r0;
    const double2 zero = make_double2(0.0, 0.0);
    for (int pass = 0; pass < 2; ++pass) {  // 0: forward, 1: back
        for (int k = 0; k < nlev; ++k) {
            const int lv = pass == 0 ? k : nlev - 1 - k;
            const int a = __ldg(off + lv), n = (__ldg(off + lv + 1) - a) * R;
            // a warp holds items 2w and 2w + 1; warps with neither leave (the
            // condition is uniform over the warp, so its shuffles stay converged)
            for (int base = 0; base + (item & ~1) < n; base += kItems) {
                const int i = base + item;
                const int c = i % R;
                const bool on = i < n && s_mask[c] != 0;
                double2 t0 = zero, t1 = zero, t2 = zero, b0 = zero, b1 = zero, b2 = zero;
                size_t o = 0;
                int node = 0;
                if (on) {
                    const int4 e = __ldg(tab + a + i / R);
                    node = e.x;
                    o = (size_t)3 * node * R + c;
                    if (sub == 0) {  // the node's own values, needed after the sum
                        const double2* own = pass == 0 ? rv : z;
                        b0 = __ldcg(own + o);
                        b1 = __ldcg(own + o + R);
                        b2 = __ldcg(own + o + 2 * R);
                    }
                    const int p = (pass == 0 ? e.y : e.z + 1) + sub;
                    if (p < (pass == 0 ? e.z : e.w)) {
                        const int J = __ldg(P.col + p);
                        const size_t oj = (size_t)3 * J * R + c;
                        if (pass == 0)
                            block_times<false>(P.bicp_l + (size_t)p * 9, __ldcg(z + oj), __ldcg(z + oj + R),
                                               __ldcg(z + oj + 2 * R), t0, t1, t2);
                        else  // L_JI^T z_J
                            block_times<true>(P.bicp_l + (size_t)__ldg(P.bicp_tpos + p) * 9, __ldcg(z + oj),
                                              __ldcg(z + oj + R), __ldcg(z + oj + 2 * R), t0, t1, t2);
                    }
                }
                t0 = half_warp_csum(t0);
                t1 = half_warp_csum(t1);
                t2 = half_warp_csum(t2);
                if (on && sub == 0) {
                    t0 = make_double2(b0.x - t0.x, b0.y - t0.y);
                    t1 = make_double2(b1.x - t1.x, b1.y - t1.y);
                    t2 = make_double2(b2.x - t2.x, b2.y - t2.y);
                    const double2* M = P.bicp_linv + (size_t)node * 9;  // lower triangular
                    if (pass == 0) {  // z = M t
                        z[o] = cfma(__ldg(M + 0), t0, zero);
                        z[o + R] = cfma(__ldg(M + 4), t1, cfma(__ldg(M + 3), t0, zero));
                        z[o + 2 * R] = cfma(__ldg(M + 8), t2, cfma(__ldg(M + 7), t1, cfma(__ldg(M + 6), t0, zero)));
                    } else {  // z = M^T t
                        z[o] = cfma(__ldg(M + 6), t2, cfma(__ldg(M + 3), t1, cfma(__ldg(M + 0), t0, zero)));
                        z[o + R] = cfma(__ldg(M + 7), t2, cfma(__ldg(M + 4), t1, zero));
                        z[o + 2 * R] = cfma(__ldg(M + 8), t2, zero);
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Product phase of one CTA: optional TMA staging of its halo of uM, then the
// products with NV fused dots.  Returns false when a bounded wait expired (the
// error is recorded).
template <typename TM, int R, int NV>
__device__ __forceinline__ bool product_step(const SolveParams& P, int cta, bool stage_fits,
                                             const typename CplxT<TM>::type* uM, int pr0, int pr1, char* halo_buf,
                                             uint64_t* mbar, unsigned& mbar_phase, const int* s_refresh,
                                             bool any_refresh, int* s_cols, double (&acc)[NV], int trace_it) {
    using C = typename CplxT<TM>::type;
    const int tid = threadIdx.x;
    bool ok;
    if (stage_fits) {
        int shift = 0;
        if (!stage_halo<C, R>(P, uM, pr0, pr1, halo_buf, mbar, mbar_phase, shift)) return false;
        FE_TRACE_MARK(1);
        ok = product_phase<TM, R, true, NV>(P, (const C*)halo_buf, shift, pr0, pr1, s_refresh, any_refresh, s_cols,
                                            acc);
    } else {
        ok = product_phase<TM, R, false, NV>(P, nullptr, 0, pr0, pr1, s_refresh, any_refresh, s_cols, acc);
    }
    if (!ok && tid == 0) atomicCAS(&P.sync->err, 0, kDevTimeout);
    return ok;
}

// The persistent solve of A X = B for R right-hand sides.
//   [R] replacement: r = b - A x in FP64 for the columns that ask for it
//       (all at the start), norms, convergence test on the true residual;
//       then u = Dinv r and the inner-precision copies.
//   [A] product: w = A uM (s = A pM after a replacement), fused dots.
//   [B] scalars of the single-reduction COCG (Chronopoulos and Gear); after
//       a replacement the denominator p^T A p is expanded exactly from the
//       refreshed products instead of the recurrence.
//   [C] update: p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s,
//       u = Dinv r (one thread per dof, node components exchanged in shared
//       memory).
// Grid barriers separate the phases; [A] and [R] end in fused reductions.
template <typename TM, int R>
__device__ __forceinline__ void solve_body(const SolveParams& P, const int cta) {
    using C = typename CplxT<TM>::type;
    // Krylov vectors: FP64, or FP32 pairs in the FE_PREC_DF mode with several
    // columns (then the products read u and p directly and the updates run
    // on the FP32 pipes; with one column the FP64 recurrences converge in
    // fewer iterations and the update is cheap either way)
    constexpr bool kDFV = std::is_same<TM, DFloat>::value && (R > 1);
    using VT = std::conditional_t<kDFV, float4, double2>;
    VT* X = (VT*)P.x;
    VT* Rv = (VT*)P.r;
    VT* U = (VT*)P.u;
    VT* Pv = (VT*)P.p;
    VT* Sv = (VT*)P.s;
    C* uM = (C*)P.uM;
    C* pM = (C*)P.pM;
    const C* wv = (const C*)P.w;
    constexpr bool kSplit = !std::is_same<C, VT>::value;  // inner copies are separate buffers
    // block incomplete Cholesky instead of block Jacobi (FP64 solves only)
    constexpr bool kBicpType = std::is_same<TM, double>::value;
    const bool bicp = kBicpType && P.bicp_l != nullptr;

    extern __shared__ __align__(128) char dyn[];
    double* s_red = (double*)dyn;
    int* s_cols = (int*)(dyn + P.red_bytes);
    char* halo_buf = dyn + P.red_bytes + P.col_bytes;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ double s_in[kMaxNV * R], s_out[kMaxNV * R];
    __shared__ double s_bn[R], s_rr_ref[R], s_rel[R];
    __shared__ double s_gam_r[R], s_gam_i[R], s_al_r[R], s_al_i[R], s_be_r[R], s_be_i[R];
    __shared__ int s_bmask[R];  // columns a block incomplete Cholesky application writes
    __shared__ int s_active[R], s_done[R], s_status[R], s_iters[R], s_outer[R], s_first[R], s_refresh[R],
        s_repl[R], s_pass_it[R];
    __shared__ int s_any_repl, s_any_active, s_any_refresh;
    __shared__ double2 s_exch[kThreads];

    const int tid = threadIdx.x;
    // vector phases: equal row counts; product phases: equal product cost
    const int r0 = (int)((int64_t)cta * P.n_rows / P.n_cta);
    const int r1 = (int)((int64_t)(cta + 1) * P.n_rows / P.n_cta);
    __shared__ int s_pr[2];
    if (tid < 2 && !P.cost_prefix) s_pr[tid] = (int)((int64_t)(cta + tid) * P.n_rows / P.n_cta);
    if (tid < 2 && P.cost_prefix) {
        const int64_t total = P.cost_prefix[P.n_rows];
        const int64_t target = (int64_t)(cta + tid) * total / P.n_cta;
        int lo = 0, hi = P.n_rows;  // first row whose prefix >= target
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((int64_t)P.cost_prefix[mid] < target) lo = mid + 1;
            else hi = mid;
        }
        s_pr[tid] = (cta + tid == P.n_cta) ? P.n_rows : lo;
    }
    __syncthreads();
    const int pr0 = s_pr[0], pr1 = s_pr[1];
    if (P.trace && tid == 0) {  // product rows of this CTA: explicit rows and blocks, general, diagonal
        unsigned long long ne = 0, nb = 0, ng = 0, nd = 0;
        for (int row = pr0; row < pr1; ++row) {
            const int c = (kClassPath<TM> && P.row_class) ? P.row_class[row] : -1;
            const int kind = c >= 0 ? P.stencil->kind[c] : 0;
            if (kind == 1) ++ng;
            else if (kind == 2) ++nd;
            else {
                ++ne;
                nb += (unsigned long long)(P.rp[row + 1] - P.rp[row]);
            }
        }
        unsigned long long* st = P.trace + (size_t)P.n_cta * kTraceIters * kTracePhases + (size_t)cta * kTraceStats;
        st[0] = (unsigned long long)pr0;
        st[1] = (unsigned long long)pr1;
        st[2] = ne;
        st[3] = nb;
        st[4] = ng;
        st[5] = nd;
    }
    // stage the product input only if this CTA's halo fits the buffer
    const bool stage_fits = P.stage && [&] {
        const int h0 = max(0, pr0 - P.halo), h1 = min(P.n_rows, pr1 + P.halo);
        const size_t a0 = ((size_t)3 * h0 * R * sizeof(C)) & ~(size_t)15;
        const size_t a1 = ((size_t)3 * h1 * R * sizeof(C) + 15) & ~(size_t)15;
        return a1 - a0 <= (size_t)P.halo_bytes;
    }();
    const int n_items = (r1 - r0) * R;  // (node, column) pairs owned by this CTA
    const int my_c = tid % R;           // column of every item this thread handles
    const size_t base_o = (size_t)3 * r0 * R;
    unsigned mbar_phase = 0;
    int trace_it = 0;

    if (tid == 0) mbar_init(&s_mbar, 1);
    if (tid < R) {
        s_done[tid] = 0;
        s_status[tid] = FE_OK;
        s_iters[tid] = 0;
        s_pass_it[tid] = 0;
        s_outer[tid] = 0;
        s_active[tid] = 0;
        s_first[tid] = 1;
        s_refresh[tid] = 0;
        s_repl[tid] = 1;  // the first pass computes the initial residual
        s_rel[tid] = 0.0;
        s_bn[tid] = 0.0;
    }
    for (int i = tid; i < 3 * n_items; i += kThreads) {
        if (!P.use_x0) P.x[base_o + i] = make_double2(0.0, 0.0);  // zero bits: also a zero FP32 pair
        else if constexpr (kDFV) X[base_o + i] = from_c128<float4>(P.x[base_o + i]);  // in place, same size
        P.p[base_o + i] = make_double2(0.0, 0.0);
        P.s[base_o + i] = make_double2(0.0, 0.0);
    }
    if (tid == 0) s_any_repl = 1;
    __syncthreads();
    if (!grid_reduce<0>(P, cta, s_in, s_out)) goto out;

    for (;;) {
        if (s_any_repl) {
            // ---- [R] FP64 true residual for the columns that ask for it ----
            if constexpr (kDFV) {  // FP64 copy of x for the product (w is free until the next product)
                double2* xd = (double2*)P.w;
                for (int i = tid; i < 3 * n_items; i += kThreads) xd[base_o + i] = to_c128(X[base_o + i]);
                if (!grid_reduce<0>(P, cta, s_in, s_out)) goto out;
            }
            {
                const double2* xsrc = kDFV ? (const double2*)P.w : P.x;
                double acc[2] = {0.0, 0.0};
                const int lane = tid & 31, warp = tid >> 5;
                if (R == 1) {
                    if (s_repl[0]) {
                        int* cols = s_cols + warp * kColsPerWarp;
                        const int al = lane % 3;
                        for (int rb = pr0 + warp * kRowsPerWarpR1; rb < pr1; rb += kWarps * kRowsPerWarpR1) {
                            const int re = min(rb + kRowsPerWarpR1, pr1);
                            const int sb = stage_cols(P.rp, P.col, rb, re, cols, lane);
                            const int row = rb + lane / 3;
                            if (lane < 30 && row < re) {
                                const int s0 = __ldg(P.rp + row), s1 = __ldg(P.rp + row + 1);
                                const size_t o = (size_t)3 * row + al;
                                const double2 bv = __ldg(P.b + o);
                                const int cls = (kClassPath<TM> && P.row_class) ? __ldg(P.row_class + row) : -1;
                                const int kind = cls >= 0 ? __ldg(&P.stencil->kind[cls]) : 0;
                                const double2 y =
                                    kind ? row_component_class<double2, false>(P.stencil, cls, kind, cols + (s0 - sb),
                                                                               al, xsrc, 0)
                                         : row_component<double2, false>(P.val64, P.stride, cols + (s0 - sb), s0, s1,
                                                                         al, xsrc, 0);
                                const double2 rv = make_double2(bv.x - y.x, bv.y - y.y);
                                Rv[o] = from_c128<VT>(rv);
                                acc[0] += rv.x * rv.x + rv.y * rv.y;
                                acc[1] += bv.x * bv.x + bv.y * bv.y;
                            }
                            __syncwarp();
                        }
                    }
                } else {
                    constexpr int kRowsPerWarp = 32 / R;
                    const int c = lane % R;
                    if (s_repl[c]) {
                        for (int row = pr0 + warp * kRowsPerWarp + lane / R; row < pr1;
                             row += kWarps * kRowsPerWarp) {
                            double2 y[3];
                            row_product_colx<double2, false>(P.val64, P.stride, P.col, __ldg(P.rp + row),
                                                             __ldg(P.rp + row + 1), xsrc, 0, R, c, y[0], y[1], y[2]);
#pragma unroll
                            for (int al = 0; al < 3; ++al) {
                                const size_t o = (size_t)(3 * row + al) * R + c;
                                const double2 bv = __ldg(P.b + o);
                                const double2 rv = make_double2(bv.x - y[al].x, bv.y - y[al].y);
                                Rv[o] = from_c128<VT>(rv);
                                acc[0] += rv.x * rv.x + rv.y * rv.y;
                                acc[1] += bv.x * bv.x + bv.y * bv.y;
                            }
                        }
                    }
                }
                cta_colsum<R, 2>(acc, s_red, s_in);
                if (!grid_reduce<2 * R>(P, cta, s_in, s_out)) goto out;
            }
            if (tid < R) {
                const int c = tid;
                if (s_repl[c] && !s_done[c]) {
                    if (s_first[c] && s_outer[c] == 0) s_bn[c] = sqrt(s_out[R + c]);
                    const double rn = sqrt(s_out[c]), bn = s_bn[c];
                    const double rel = bn > 0.0 ? rn / bn : 0.0;
                    s_rel[c] = rel;
                    s_outer[c] += 1;
                    s_active[c] = 0;
                    if (!(rel == rel)) {
                        s_done[c] = 1;
                        s_status[c] = FE_ERR_NOT_CONVERGED;
                    } else if (rel <= P.tol) {
                        s_done[c] = 1;
                        s_status[c] = FE_OK;
                    } else if (s_iters[c] >= P.max_iter || s_outer[c] > P.max_outer) {
                        s_done[c] = 1;
                        s_status[c] = FE_ERR_NOT_CONVERGED;
                    } else {
                        s_active[c] = 1;
                        s_rr_ref[c] = rn * rn;
                        s_pass_it[c] = 0;
                        s_refresh[c] = s_first[c] ? 0 : 1;
                    }
                } else if (s_repl[c]) {
                    s_active[c] = 0;
                }
            }
            __syncthreads();
            // u = Dinv r and the inner-precision copies for the replaced columns
            {
                constexpr int kChunk = (kThreads / (3 * R)) * (3 * R);
                const bool act = s_repl[my_c] && s_active[my_c];
                const int n3 = 3 * n_items;
                for (int base = 0; base < n3; base += kChunk) {
                    const int i = base + tid;
                    const bool valid = act && tid < kChunk && i < n3;
                    const size_t o = base_o + i;
                    double2 rv = make_double2(0.0, 0.0);
                    if (valid) {
                        rv = to_c128(ld_cg(Rv + o));
                        if (kSplit) pM[o] = from_c128<C>(__ldcg(P.p + o));
                    }
                    s_exch[tid] = rv;
                    __syncthreads();
                    if (valid && !bicp) {
                        const int node = r0 + i / (3 * R);
                        const int al = (i / R) % 3;
                        const double2* drow = P.dinv64 + (size_t)node * 9 + 3 * al;
                        double2 uu = make_double2(0.0, 0.0);
#pragma unroll
                        for (int be = 0; be < 3; ++be) uu = cfma(__ldg(drow + be), s_exch[tid + (be - al) * R], uu);
                        U[o] = from_c128<VT>(uu);
                        if (kSplit) uM[o] = from_c128<C>(uu);
                    }
                    __syncthreads();
                }
                if constexpr (kBicpType) {
                    if (bicp) {
                        if (tid < R) s_bmask[tid] = s_repl[tid] && s_active[tid];
                        __syncthreads();
                        bicp_apply<R>(P, cta, r0, P.r, P.u, s_bmask);
                    }
                }
            }
            if (tid == 0) {
                int any = 0, refr = 0;
                for (int c = 0; c < R; ++c) {
                    s_repl[c] = 0;
                    any |= s_active[c];
                    refr |= s_refresh[c];
                }
                s_any_active = any;
                s_any_refresh = refr;
                s_any_repl = 0;
            }
            if (!grid_reduce<0>(P, cta, s_in, s_out)) goto out;
            {
                int any = 0;
                for (int c = 0; c < R; ++c) any |= !s_done[c];
                if (!any) break;
            }
        }

        // ---- [A] products and fused dots ----
        FE_TRACE_MARK(0);
        if (s_any_refresh) {
            double acc[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
            if (!product_step<TM, R, 11>(P, cta, stage_fits, uM, pr0, pr1, halo_buf, &s_mbar, mbar_phase, s_refresh,
                                         s_any_refresh, s_cols, acc, trace_it))
                goto out;
            FE_TRACE_MARK(2);
            cta_colsum<R, 11>(acc, s_red, s_in);
            FE_TRACE_MARK(3);
            if (!grid_reduce<11 * R>(P, cta, s_in, s_out)) goto out;
        } else {
            double acc[5] = {0, 0, 0, 0, 0};
            if (!product_step<TM, R, 5>(P, cta, stage_fits, uM, pr0, pr1, halo_buf, &s_mbar, mbar_phase, s_refresh,
                                        s_any_refresh, s_cols, acc, trace_it))
                goto out;
            FE_TRACE_MARK(2);
            cta_colsum<R, 5>(acc, s_red, s_in);
            FE_TRACE_MARK(3);
            if (!grid_reduce<5 * R>(P, cta, s_in, s_out)) goto out;
        }
        FE_TRACE_MARK(4);
        // ---- [B] scalars ----
        // B1: does any column need its true residual first?  (No state of the
        // other columns changes in a replacement round: they redo the same
        // products next round.)
        if (tid < R) {
            const int c = tid;
            if (s_active[c]) {
                const double rr = s_out[4 * R + c];
                const double tb = P.tol * s_bn[c];
                const bool small = rr <= tb * tb || rr < P.reliable * P.reliable * s_rr_ref[c];
                const bool stalled = P.restart && P.max_pass > 0 && s_pass_it[c] >= P.max_pass;
                if (!(rr == rr) || s_iters[c] >= P.max_iter || (!s_first[c] && (small || stalled))) {
                    s_repl[c] = 1;
                    if (P.restart) s_first[c] = 1;
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            int any_repl = 0;
            for (int c = 0; c < R; ++c) any_repl |= s_repl[c];
            s_any_repl = any_repl;
        }
        __syncthreads();
        if (s_any_repl) {
            for (int i = tid; i < 3 * n_items; i += kThreads) {
                const int c = i % R;
                if (s_repl[c] && s_first[c]) {
                    P.p[base_o + i] = make_double2(0.0, 0.0);
                    P.s[base_o + i] = make_double2(0.0, 0.0);
                }
            }
            continue;
        }
        // B2: Chronopoulos-Gear scalars (exact p^T A p after a replacement)
        if (tid < R) {
            const int c = tid;
            if (s_active[c]) {
                const double gr = s_out[c], gi = s_out[R + c];
                const double dr = s_out[2 * R + c], di = s_out[3 * R + c];
                double br = 0.0, bi = 0.0, er = dr, ei = di;
                if (!s_first[c]) {
                    // beta = gamma / gamma_old
                    const double ig = rcp64(s_gam_r[c] * s_gam_r[c] + s_gam_i[c] * s_gam_i[c]);
                    br = (gr * s_gam_r[c] + gi * s_gam_i[c]) * ig;
                    bi = (gi * s_gam_r[c] - gr * s_gam_i[c]) * ig;
                    if (s_refresh[c]) {
                        // p^T A p for p = u + beta p_old: u^T w + beta (u^T s + p^T w) + beta^2 p^T s
                        const double e12r = s_out[5 * R + c] + s_out[7 * R + c];
                        const double e12i = s_out[6 * R + c] + s_out[8 * R + c];
                        const double e3r = s_out[9 * R + c], e3i = s_out[10 * R + c];
                        const double b2r = br * br - bi * bi, b2i = 2.0 * br * bi;
                        er = dr + (br * e12r - bi * e12i) + (b2r * e3r - b2i * e3i);
                        ei = di + (br * e12i + bi * e12r) + (b2r * e3i + b2i * e3r);
                    } else {
                        // delta - beta gamma / alpha_old
                        const double tr = br * gr - bi * gi, ti = br * gi + bi * gr;
                        const double ia = rcp64(s_al_r[c] * s_al_r[c] + s_al_i[c] * s_al_i[c]);
                        er = dr - (tr * s_al_r[c] + ti * s_al_i[c]) * ia;
                        ei = di - (ti * s_al_r[c] - tr * s_al_i[c]) * ia;
                    }
                }
                const double ed = er * er + ei * ei;
                const double gg = gr * gr + gi * gi;
                if (!(ed > 0.0) || !(ed < 1e300) || !(gg > 0.0)) {
                    if (s_first[c]) {  // breakdown right after a (re)start
                        s_active[c] = 0;
                        s_done[c] = 1;
                        s_status[c] = FE_ERR_BREAKDOWN;
                    } else {  // restart from the true residual next round
                        s_repl[c] = 1;
                        s_first[c] = 1;
                    }
                } else {
                    const double ie = rcp64(ed);
                    s_al_r[c] = (gr * er + gi * ei) * ie;
                    s_al_i[c] = (gi * er - gr * ei) * ie;
                    s_be_r[c] = br;
                    s_be_i[c] = bi;
                    s_gam_r[c] = gr;
                    s_gam_i[c] = gi;
                    s_iters[c] += 1;
                    s_pass_it[c] += 1;
                    s_first[c] = 0;
                    s_refresh[c] = 0;
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            int any_repl = 0, refr = 0;
            for (int c = 0; c < R; ++c) {
                any_repl |= s_repl[c];
                refr |= s_refresh[c];
            }
            s_any_repl = any_repl;  // a breakdown restarts at the top of the next round
            s_any_refresh = refr;
        }
        __syncthreads();
        FE_TRACE_MARK(5);
        // ---- [C] update, one thread per (dof, column) ----
        {
            const bool act = s_active[my_c] != 0 && !s_repl[my_c];
            if (s_active[my_c] && s_repl[my_c])
                for (int i = tid; i < 3 * n_items; i += kThreads) {
                    P.p[base_o + i] = make_double2(0.0, 0.0);
                    P.s[base_o + i] = make_double2(0.0, 0.0);
                }
            const double2 alpha = make_double2(s_al_r[my_c], s_al_i[my_c]);
            const double2 nalpha = make_double2(-s_al_r[my_c], -s_al_i[my_c]);
            const double2 beta = make_double2(s_be_r[my_c], s_be_i[my_c]);
            constexpr int kChunk = (kThreads / (3 * R)) * (3 * R);
            const int n3 = 3 * n_items;
            if constexpr (kDFV) {  // the same update in FP32-pair arithmetic
                const float4 a4 = from_c128<float4>(alpha), na4 = from_c128<float4>(nalpha);
                const float4 b4 = from_c128<float4>(beta);
                float4* ex = (float4*)s_exch;
                for (int base = 0; base < n3; base += kChunk) {
                    const int i = base + tid;
                    const bool valid = act && tid < kChunk && i < n3;
                    const size_t o = base_o + i;
                    float4 rn = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (valid) {
                        const float4 pp = dfc_axpy(ld_cg(U + o), b4, ld_cg(Pv + o));
                        const float4 ss = dfc_axpy(ld_cg(wv + o), b4, ld_cg(Sv + o));
                        Pv[o] = pp;
                        Sv[o] = ss;
                        X[o] = dfc_axpy(ld_cg(X + o), a4, pp);
                        rn = dfc_axpy(ld_cg(Rv + o), na4, ss);
                        Rv[o] = rn;
                    }
                    ex[tid] = rn;
                    __syncthreads();
                    if (valid) {
                        const int node = r0 + i / (3 * R);
                        const int al = (i / R) % 3;
                        const float4* drow = P.dinvdf + (size_t)node * 9 + 3 * al;
                        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                        for (int be = 0; be < 3; ++be) dfc_mac(acc, __ldg(drow + be), ex[tid + (be - al) * R]);
                        U[o] = df_result_norm(acc);
                    }
                    __syncthreads();
                }
            } else
            for (int base = 0; base < n3; base += kChunk) {
                const int i = base + tid;
                const bool valid = act && tid < kChunk && i < n3;
                const size_t o = base_o + i;
                double2 rn = make_double2(0.0, 0.0);
                if (valid) {
                    const double2 pp = cfma(beta, __ldcg(P.p + o), __ldcg(P.u + o));
                    const double2 ss = cfma(beta, __ldcg(P.s + o), to_c128(ld_cg(wv + o)));
                    P.p[o] = pp;
                    P.s[o] = ss;
                    P.x[o] = cfma(alpha, pp, __ldcg(P.x + o));
                    rn = cfma(nalpha, ss, __ldcg(P.r + o));
                    P.r[o] = rn;
                }
                s_exch[tid] = rn;
                __syncthreads();
                if (valid && !bicp) {
                    const int node = r0 + i / (3 * R);
                    const int al = (i / R) % 3;
                    const double2* drow = P.dinv64 + (size_t)node * 9 + 3 * al;
                    double2 uu = make_double2(0.0, 0.0);
#pragma unroll
                    for (int be = 0; be < 3; ++be) uu = cfma(__ldg(drow + be), s_exch[tid + (be - al) * R], uu);
                    P.u[o] = uu;
                    if (kSplit) uM[o] = from_c128<C>(uu);
                }
                __syncthreads();
            }
            if constexpr (kBicpType) {
                if (bicp) {
                    if (tid < R) s_bmask[tid] = s_active[tid] && !s_repl[tid];
                    __syncthreads();
                    bicp_apply<R>(P, cta, r0, P.r, P.u, s_bmask);
                }
            }
        }
        FE_TRACE_MARK(6);
        if (!grid_reduce<0>(P, cta, s_in, s_out)) goto out;
        FE_TRACE_MARK(7);
        ++trace_it;
    }
out:
    if constexpr (kDFV) {  // the solution back to FP64, in place (every CTA its own rows)
        __syncthreads();
        for (int i = tid; i < 3 * n_items; i += kThreads) P.x[base_o + i] = to_c128(X[base_o + i]);
    }
    if (cta == 0 && tid < R) {
        P.rep_status[tid] = s_status[tid];
        P.rep_iters[tid] = s_iters[tid];
        P.rep_outer[tid] = s_outer[tid];
        P.rep_rel[tid] = s_rel[tid];
    }
}

// One system: CTA b of the grid is CTA b of the system.
template <typename TM, int R>
__global__ void __launch_bounds__(kThreads, 1) k_solve(SolveParams P) {
    solve_body<TM, R>(P, blockIdx.x);
}

// Several independent systems in one cooperative launch: job j owns the CTAs
// [cta0[j], cta0[j + 1]) and synchronises only among them (its own barrier
// state, partials and reports).  A CTA copies its job's parameters into
// shared memory once.
template <typename TM, int R>
__global__ void __launch_bounds__(kThreads, 1)
    k_solve_jobs(const SolveParams* __restrict__ jobs, const int* __restrict__ cta0, int n_jobs) {
    __shared__ __align__(16) SolveParams sP;
    __shared__ int s_job;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n_jobs - 1;  // last job whose first CTA is <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cta0[mid] <= (int)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        s_job = lo;
    }
    __syncthreads();
    const int j = s_job;
    static_assert(sizeof(SolveParams) % sizeof(int) == 0, "parameter block copied as ints");
    const int* src = (const int*)(jobs + j);
    int* dst = (int*)&sP;
    for (int i = threadIdx.x; i < (int)(sizeof(SolveParams) / sizeof(int)); i += kThreads) dst[i] = src[i];
    __syncthreads();
    solve_body<TM, R>(sP, (int)blockIdx.x - cta0[j]);
}

struct Workspace {
    DevBuf b, x, r, u, p, s, uM, pM, w, partial, result, sync, rep, trace;
};

constexpr size_t kSmemBudget = 200 * 1024;  // dynamic; static shared memory adds ~20 KB

template <typename T, int R>
fe_status launch_solve(fe_ctx* ctx, SolveParams& P) {
    static_assert(kWarps == 32, "cta_colsum assumes 32 warps");
    using C = typename CplxT<T>::type;
    // one CTA per SM; the reduction scratch and (when it fits) the CTA's
    // vector halo live in dynamic shared memory
    P.n_cta = std::min(ctx->num_sms, std::max(1, P.n_rows));
    P.red_bytes = (int)(kMaxNV * kWarps * R * sizeof(double));
    P.col_bytes = R == 1 ? (int)(kWarps * kColsPerWarp * sizeof(int)) : 0;
    // product phases: a CTA's range costs at most total / n_cta plus one row
    const int64_t rows_per_cta =
        std::min<int64_t>(P.n_rows, (P.cost_total / P.n_cta + P.cost_max) / P.cost_min + 2);
    const int64_t halo_bytes = (rows_per_cta + 2 * (int64_t)P.halo + 2) * 3 * R * (int64_t)sizeof(C) + 64;
    P.stage = (P.halo > 0 && (size_t)P.red_bytes + P.col_bytes + (size_t)halo_bytes <= kSmemBudget) ? 1 : 0;
    P.halo_bytes = P.stage ? halo_bytes : 0;
    const size_t dyn = (size_t)P.red_bytes + P.col_bytes + (P.stage ? (size_t)halo_bytes : 0);
    FE_CUDA(cudaFuncSetAttribute((const void*)k_solve<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    int per_sm = 0;
    FE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve<T, R>, kThreads, dyn));
    if (per_sm < 1) {
        set_error("solve kernel does not fit on an SM");
        return FE_ERR_CUDA;
    }
    void* args[] = {&P};
    FE_CUDA(cudaEventRecord(ctx->ev0, ctx->stream));
    FE_CUDA(cudaLaunchCooperativeKernel((void*)k_solve<T, R>, dim3(P.n_cta), dim3(kThreads), args, dyn,
                                        ctx->stream));
    FE_CUDA(cudaEventRecord(ctx->ev1, ctx->stream));
    count_launches(1);
    ctx->last_solve.launches += 1;
    ctx->last_solve.tile_width = R;
    ctx->last_solve.grid_ctas = P.n_cta;
    return FE_OK;
}

template <typename T>
fe_status dispatch(fe_ctx* ctx, int R, SolveParams& P) {
    switch (R) {
        case 1: return launch_solve<T, 1>(ctx, P);
        case 2: return launch_solve<T, 2>(ctx, P);
        case 4: return launch_solve<T, 4>(ctx, P);
        case 8: return launch_solve<T, 8>(ctx, P);
        case 16: return launch_solve<T, 16>(ctx, P);
        case 32: return launch_solve<T, 32>(ctx, P);
        default: set_error("unsupported tile width %d", R); return FE_ERR_UNSUPPORTED;
    }
}

// ---------------------------------------------------------------------------
// Jobs: independent solves that share one cooperative launch.  A job is one
// system with up to 32 right-hand sides, padded to a power-of-two tile width
// with zero columns (a zero right-hand side is converged at its first
// residual).  The server packs jobs of one width and precision into a launch.
// ---------------------------------------------------------------------------
struct SolveJob {
    const fe_system* sys = nullptr;
    int nrhs = 0, R = 1;
    int prec = FE_PREC_FP64;
    int64_t n_dof = 0;
    Workspace w;
    SolveParams P{};
};

template <typename T, int R>
fe_status launch_jobs_t(fe_ctx* ctx, SolveJob* const* jobs, const int* n_cta, int n) {
    using C = typename CplxT<T>::type;
    std::vector<SolveParams> Ps(n);
    std::vector<int> cta0(n + 1, 0);
    const int red_bytes = (int)(kMaxNV * kWarps * R * sizeof(double));
    const int col_bytes = R == 1 ? (int)(kWarps * kColsPerWarp * sizeof(int)) : 0;
    size_t dyn = (size_t)red_bytes + col_bytes;
    for (int i = 0; i < n; ++i) {
        SolveParams& P = Ps[i];
        P = jobs[i]->P;
        P.n_cta = n_cta[i];
        P.red_bytes = red_bytes;
        P.col_bytes = col_bytes;
        const int64_t rows_per_cta =
            std::min<int64_t>(P.n_rows, (P.cost_total / P.n_cta + P.cost_max) / P.cost_min + 2);
        const int64_t halo_bytes = (rows_per_cta + 2 * (int64_t)P.halo + 2) * 3 * R * (int64_t)sizeof(C) + 64;
        const size_t need = (size_t)red_bytes + col_bytes + (size_t)halo_bytes;
        P.stage = (P.halo > 0 && need <= kSmemBudget) ? 1 : 0;
        if (P.stage) dyn = std::max(dyn, need);
        cta0[i + 1] = cta0[i] + n_cta[i];
        FE_CUDA(cudaMemsetAsync(P.sync, 0, sizeof(SyncState), ctx->stream));
    }
    for (int i = 0; i < n; ++i) Ps[i].halo_bytes = (int64_t)dyn - red_bytes - col_bytes;
    const int grid = cta0[n];
    DevBuf dparams, dcta;
    FE_TRY(dev_alloc(ctx->stream, dparams, (size_t)n * sizeof(SolveParams)));
    fe_status e = dev_alloc(ctx->stream, dcta, (size_t)(n + 1) * sizeof(int));
    if (e != FE_OK) {
        dev_free(ctx->stream, dparams);
        return e;
    }
    auto done = [&](fe_status st) {
        dev_free(ctx->stream, dparams);
        dev_free(ctx->stream, dcta);
        return st;
    };
    if (cudaMemcpyAsync(dparams.ptr, Ps.data(), (size_t)n * sizeof(SolveParams), cudaMemcpyHostToDevice,
                        ctx->stream) != cudaSuccess ||
        cudaMemcpyAsync(dcta.ptr, cta0.data(), (size_t)(n + 1) * sizeof(int), cudaMemcpyHostToDevice,
                        ctx->stream) != cudaSuccess) {
        set_error("jobs: parameter upload failed");
        return done(FE_ERR_CUDA);
    }
    if (cudaFuncSetAttribute((const void*)k_solve_jobs<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)dyn) != cudaSuccess) {
        set_error("jobs: shared-memory attribute rejected");
        return done(FE_ERR_CUDA);
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_jobs<T, R>, kThreads, dyn);
    if (per_sm < 1 || grid > per_sm * ctx->num_sms) {
        set_error("jobs: %d CTAs do not fit on the device at once", grid);
        return done(FE_ERR_INVALID_ARG);
    }
    const SolveParams* pp = (const SolveParams*)dparams.ptr;
    const int* pc = (const int*)dcta.ptr;
    void* args[] = {(void*)&pp, (void*)&pc, (void*)&n};
    cudaEventRecord(ctx->ev0, ctx->stream);
    const cudaError_t le = cudaLaunchCooperativeKernel((void*)k_solve_jobs<T, R>, dim3(grid), dim3(kThreads), args,
                                                       dyn, ctx->stream);
    if (le != cudaSuccess) {
        set_error("jobs: launch failed: %s", cudaGetErrorString(le));
        return done(FE_ERR_CUDA);
    }
    cudaEventRecord(ctx->ev1, ctx->stream);
    count_launches(1);
    return done(FE_OK);
}

template <typename T>
fe_status launch_jobs_w(fe_ctx* ctx, int R, SolveJob* const* jobs, const int* n_cta, int n) {
    switch (R) {
        case 1: return launch_jobs_t<T, 1>(ctx, jobs, n_cta, n);
        case 2: return launch_jobs_t<T, 2>(ctx, jobs, n_cta, n);
        case 4: return launch_jobs_t<T, 4>(ctx, jobs, n_cta, n);
        case 8: return launch_jobs_t<T, 8>(ctx, jobs, n_cta, n);
        case 16: return launch_jobs_t<T, 16>(ctx, jobs, n_cta, n);
        case 32: return launch_jobs_t<T, 32>(ctx, jobs, n_cta, n);
        default: set_error("jobs: unsupported tile width %d", R); return FE_ERR_UNSUPPORTED;
    }
}

}  // namespace fe
