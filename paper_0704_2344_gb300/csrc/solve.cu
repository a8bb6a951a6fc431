// Solve of the complex-symmetric system A X = B.
//
// The paper solves with conjugate gradients and diagonal preconditioning
// (Sections 3.1.5.1 and 4.2.5.1): per iteration one matrix-vector product
// plus vector updates.  On a complex symmetric matrix the consistent variant
// uses the unconjugated bilinear form u^T v (COCG); the diagonal
// preconditioner becomes the inverse of each node's 3x3 diagonal block.
//
// Everything of one solve runs in ONE persistent cooperative launch: the FP64
// true residual r = b - A x, the inner COCG passes (complex64 in the mixed
// mode, complex128 in the plain mode), the FP64 solution update, and every
// convergence decision.  CTAs own contiguous ranges of block rows and meet
// at a grid barrier whose wait is bounded in time; the barrier also performs
// the dot-product reductions: each CTA publishes its partial sums and the
// last CTA to arrive adds them in a fixed order, so every CTA sees bitwise the
// same scalars and takes the same branch.
#include "krylov.cuh"

#include <algorithm>
#include <new>

namespace fe {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;

struct SyncState {
    unsigned count;
    unsigned gen;
    int err;
    int pad;
};

struct SolveParams {
    int n_rows, n_cta;
    const int* rp;
    const int* col;
    const double2* val64;
    const void* valT;
    const void* dinvT;
    const double2* b;
    double2* x;
    double2* r64;
    void* d;
    void* r;
    void* z;
    void* p;
    void* q;
    SyncState* sync;
    double* partial;
    double* result;
    double tol, inner_tol;
    int max_iter, max_outer, use_x0, pad;
    int* rep_status;
    int* rep_iters;
    int* rep_outer;
    double* rep_rel;
    unsigned long long timeout_ns;
};

// ---------------------------------------------------------------------------
// Grid barrier with fused reduction.  Every CTA writes NV partial values,
// arrives on a counter; the last arrival sums the partials of all CTAs in
// CTA order (lane-strided, then a fixed butterfly), publishes the NV results
// and bumps the generation.  Waits are bounded by P.timeout_ns; on expiry the
// CTA records kDevTimeout and every CTA leaves at its next barrier.
// ---------------------------------------------------------------------------
template <int NV>
__device__ __noinline__ bool grid_reduce(const SolveParams& P, const double* s_in, double* s_out) {
    __shared__ int s_last, s_ok;
    __shared__ unsigned s_gen;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int v = threadIdx.x; v < NV; v += kThreads) P.partial[(size_t)blockIdx.x * NV + v] = s_in[v];
    __threadfence();
    __syncthreads();
    volatile unsigned* vgen = &P.sync->gen;
    volatile int* verr = &P.sync->err;
    if (threadIdx.x == 0) {
        const unsigned g = *vgen;
        __threadfence();
        const unsigned old = atomicAdd(&P.sync->count, 1u);
        s_last = old == (unsigned)P.n_cta - 1u;
        s_gen = g;
        s_ok = 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int v = warp; v < NV; v += kWarps) {
            double acc = 0.0;
            for (int c = lane; c < P.n_cta; c += 32) acc += __ldcg(P.partial + (size_t)c * NV + v);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) P.result[v] = acc;
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicExch(&P.sync->count, 0u);
            __threadfence();
            atomicAdd(&P.sync->gen, 1u);
        }
    } else if (threadIdx.x == 0) {
        const unsigned long long t0 = globaltimer_ns();
        while (*vgen == s_gen) {
            if (*verr) {
                s_ok = 0;
                break;
            }
            if (globaltimer_ns() - t0 > P.timeout_ns) {
                atomicCAS(&P.sync->err, 0, kDevTimeout);
                s_ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0 && *verr) s_ok = 0;
    for (int v = threadIdx.x; v < NV; v += kThreads) s_out[v] = __ldcg(P.result + v);
    __syncthreads();
    return s_ok != 0;
}

// Sum over the CTA of per-thread values, per column (thread t holds column
// t % R): fixed butterfly inside a warp, then warps in order.
template <int R, int NV>
__device__ __forceinline__ void cta_colsum(const double (&v)[NV], double* s_red, double* s_in) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double w[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        w[k] = v[k];
#pragma unroll
        for (int o = 16; o >= R; o >>= 1) w[k] += __shfl_xor_sync(0xffffffffu, w[k], o);
    }
    if (lane < R) {
#pragma unroll
        for (int k = 0; k < NV; ++k) s_red[(k * kWarps + warp) * R + lane] = w[k];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NV * R; i += kThreads) {
        const int k = i / R, c = i % R;
        double acc = 0.0;
        for (int ww = 0; ww < kWarps; ++ww) acc += s_red[(k * kWarps + ww) * R + c];
        s_in[i] = acc;
    }
    __syncthreads();
}

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// z = Dinv r for one node and column (3x3 complex block times 3-vector).
template <typename C>
__device__ __forceinline__ void apply_dinv(const C* __restrict__ dinv, int node, const C (&r)[3], C (&z)[3]) {
#pragma unroll
    for (int al = 0; al < 3; ++al) {
        C acc = mk(decltype(C{}.x)(0), decltype(C{}.x)(0));
#pragma unroll
        for (int be = 0; be < 3; ++be) {
            const C m = ld_ro(dinv + (size_t)node * 9 + 3 * al + be);
            acc.x += m.x * r[be].x - m.y * r[be].y;
            acc.y += m.x * r[be].y + m.y * r[be].x;
        }
        z[al] = acc;
    }
}

template <typename T, int R>
__global__ void __launch_bounds__(kThreads) k_solve(SolveParams P) {
    using C = typename CplxT<T>::type;
    const C* valT = (const C*)P.valT;
    const C* dinvT = (const C*)P.dinvT;
    C* vd = (C*)P.d;
    C* vr = (C*)P.r;
    C* vz = (C*)P.z;
    C* vp = (C*)P.p;
    C* vq = (C*)P.q;

    __shared__ double s_red[3 * kWarps * R];
    __shared__ double s_in[3 * R], s_out[3 * R];
    __shared__ double s_rn[R], s_bn[R], s_itol[R], s_rel[R];
    __shared__ double s_rho_r[R], s_rho_i[R];
    __shared__ T s_ar[R], s_ai[R], s_br[R], s_bi[R];
    __shared__ int s_active[R], s_pass[R], s_done[R], s_status[R], s_iters[R], s_outer[R], s_pass_it[R];
    __shared__ int s_any;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r0 = (int)((int64_t)blockIdx.x * P.n_rows / P.n_cta);
    const int r1 = (int)((int64_t)(blockIdx.x + 1) * P.n_rows / P.n_cta);
    const int n_items = (r1 - r0) * R;  // (node, column) pairs owned by this CTA
    const int my_c = tid % R;           // column of every item this thread handles

    if (tid < R) {
        s_done[tid] = 0;
        s_status[tid] = FE_OK;
        s_iters[tid] = 0;
        s_outer[tid] = 0;
        s_active[tid] = 0;
        s_pass[tid] = 0;
        s_rel[tid] = 0.0;
    }
    if (!P.use_x0)
        for (int i = tid; i < 3 * n_items; i += kThreads) P.x[(size_t)3 * r0 * R + i] = make_double2(0.0, 0.0);
    __syncthreads();
    if (!grid_reduce<0>(P, s_in, s_out)) goto out;

    for (;;) {
        // ---- FP64 true residual r = b - A x and the norms ||r||, ||b|| ----
        {
            double acc[2] = {0.0, 0.0};
            if (R == 1) {
                for (int row = r0 + warp; row < r1; row += kWarps) {
                    double2 y0, y1, y2;
                    row_product_r1<double2, true>(P.val64, P.col, __ldg(P.rp + row), __ldg(P.rp + row + 1), P.x,
                                                  lane, y0, y1, y2);
                    if (lane < 3) {
                        const double2 y = lane == 0 ? y0 : (lane == 1 ? y1 : y2);
                        const double2 bv = __ldg(P.b + 3 * row + lane);
                        const double2 rv = make_double2(bv.x - y.x, bv.y - y.y);
                        P.r64[3 * row + lane] = rv;
                        acc[0] += rv.x * rv.x + rv.y * rv.y;
                        acc[1] += bv.x * bv.x + bv.y * bv.y;
                    }
                }
            } else {
                constexpr int kRowsPerWarp = 32 / R;
                const int c = lane % R;
                for (int row = r0 + warp * kRowsPerWarp + lane / R; row < r1; row += kWarps * kRowsPerWarp) {
                    double2 y[3];
                    row_product_col<double2, true>(P.val64, P.col, __ldg(P.rp + row), __ldg(P.rp + row + 1), P.x, R,
                                                   c, y[0], y[1], y[2]);
#pragma unroll
                    for (int al = 0; al < 3; ++al) {
                        const size_t o = (size_t)(3 * row + al) * R + c;
                        const double2 bv = __ldg(P.b + o);
                        const double2 rv = make_double2(bv.x - y[al].x, bv.y - y[al].y);
                        P.r64[o] = rv;
                        acc[0] += rv.x * rv.x + rv.y * rv.y;
                        acc[1] += bv.x * bv.x + bv.y * bv.y;
                    }
                }
            }
            cta_colsum<R, 2>(acc, s_red, s_in);
            if (!grid_reduce<2 * R>(P, s_in, s_out)) goto out;
        }
        if (tid < R) {
            const int c = tid;
            const double rn = sqrt(s_out[c]), bn = sqrt(s_out[R + c]);
            s_pass[c] = 0;
            s_active[c] = 0;
            if (!s_done[c]) {
                const double rel = bn > 0.0 ? rn / bn : 0.0;
                s_rel[c] = rel;
                if (!(rel == rel)) {
                    s_done[c] = 1;
                    s_status[c] = FE_ERR_NOT_CONVERGED;
                } else if (rel <= P.tol) {
                    s_done[c] = 1;
                    s_status[c] = FE_OK;
                } else if (s_outer[c] >= P.max_outer || s_iters[c] >= P.max_iter || s_status[c] == FE_ERR_BREAKDOWN) {
                    s_done[c] = 1;
                    if (s_status[c] == FE_OK) s_status[c] = FE_ERR_NOT_CONVERGED;
                } else {
                    s_active[c] = 1;
                    s_pass[c] = 1;
                    s_pass_it[c] = 0;
                    s_rn[c] = rn;
                    s_bn[c] = bn;
                    s_itol[c] = fmax(P.inner_tol, 0.5 * P.tol * bn / rn);
                    s_outer[c] += 1;
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            int any = 0;
            for (int c = 0; c < R; ++c) any |= s_active[c];
            s_any = any;
        }
        __syncthreads();
        if (!s_any) break;

        // ---- inner start: r = RN(r64 / ||r64||), d = 0, z = Dinv r, p = z ----
        {
            double acc[2] = {0.0, 0.0};
            const bool act = s_active[my_c];
            const double sc = act ? 1.0 / s_rn[my_c] : 0.0;
            for (int i = tid; i < n_items; i += kThreads) {
                const int node = r0 + i / R;
                C rv[3], zv[3];
#pragma unroll
                for (int al = 0; al < 3; ++al) {
                    const double2 w = __ldcg(P.r64 + (size_t)(3 * node + al) * R + my_c);
                    rv[al] = mk((T)(w.x * sc), (T)(w.y * sc));
                }
                apply_dinv(dinvT, node, rv, zv);
                T ar = 0, ai = 0;
#pragma unroll
                for (int al = 0; al < 3; ++al) {
                    const size_t o = (size_t)(3 * node + al) * R + my_c;
                    if (!act) zv[al] = mk((T)0, (T)0);
                    vr[o] = rv[al];
                    vz[o] = zv[al];
                    vp[o] = zv[al];
                    vd[o] = mk((T)0, (T)0);
                    ar += rv[al].x * zv[al].x - rv[al].y * zv[al].y;
                    ai += rv[al].x * zv[al].y + rv[al].y * zv[al].x;
                }
                acc[0] += (double)ar;
                acc[1] += (double)ai;
            }
            cta_colsum<R, 2>(acc, s_red, s_in);
            if (!grid_reduce<2 * R>(P, s_in, s_out)) goto out;
            if (tid < R) {
                s_rho_r[tid] = s_out[tid];
                s_rho_i[tid] = s_out[R + tid];
            }
            __syncthreads();
        }

        // ---- inner COCG passes ----
        for (;;) {
            // q = A p and p^T q
            {
                T pr = 0, pi = 0;
                if (R == 1) {
                    for (int row = r0 + warp; row < r1; row += kWarps) {
                        C y0, y1, y2;
                        row_product_r1<C, true>(valT, P.col, __ldg(P.rp + row), __ldg(P.rp + row + 1), vp, lane, y0,
                                                y1, y2);
                        if (lane < 3) {
                            const C y = lane == 0 ? y0 : (lane == 1 ? y1 : y2);
                            vq[3 * row + lane] = y;
                            const C pv = ld_cg(vp + 3 * row + lane);
                            pr += pv.x * y.x - pv.y * y.y;
                            pi += pv.x * y.y + pv.y * y.x;
                        }
                    }
                } else {
                    constexpr int kRowsPerWarp = 32 / R;
                    const int c = lane % R;
                    for (int row = r0 + warp * kRowsPerWarp + lane / R; row < r1; row += kWarps * kRowsPerWarp) {
                        C y[3];
                        row_product_col<C, true>(valT, P.col, __ldg(P.rp + row), __ldg(P.rp + row + 1), vp, R, c,
                                                 y[0], y[1], y[2]);
#pragma unroll
                        for (int al = 0; al < 3; ++al) {
                            const size_t o = (size_t)(3 * row + al) * R + c;
                            vq[o] = y[al];
                            const C pv = ld_cg(vp + o);
                            pr += pv.x * y[al].x - pv.y * y[al].y;
                            pi += pv.x * y[al].y + pv.y * y[al].x;
                        }
                    }
                }
                double acc[2] = {(double)pr, (double)pi};
                cta_colsum<R, 2>(acc, s_red, s_in);
                if (!grid_reduce<2 * R>(P, s_in, s_out)) goto out;
            }
            if (tid < R) {
                const int c = tid;
                if (s_active[c]) {
                    const double mr = s_out[c], mi = s_out[R + c];
                    const double den = mr * mr + mi * mi;
                    if (!(den > 0.0) || !(den < 1e300)) {
                        s_active[c] = 0;
                        if (s_pass_it[c] == 0) s_status[c] = FE_ERR_BREAKDOWN;
                        s_ar[c] = 0;
                        s_ai[c] = 0;
                    } else {
                        // alpha = rho / mu
                        s_ar[c] = (T)((s_rho_r[c] * mr + s_rho_i[c] * mi) / den);
                        s_ai[c] = (T)((s_rho_i[c] * mr - s_rho_r[c] * mi) / den);
                    }
                } else {
                    s_ar[c] = 0;
                    s_ai[c] = 0;
                }
            }
            __syncthreads();
            // d += alpha p, r -= alpha q, z = Dinv r, rho' = r^T z, ||r||^2
            {
                double acc[3] = {0.0, 0.0, 0.0};
                if (s_active[my_c]) {
                    const C alpha = mk(s_ar[my_c], s_ai[my_c]);
                    T rho_r = 0, rho_i = 0, rr = 0;
                    for (int i = tid; i < n_items; i += kThreads) {
                        const int node = r0 + i / R;
                        C rv[3], zv[3];
#pragma unroll
                        for (int al = 0; al < 3; ++al) {
                            const size_t o = (size_t)(3 * node + al) * R + my_c;
                            const C pv = ld_cg(vp + o), qv = ld_cg(vq + o);
                            C dv = ld_cg(vd + o);
                            C rw = ld_cg(vr + o);
                            const C ap = cmul(alpha, pv), aq = cmul(alpha, qv);
                            dv.x += ap.x;
                            dv.y += ap.y;
                            rw.x -= aq.x;
                            rw.y -= aq.y;
                            vd[o] = dv;
                            vr[o] = rw;
                            rv[al] = rw;
                        }
                        apply_dinv(dinvT, node, rv, zv);
#pragma unroll
                        for (int al = 0; al < 3; ++al) {
                            vz[(size_t)(3 * node + al) * R + my_c] = zv[al];
                            rho_r += rv[al].x * zv[al].x - rv[al].y * zv[al].y;
                            rho_i += rv[al].x * zv[al].y + rv[al].y * zv[al].x;
                            rr += rv[al].x * rv[al].x + rv[al].y * rv[al].y;
                        }
                    }
                    acc[0] = rho_r;
                    acc[1] = rho_i;
                    acc[2] = rr;
                }
                cta_colsum<R, 3>(acc, s_red, s_in);
                if (!grid_reduce<3 * R>(P, s_in, s_out)) goto out;
            }
            if (tid < R) {
                const int c = tid;
                if (s_active[c]) {
                    s_iters[c] += 1;
                    s_pass_it[c] += 1;
                    const double nr = sqrt(s_out[2 * R + c]);
                    const double rho_r = s_out[c], rho_i = s_out[R + c];
                    const double den = s_rho_r[c] * s_rho_r[c] + s_rho_i[c] * s_rho_i[c];
                    if (!(nr == nr) || nr <= s_itol[c] || s_iters[c] >= P.max_iter || nr > 1e12) {
                        s_active[c] = 0;
                    } else if (!(den > 0.0) || (rho_r == 0.0 && rho_i == 0.0)) {
                        s_active[c] = 0;
                    } else {
                        // beta = rho' / rho
                        s_br[c] = (T)((rho_r * s_rho_r[c] + rho_i * s_rho_i[c]) / den);
                        s_bi[c] = (T)((rho_i * s_rho_r[c] - rho_r * s_rho_i[c]) / den);
                        s_rho_r[c] = rho_r;
                        s_rho_i[c] = rho_i;
                    }
                }
            }
            __syncthreads();
            if (tid == 0) {
                int any = 0;
                for (int c = 0; c < R; ++c) any |= s_active[c];
                s_any = any;
            }
            __syncthreads();
            if (!s_any) break;
            // p = z + beta p
            if (s_active[my_c]) {
                const C beta = mk(s_br[my_c], s_bi[my_c]);
                for (int i = tid; i < n_items; i += kThreads) {
                    const int node = r0 + i / R;
#pragma unroll
                    for (int al = 0; al < 3; ++al) {
                        const size_t o = (size_t)(3 * node + al) * R + my_c;
                        const C pv = ld_cg(vp + o), zv = ld_cg(vz + o);
                        const C bp = cmul(beta, pv);
                        vp[o] = mk(zv.x + bp.x, zv.y + bp.y);
                    }
                }
            }
            if (!grid_reduce<0>(P, s_in, s_out)) goto out;
        }

        // ---- FP64 solution update x += ||r|| d ----
        if (s_pass[my_c]) {
            const double sc = s_rn[my_c];
            for (int i = tid; i < n_items; i += kThreads) {
                const int node = r0 + i / R;
#pragma unroll
                for (int al = 0; al < 3; ++al) {
                    const size_t o = (size_t)(3 * node + al) * R + my_c;
                    const C dv = ld_cg(vd + o);
                    double2 xv = P.x[o];
                    xv.x += sc * (double)dv.x;
                    xv.y += sc * (double)dv.y;
                    P.x[o] = xv;
                }
            }
        }
        if (!grid_reduce<0>(P, s_in, s_out)) goto out;
    }
out:
    if (blockIdx.x == 0 && tid < R) {
        P.rep_status[tid] = s_status[tid];
        P.rep_iters[tid] = s_iters[tid];
        P.rep_outer[tid] = s_outer[tid];
        P.rep_rel[tid] = s_rel[tid];
    }
}

// ---------------------------------------------------------------------------
// Standalone products for fe_spmv: y = A x.
// ---------------------------------------------------------------------------
template <typename C>
__global__ void __launch_bounds__(256) k_spmv_r1(const C* __restrict__ val, const int* __restrict__ col,
                                                 const int* __restrict__ rp, const C* __restrict__ x, C* __restrict__ y,
                                                 int n_rows) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n_rows; row += nw) {
        C y0, y1, y2;
        row_product_r1<C, false>(val, col, __ldg(rp + row), __ldg(rp + row + 1), x, lane, y0, y1, y2);
        if (lane < 3) y[3 * row + lane] = lane == 0 ? y0 : (lane == 1 ? y1 : y2);
    }
}

template <typename C>
__global__ void __launch_bounds__(256) k_spmv_cols(const C* __restrict__ val, const int* __restrict__ col,
                                                   const int* __restrict__ rp, const C* __restrict__ x,
                                                   C* __restrict__ y, int n_rows, int nrhs) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_rows * nrhs) return;
    const int row = (int)(t / nrhs), c = (int)(t - (int64_t)row * nrhs);
    C v[3];
    row_product_col<C, false>(val, col, __ldg(rp + row), __ldg(rp + row + 1), x, nrhs, c, v[0], v[1], v[2]);
#pragma unroll
    for (int al = 0; al < 3; ++al) y[(size_t)(3 * row + al) * nrhs + c] = v[al];
}

// Column gather / scatter between [n_dof][nrhs] and a [n_dof][R] tile.
__global__ void k_gather_cols(const double2* __restrict__ src, int lds, int c0, int ncols, double2* __restrict__ dst,
                              int R, int64_t n_dof) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_dof * R) return;
    const int64_t dof = t / R;
    const int c = (int)(t - dof * R);
    dst[t] = c < ncols ? src[dof * lds + c0 + c] : make_double2(0.0, 0.0);
}

__global__ void k_scatter_cols(const double2* __restrict__ src, int R, int ncols, double2* __restrict__ dst, int ldd,
                               int c0, int64_t n_dof) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_dof * ncols) return;
    const int64_t dof = t / ncols;
    const int c = (int)(t - dof * ncols);
    dst[dof * ldd + c0 + c] = src[dof * R + c];
}

fe_status build_rhs(fe_ctx* ctx, const fe_system* s, int nrhs, const fe_planewave* waves, double2* d_B,
                    DevBuf& wave_buf);

struct Workspace {
    DevBuf b, x, r64, d, r, z, p, q, partial, result, sync, rep;
};

template <typename T, int R>
static fe_status launch_solve(fe_ctx* ctx, SolveParams& P) {
    int per_sm = 0;
    FE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve<T, R>, kThreads, 0));
    if (per_sm < 1) {
        set_error("solve kernel does not fit on an SM");
        return FE_ERR_CUDA;
    }
    per_sm = std::min(per_sm, 2);
    P.n_cta = std::min(per_sm * ctx->num_sms, std::max(1, P.n_rows));
    void* args[] = {&P};
    FE_CUDA(cudaEventRecord(ctx->ev0, ctx->stream));
    FE_CUDA(cudaLaunchCooperativeKernel((void*)k_solve<T, R>, dim3(P.n_cta), dim3(kThreads), args, 0, ctx->stream));
    FE_CUDA(cudaEventRecord(ctx->ev1, ctx->stream));
    count_launches(1);
    ctx->last_solve.launches += 1;
    ctx->last_solve.tile_width = R;
    ctx->last_solve.grid_ctas = P.n_cta;
    return FE_OK;
}

template <typename T>
static fe_status dispatch(fe_ctx* ctx, int R, SolveParams& P) {
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

static int pick_tile(int nrhs, int requested) {
    int want = requested > 0 ? requested : std::min(nrhs, 32);
    int R = 1;
    while (R < want && R < 32) R <<= 1;
    return R;
}

// Solves tile by tile; b and x are device arrays [n_dof][nrhs].
static fe_status solve_device(fe_ctx* ctx, const fe_system* s, int nrhs, const double2* d_b, double2* d_x,
                              bool use_x0, const fe_solve_opts& o, fe_solve_report* rep) {
    const fe_mesh* m = s->mesh;
    cudaStream_t st = ctx->stream;
    const int64_t n_dof = 3 * (int64_t)m->n_act;
    const int R = pick_tile(nrhs, o.rhs_tile);
    const bool fp64 = o.precision == FE_PREC_FP64;
    if (!fp64 && !s->val32.ptr) {
        set_error("mixed-precision solve of a system assembled in FP64 only");
        return FE_ERR_INVALID_ARG;
    }
    const size_t esz = fp64 ? sizeof(double2) : sizeof(float2);
    Workspace w;
    auto cleanup = [&]() {
        for (DevBuf* b : {&w.b, &w.x, &w.r64, &w.d, &w.r, &w.z, &w.p, &w.q, &w.partial, &w.result, &w.sync, &w.rep})
            dev_free(st, *b);
    };
    fe_status e = FE_OK;
    const size_t nv = (size_t)n_dof * R;
    const int max_cta = 2 * ctx->num_sms;
    for (auto pr : {std::make_pair(&w.b, nv * sizeof(double2)), std::make_pair(&w.x, nv * sizeof(double2)),
                    std::make_pair(&w.r64, nv * sizeof(double2)), std::make_pair(&w.d, nv * esz),
                    std::make_pair(&w.r, nv * esz), std::make_pair(&w.z, nv * esz), std::make_pair(&w.p, nv * esz),
                    std::make_pair(&w.q, nv * esz),
                    std::make_pair(&w.partial, (size_t)max_cta * 3 * R * sizeof(double)),
                    std::make_pair(&w.result, (size_t)3 * R * sizeof(double)),
                    std::make_pair(&w.sync, sizeof(SyncState)),
                    std::make_pair(&w.rep, (size_t)R * (3 * sizeof(int) + sizeof(double)) + 64)}) {
        if ((e = dev_alloc(st, *pr.first, pr.second)) != FE_OK) {
            cleanup();
            return e;
        }
    }
    std::vector<int> h_rep_i(3 * R);
    std::vector<double> h_rep_d(R);
    fe_status worst = FE_OK;
    ctx->last_solve = fe_solve_stats{};
    for (int c0 = 0; c0 < nrhs; c0 += R) {
        const int nc = std::min(R, nrhs - c0);
        const unsigned gb = (unsigned)((n_dof * R + 255) / 256);
        k_gather_cols<<<gb, 256, 0, st>>>(d_b, nrhs, c0, nc, (double2*)w.b.ptr, R, n_dof);
        count_launches(1);
        if (use_x0) {
            k_gather_cols<<<gb, 256, 0, st>>>(d_x, nrhs, c0, nc, (double2*)w.x.ptr, R, n_dof);
            count_launches(1);
        }
        cudaMemsetAsync(w.sync.ptr, 0, sizeof(SyncState), st);
        SolveParams P{};
        P.n_rows = m->n_act;
        P.rp = (const int*)m->row_ptr.ptr;
        P.col = (const int*)m->col_idx.ptr;
        P.val64 = (const double2*)s->val64.ptr;
        P.valT = fp64 ? s->val64.ptr : s->val32.ptr;
        P.dinvT = fp64 ? s->dinv64.ptr : s->dinv32.ptr;
        P.b = (const double2*)w.b.ptr;
        P.x = (double2*)w.x.ptr;
        P.r64 = (double2*)w.r64.ptr;
        P.d = w.d.ptr;
        P.r = w.r.ptr;
        P.z = w.z.ptr;
        P.p = w.p.ptr;
        P.q = w.q.ptr;
        P.sync = (SyncState*)w.sync.ptr;
        P.partial = (double*)w.partial.ptr;
        P.result = (double*)w.result.ptr;
        P.tol = o.tol;
        P.inner_tol = fp64 ? 0.0 : o.inner_tol;
        P.max_iter = o.max_iter;
        P.max_outer = o.max_outer;
        P.use_x0 = use_x0 ? 1 : 0;
        int* ri = (int*)w.rep.ptr;
        P.rep_status = ri;
        P.rep_iters = ri + R;
        P.rep_outer = ri + 2 * R;
        P.rep_rel = (double*)((char*)w.rep.ptr + ((3 * R * sizeof(int) + 15) / 16) * 16);
        P.timeout_ns = 4000000000ull;
        e = fp64 ? dispatch<double>(ctx, R, P) : dispatch<float>(ctx, R, P);
        if (e != FE_OK) break;
        const unsigned gs = (unsigned)((n_dof * nc + 255) / 256);
        k_scatter_cols<<<gs, 256, 0, st>>>((const double2*)w.x.ptr, R, nc, d_x, nrhs, c0, n_dof);
        count_launches(1);
        SyncState hs{};
        cudaMemcpyAsync(&hs, w.sync.ptr, sizeof(SyncState), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(h_rep_i.data(), ri, 3 * R * sizeof(int), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(h_rep_d.data(), P.rep_rel, R * sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaError_t ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) {
            set_error("solve: %s", cudaGetErrorString(ce));
            e = FE_ERR_CUDA;
            break;
        }
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1) == cudaSuccess) ctx->last_solve.kernel_ms += ms;
        if (hs.err) {
            set_error("solve: a grid barrier wait expired (device status %d)", hs.err);
            e = FE_ERR_TIMEOUT;
            break;
        }
        for (int c = 0; c < nc; ++c) {
            const int st_c = h_rep_i[c];
            if (rep) {
                rep[c0 + c].status = st_c;
                rep[c0 + c].iterations = h_rep_i[R + c];
                rep[c0 + c].outer = h_rep_i[2 * R + c];
                rep[c0 + c].reserved = 0;
                rep[c0 + c].rel_residual = h_rep_d[c];
            }
            if (st_c != FE_OK && worst == FE_OK) worst = (fe_status)st_c;
            ctx->last_solve.inner_iters += h_rep_i[R + c];
            ctx->last_solve.passes = std::max<int64_t>(ctx->last_solve.passes, h_rep_i[2 * R + c] + 1);
        }
    }
    cleanup();
    if (e != FE_OK) return e;
    if (worst != FE_OK) set_error("solve: at least one right-hand side did not reach the tolerance");
    return worst;
}

static fe_status check_opts(const fe_solve_opts* o, fe_solve_opts& out) {
    fe_solve_opts_default(&out);
    if (o) out = *o;
    if (out.precision != FE_PREC_FP64 && out.precision != FE_PREC_MIXED) {
        set_error("solve: precision must be FP64 or MIXED");
        return FE_ERR_INVALID_ARG;
    }
    if (!(out.tol > 0.0) || out.max_iter < 1 || out.max_outer < 1 || out.inner_tol < 0.0 || out.rhs_tile < 0) {
        set_error("solve: bad tolerance or iteration limits");
        return FE_ERR_INVALID_ARG;
    }
    return FE_OK;
}

}  // namespace fe

using namespace fe;

extern "C" {

void fe_solve_opts_default(fe_solve_opts* o) {
    if (!o) return;
    o->precision = FE_PREC_MIXED;
    o->tol = 1e-8;
    o->inner_tol = 1e-4;
    o->max_iter = 20000;
    o->max_outer = 30;
    o->rhs_tile = 0;
}

fe_status fe_spmv(fe_ctx* ctx, const fe_system* s, int32_t precision, int32_t nrhs, const void* x, void* y) {
    if (!ctx || !s || !x || !y || nrhs < 1) {
        set_error("fe_spmv: NULL argument or nrhs < 1");
        return FE_ERR_INVALID_ARG;
    }
    const fe_mesh* m = s->mesh;
    cudaStream_t st = ctx->stream;
    const int* rp = (const int*)m->row_ptr.ptr;
    const int* col = (const int*)m->col_idx.ptr;
    if (precision == FE_PREC_FP64) {
        if (nrhs == 1) {
            k_spmv_r1<double2><<<ctx->num_sms * 8, 256, 0, st>>>((const double2*)s->val64.ptr, col, rp,
                                                                  (const double2*)x, (double2*)y, m->n_act);
        } else {
            const int64_t n = (int64_t)m->n_act * nrhs;
            k_spmv_cols<double2><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                (const double2*)s->val64.ptr, col, rp, (const double2*)x, (double2*)y, m->n_act, nrhs);
        }
    } else if (precision == FE_PREC_MIXED) {
        if (!s->val32.ptr) {
            set_error("fe_spmv: no complex64 copy (system assembled in FP64)");
            return FE_ERR_INVALID_ARG;
        }
        if (nrhs == 1) {
            k_spmv_r1<float2><<<ctx->num_sms * 8, 256, 0, st>>>((const float2*)s->val32.ptr, col, rp,
                                                                 (const float2*)x, (float2*)y, m->n_act);
        } else {
            const int64_t n = (int64_t)m->n_act * nrhs;
            k_spmv_cols<float2><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                (const float2*)s->val32.ptr, col, rp, (const float2*)x, (float2*)y, m->n_act, nrhs);
        }
    } else {
        set_error("fe_spmv: bad precision");
        return FE_ERR_INVALID_ARG;
    }
    FE_LAUNCHED();
    return FE_OK;
}

fe_status fe_solve_rhs(fe_ctx* ctx, const fe_system* s, int32_t nrhs, const void* b, int32_t b_on_device,
                       const fe_solve_opts* o, void* x_out, int32_t x_on_device, int32_t use_x0,
                       fe_solve_report* rep) {
    if (!ctx || !s || !b || !x_out || nrhs < 1) {
        set_error("fe_solve_rhs: NULL argument or nrhs < 1");
        return FE_ERR_INVALID_ARG;
    }
    fe_solve_opts opt;
    FE_TRY(check_opts(o, opt));
    cudaSetDevice(ctx->device);
    cudaStream_t st = ctx->stream;
    const size_t bytes = (size_t)3 * s->mesh->n_act * nrhs * sizeof(double2);
    DevBuf hb, hx;
    const double2* db = (const double2*)b;
    double2* dx = (double2*)x_out;
    fe_status e = FE_OK;
    if (!b_on_device) {
        if ((e = dev_alloc(st, hb, bytes)) != FE_OK) return e;
        cudaMemcpyAsync(hb.ptr, b, bytes, cudaMemcpyHostToDevice, st);
        db = (const double2*)hb.ptr;
    }
    if (!x_on_device) {
        if ((e = dev_alloc(st, hx, bytes)) != FE_OK) {
            dev_free(st, hb);
            return e;
        }
        if (use_x0) cudaMemcpyAsync(hx.ptr, x_out, bytes, cudaMemcpyHostToDevice, st);
        dx = (double2*)hx.ptr;
    }
    e = solve_device(ctx, s, nrhs, db, dx, use_x0 != 0, opt, rep);
    if (!x_on_device && (e == FE_OK || e == FE_ERR_NOT_CONVERGED || e == FE_ERR_BREAKDOWN)) {
        cudaMemcpyAsync(x_out, dx, bytes, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
    }
    dev_free(st, hb);
    dev_free(st, hx);
    return e;
}

fe_status fe_solve_batch(fe_ctx* ctx, const fe_system* s, int32_t nrhs, const fe_planewave* waves,
                         const fe_solve_opts* o, void* x_out, int32_t x_on_device, fe_solve_report* rep) {
    if (!ctx || !s || !waves || !x_out || nrhs < 1) {
        set_error("fe_solve_batch: NULL argument or nrhs < 1");
        return FE_ERR_INVALID_ARG;
    }
    fe_solve_opts opt;
    FE_TRY(check_opts(o, opt));
    cudaSetDevice(ctx->device);
    cudaStream_t st = ctx->stream;
    const size_t bytes = (size_t)3 * s->mesh->n_act * nrhs * sizeof(double2);
    DevBuf bb, wb, hx;
    fe_status e = dev_alloc(st, bb, bytes);
    if (e == FE_OK) e = build_rhs(ctx, s, nrhs, waves, (double2*)bb.ptr, wb);
    double2* dx = (double2*)x_out;
    if (e == FE_OK && !x_on_device) {
        e = dev_alloc(st, hx, bytes);
        dx = (double2*)hx.ptr;
    }
    if (e == FE_OK) e = solve_device(ctx, s, nrhs, (const double2*)bb.ptr, dx, false, opt, rep);
    if (!x_on_device && hx.ptr && (e == FE_OK || e == FE_ERR_NOT_CONVERGED || e == FE_ERR_BREAKDOWN)) {
        cudaMemcpyAsync(x_out, dx, bytes, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
    }
    dev_free(st, bb);
    dev_free(st, wb);
    dev_free(st, hx);
    return e;
}

}  // extern "C"
