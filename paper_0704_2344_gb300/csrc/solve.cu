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
#include <cstddef>
#include <cstdlib>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include "solve_kernels.cuh"

namespace fe {

// The kernels are instantiated in solve_fp64.cu, solve_mixed.cu and solve_df.cu.
extern template fe_status dispatch<double>(fe_ctx*, int, SolveParams&);
extern template fe_status dispatch<float>(fe_ctx*, int, SolveParams&);
extern template fe_status dispatch<DFloat>(fe_ctx*, int, SolveParams&);
extern template fe_status launch_jobs_w<double>(fe_ctx*, int, SolveJob* const*, const int*, int, cudaStream_t, const int*);
extern template fe_status launch_jobs_w<float>(fe_ctx*, int, SolveJob* const*, const int*, int, cudaStream_t, const int*);
extern template fe_status launch_jobs_w<DFloat>(fe_ctx*, int, SolveJob* const*, const int*, int, cudaStream_t, const int*);

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

static int pick_tile(int nrhs, int requested) {
    int want = requested > 0 ? requested : std::min(nrhs, 32);
    int R = 1;
    while (R < want && R < 32) R <<= 1;
    return R;
}

static void free_workspace(cudaStream_t st, Workspace& w) {
    for (DevBuf* b : {&w.b, &w.x, &w.r, &w.u, &w.p, &w.s, &w.uM, &w.pM, &w.w, &w.partial, &w.result, &w.sync, &w.rep,
                      &w.trace, &w.pk, &w.state})
        dev_free(st, *b);
}

// Krylov workspace of one tile of R columns for up to max_cta CTAs.
// Bytes of one inner-precision vector entry (uM, pM, w): complex128,
// complex64 or a complex FP32 pair.
static size_t inner_bytes(int prec) { return prec == FE_PREC_MIXED ? sizeof(float2) : sizeof(double2); }

// Whether the products read separate inner-precision copies of u and p
// (complex64; FP32 pairs with one column) instead of the vectors themselves.
static bool split_copies(int prec, int R) {
    (void)R;
    return prec == FE_PREC_MIXED;
}

// Inner-precision matrix planes of a system, or NULL when it was not
// assembled for that precision.
static const void* inner_matrix(const fe_system* s, int prec) {
    return prec == FE_PREC_FP64 ? s->val64.ptr : (prec == FE_PREC_MIXED ? s->val32.ptr : s->valdf.ptr);
}

static fe_status check_precond(const fe_ctx* ctx, const fe_system* s, const fe_solve_opts& o, const char* what);

static fe_status check_system_precision(const fe_system* s, int prec, const char* who) {
    if (!inner_matrix(s, prec)) {
        set_error("%s: the system was not assembled for precision %d (assemble with that precision)", who, prec);
        return FE_ERR_INVALID_ARG;
    }
    if (s->variant == FE_VARIANT_L) {
        // the literal Eq. 4 matrix is not symmetric: COCG does not apply to it
        set_error("%s: variant L (the literal, non-symmetric form of Eq. 4) has no symmetric solve; use S or P", who);
        return FE_ERR_INVALID_ARG;
    }
    return FE_OK;
}

template <typename F>
static fe_status with_inner_type(int prec, F&& f) {
    switch (prec) {
        case FE_PREC_FP64: return f((double*)nullptr);
        case FE_PREC_MIXED: return f((float*)nullptr);
        case FE_PREC_DF: return f((DFloat*)nullptr);
        default: set_error("unknown precision %d", prec); return FE_ERR_INVALID_ARG;
    }
}

// Entries of the packed explicit rows a single-column complex64 or
// FP32-pair launch copies its explicit rows into (0: none).
// A system's block dictionary serves single-column solves when it holds at
// most kDictSmemMax bytes (it is copied into every CTA's shared memory).
constexpr size_t kDictSmemMax = 64 * 1024;
static bool dict_usable(const fe_system* s, int prec, int R) {
    return R == 1 && prec != FE_PREC_FP64 && s->n_dict > 0 &&
           (size_t)s->n_dict * 9 * inner_bytes(prec) <= kDictSmemMax;
}

static int64_t packed_entries(const fe_system* s, int prec, int R) {
    if (R != 1 || prec == FE_PREC_FP64 || !s->expl_prefix.ptr || dict_usable(s, prec, R)) return 0;
    return 9 * s->blocks_explicit;
}

static fe_status alloc_workspace(cudaStream_t st, int64_t n_dof, int R, int prec, int max_cta, Workspace& w,
                                 int64_t pk_entries = 0) {
    const size_t esz = inner_bytes(prec);  // inner-precision vectors (uM, w)
    const size_t nv = (size_t)n_dof * R;
    for (auto pr : {std::make_pair(&w.b, nv * sizeof(double2)), std::make_pair(&w.x, nv * sizeof(double2)),
                    std::make_pair(&w.r, nv * sizeof(double2)), std::make_pair(&w.u, nv * sizeof(double2)),
                    std::make_pair(&w.p, nv * sizeof(double2)), std::make_pair(&w.s, nv * sizeof(double2)),
                    std::make_pair(&w.uM, split_copies(prec, R) ? nv * esz : (size_t)16),
                    std::make_pair(&w.pM, split_copies(prec, R) ? nv * esz : (size_t)16), std::make_pair(&w.w, nv * esz),
                    std::make_pair(&w.partial, (size_t)max_cta * kMaxNV * R * sizeof(double)),
                    std::make_pair(&w.result, (size_t)kMaxNV * R * sizeof(double)),
                    std::make_pair(&w.sync, sync_bytes(max_cta)),
                    std::make_pair(&w.rep, (size_t)R * (3 * sizeof(int) + sizeof(double)) + 64)}) {
        const fe_status e = dev_alloc(st, *pr.first, pr.second);
        if (e != FE_OK) {
            free_workspace(st, w);
            return e;
        }
    }
    if (pk_entries > 0) {
        const fe_status e = dev_alloc(st, w.pk, (size_t)pk_entries * inner_bytes(prec));
        if (e != FE_OK) {
            free_workspace(st, w);
            return e;
        }
    }
    return FE_OK;
}

// Bytes alloc_workspace takes (before allocator rounding).
size_t workspace_bytes(int64_t n_dof, int R, int prec, int max_cta, int64_t pk_entries) {
    const size_t nv = (size_t)n_dof * R;
    const size_t esz = inner_bytes(prec);
    return nv * (6 * sizeof(double2) + (split_copies(prec, R) ? 3 : 1) * esz) + (size_t)(max_cta + 1) * kMaxNV * R * sizeof(double) +
           (size_t)R * 32 + 4096 + (size_t)pk_entries * esz;
}

// Solve parameters for a tile of R columns held in workspace w (n_cta and the
// shared-memory layout are set at launch).
static void fill_params(SolveParams& P, const fe_system* s, const Workspace& w, int R, int prec,
                        const fe_solve_opts& o, bool use_x0) {
    const fe_mesh* m = s->mesh;
    const bool fp64 = prec == FE_PREC_FP64;
    const bool df = prec == FE_PREC_DF;
    P = SolveParams{};
    P.n_rows = m->n_act;
    P.rp = (const int*)m->row_ptr.ptr;
    P.col = (const int*)m->col_idx.ptr;
    P.val64 = (const double2*)s->val64.ptr;
    P.valM = inner_matrix(s, prec);
    P.stride = s->stride;
    P.dinv64 = (const double2*)s->dinv64.ptr;
    P.dinvdf = (const float4*)s->dinvdf.ptr;
    // class stencils and cost-balanced product ranges pay off for the
    // complex64 and FP32-pair products; the FP64 products stay explicit and
    // uniform
    const bool classes = !fp64;
    P.row_class = classes ? (const signed char*)s->row_class.ptr : nullptr;
    P.stencil = (const StencilSet*)s->stencil.ptr;
    P.cost_prefix = classes ? (const int*)(df ? s->cost_prefix_alu.ptr : s->cost_prefix.ptr) : nullptr;
    P.cost_total = classes ? (df ? s->cost_total_alu : s->cost_total) : (int64_t)m->n_act;
    P.cost_min = classes ? s->cost_min[df ? 1 : 0] : 1;
    P.cost_max = classes ? s->cost_max[df ? 1 : 0] : 1;
    P.b = (const double2*)w.b.ptr;
    P.x = (double2*)w.x.ptr;
    P.r = (double2*)w.r.ptr;
    P.u = (double2*)w.u.ptr;
    P.p = (double2*)w.p.ptr;
    P.s = (double2*)w.s.ptr;
    // FP64 vectors, and the FP32-pair vectors of FE_PREC_DF, feed the
    // products directly
    const bool direct = fp64 || df;
    P.uM = direct ? w.u.ptr : w.uM.ptr;
    P.pM = direct ? w.p.ptr : w.pM.ptr;
    P.w = w.w.ptr;
    P.trace = (unsigned long long*)w.trace.ptr;
    P.pk = classes ? w.pk.ptr : nullptr;
    P.expl_prefix = classes ? (const int*)s->expl_prefix.ptr : nullptr;
    if (classes && dict_usable(s, prec, R)) {
        P.dict_idx = (const uint16_t*)s->dict_idx.ptr;
        P.dictM = s->dict_vals.ptr;
        P.n_dict = s->n_dict;
    }
    // lexicographic node ranks: a neighbour is at most one plane, one line
    // and one node away
    P.halo = (m->nx + 1) * (m->ny + 1) + (m->nx + 1) + 1;
    P.res_tmid = (m->nx + 1) + 1;  // same-plane neighbours: one line and one node away
    P.sync = (SyncState*)w.sync.ptr;
    P.partial = (double*)w.partial.ptr;
    P.result = (double*)w.result.ptr;
    P.tol = o.tol;
    // complex64 passes restart at each refinement; FP64 and FP32-pair
    // products are accurate enough to keep the directions across refreshes
    P.reliable = prec == FE_PREC_MIXED ? o.reliable : 0.0;
    P.restart = prec == FE_PREC_MIXED ? 1 : 0;
    P.max_pass = o.max_pass_iter;
    P.max_iter = o.max_iter;
    P.max_outer = o.max_outer;
    P.use_x0 = use_x0 ? 1 : 0;
    int* ri = (int*)w.rep.ptr;
    P.rep_status = ri;
    P.rep_iters = ri + R;
    P.rep_outer = ri + 2 * R;
    P.rep_rel = (double*)((char*)w.rep.ptr + ((3 * R * sizeof(int) + 15) / 16) * 16);
    P.timeout_ns = 1000ull * (unsigned long long)(o.wait_timeout_us > 0 ? o.wait_timeout_us : 4000000);
    P.spin_ns = 0;  // barrier waits poll without back-off (measured fastest)
    // the expanded recurrence takes u^T s in the block-Jacobi update; solves
    // with the block incomplete Cholesky factor keep the recurrence
    P.expand = o.recurrence == FE_RECURRENCE_EXPANDED && !(o.preconditioner == FE_PRECOND_BICP && fp64) ? 1 : 0;
    if (o.preconditioner == FE_PRECOND_BICP && fp64) {
        P.bicp_l = (const double2*)s->bicp_l.ptr;
        P.bicp_linv = (const double2*)s->bicp_linv.ptr;
        P.bicp_tpos = (const int*)s->bicp_tpos.ptr;
        P.bicp_tab = (const int4*)s->bicp_tab.ptr;
        P.bicp_lev = (const int*)s->bicp_lev.ptr;
        P.bicp_nlev = (const int*)s->bicp_nlev.ptr;
    }
}

// Solves the first nrhs columns of b (leading dimension ldb) into x (same
// leading dimension), R columns per launch.
static fe_status solve_tiles(fe_ctx* ctx, const fe_system* s, int nrhs, int ldb, const double2* d_b, double2* d_x,
                             bool use_x0, const fe_solve_opts& o, fe_solve_report* rep, int R, int n_cta_req);

// ---------------------------------------------------------------------------
// Autotuner of the tile width and the grid of multi-column solves.  A trial
// is a real solve of the first columns capped at kTuneIters iterations; its
// measure is device time per column and iteration.  Choices are cached per
// system shape for the life of the process.
// ---------------------------------------------------------------------------
constexpr int kTuneIters = 32;

struct TuneKey {
    int64_t n_dof, nnzb;
    int nrhs, prec, variant, device;
    bool operator<(const TuneKey& o) const {
        return std::tie(n_dof, nnzb, nrhs, prec, variant, device) <
               std::tie(o.n_dof, o.nnzb, o.nrhs, o.prec, o.variant, o.device);
    }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, std::pair<int, int>> g_tune;  // (tile width, CTAs)

static fe_status autotune(fe_ctx* ctx, const fe_system* s, int nrhs, const double2* d_b, const fe_solve_opts& o,
                          int* R_out, int* cta_out, int* how, double* tune_ms) {
    const TuneKey key{3 * (int64_t)s->mesh->n_act, s->mesh->nnzb, std::min(nrhs, 32), o.precision, s->variant,
                      ctx->device};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            *R_out = it->second.first;
            *cta_out = it->second.second;
            *how = 2;
            return FE_OK;
        }
    }
    const int64_t n_dof = key.n_dof;
    const int top = pick_tile(nrhs, 0);
    DevBuf xt;
    FE_TRY(dev_alloc(ctx->stream, xt, (size_t)n_dof * nrhs * sizeof(double2)));
    fe_solve_opts t = o;
    t.max_iter = kTuneIters;
    t.tol = 1e-300;  // trials never converge early
    double best = 1e300;
    int bestR = top, bestC = ctx->num_sms;
    fe_status e = FE_OK;
    const int grids[2] = {ctx->num_sms, std::max(1, ctx->num_sms * 3 / 4)};
    for (int W = 8; W <= top && e == FE_OK; W *= 2)
        for (int g = 0; g < 2 && e == FE_OK; ++g) {
            const fe_status es = solve_tiles(ctx, s, std::min(nrhs, W), nrhs, d_b, (double2*)xt.ptr, false, t, nullptr,
                                             W, grids[g]);
            if (es != FE_OK && es != FE_ERR_NOT_CONVERGED && es != FE_ERR_BREAKDOWN) {
                e = es;
                break;
            }
            const fe_solve_stats& st = ctx->last_solve;
            *tune_ms += st.kernel_ms;
            // real columns only: the zero columns of a padded tile are done at once
            const double per = st.inner_iters > 0 ? st.kernel_ms / (double)st.inner_iters : 1e300;
            if (per < best) {
                best = per;
                bestR = W;
                bestC = grids[g];
            }
        }
    dev_free(ctx->stream, xt);
    if (e != FE_OK) return e;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = {bestR, bestC};
    }
    *R_out = bestR;
    *cta_out = bestC;
    *how = 1;
    return FE_OK;
}

// Solves tile by tile; b and x are device arrays [n_dof][nrhs].
static fe_status solve_device(fe_ctx* ctx, const fe_system* s, int nrhs, const double2* d_b, double2* d_x,
                              bool use_x0, const fe_solve_opts& o, fe_solve_report* rep) {
    FE_TRY(check_system_precision(s, o.precision, "solve"));
    FE_TRY(check_precond(ctx, s, o, "solve"));
    int R = pick_tile(nrhs, o.rhs_tile), n_cta = 0, how = 0;
    double tune_ms = 0.0;
    if (o.rhs_tile == 0 && nrhs >= 8 && o.preconditioner == FE_PRECOND_BLOCK_JACOBI)
        FE_TRY(autotune(ctx, s, nrhs, d_b, o, &R, &n_cta, &how, &tune_ms));
    const fe_status e = solve_tiles(ctx, s, nrhs, nrhs, d_b, d_x, use_x0, o, rep, R, n_cta);
    ctx->last_solve.tuned = how;
    ctx->last_solve.tune_ms = tune_ms;
    return e;
}

static fe_status solve_tiles(fe_ctx* ctx, const fe_system* s, int nrhs, int ldb, const double2* d_b, double2* d_x,
                             bool use_x0, const fe_solve_opts& o, fe_solve_report* rep, int R, int n_cta_req) {
    const fe_mesh* m = s->mesh;
    cudaStream_t st = ctx->stream;
    const int64_t n_dof = 3 * (int64_t)m->n_act;
    const int prec = o.precision;
    Workspace w;
    auto cleanup = [&]() { free_workspace(st, w); };
    fe_status e = alloc_workspace(st, n_dof, R, prec, 2 * ctx->num_sms, w, packed_entries(s, prec, R));
    if (e != FE_OK) return e;
    const bool tracing = getenv("FE_TRACE") && getenv("FE_TRACE")[0] == '1';
    const size_t trace_bytes =
        (size_t)ctx->num_sms * (kTraceIters * kTracePhases + kTraceStats) * sizeof(unsigned long long);
    if (tracing && (e = dev_alloc(st, w.trace, trace_bytes)) != FE_OK) {
        cleanup();
        return e;
    }
    if (tracing) cudaMemsetAsync(w.trace.ptr, 0, trace_bytes, st);
    std::vector<int> h_rep_i(3 * R);
    std::vector<double> h_rep_d(R);
    fe_status worst = FE_OK;
    ctx->last_solve = fe_solve_stats{};
    for (int c0 = 0; c0 < nrhs; c0 += R) {
        const int nc = std::min(R, nrhs - c0);
        const unsigned gb = (unsigned)((n_dof * R + 255) / 256);
        k_gather_cols<<<gb, 256, 0, st>>>(d_b, ldb, c0, nc, (double2*)w.b.ptr, R, n_dof);
        count_launches(1);
        if (use_x0) {
            k_gather_cols<<<gb, 256, 0, st>>>(d_x, ldb, c0, nc, (double2*)w.x.ptr, R, n_dof);
            count_launches(1);
        }
        cudaMemsetAsync(w.sync.ptr, 0, sync_bytes(ctx->num_sms), st);
        SolveParams P;
        fill_params(P, s, w, R, prec, o, use_x0);
        P.n_cta_req = n_cta_req;
        int* ri = P.rep_status;
        e = with_inner_type(prec, [&](auto* tag) { return dispatch<std::remove_pointer_t<decltype(tag)>>(ctx, R, P); });
        if (e != FE_OK) break;
        const unsigned gs = (unsigned)((n_dof * nc + 255) / 256);
        k_scatter_cols<<<gs, 256, 0, st>>>((const double2*)w.x.ptr, R, nc, d_x, ldb, c0, n_dof);
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
        if (tracing) {
            // per-phase durations (ns) of CTA 0 and the slowest CTA, averaged over traced iterations
            std::vector<unsigned long long> tr(trace_bytes / sizeof(unsigned long long));
            cudaMemcpy(tr.data(), w.trace.ptr, trace_bytes, cudaMemcpyDeviceToHost);
            double sum[kTracePhases] = {0};
            int n_it = 0;
            const size_t mid = (size_t)(P.n_cta / 2) * kTraceIters * kTracePhases;
            for (int it = 1; it + 1 < kTraceIters; ++it) {
                const unsigned long long* a = &tr[mid + (size_t)it * kTracePhases];
                const unsigned long long* b = &tr[mid + (size_t)(it + 1) * kTracePhases];
                if (!a[0] || !b[0]) break;
                for (int k = 1; k < kTracePhases; ++k) sum[k] += (double)(a[k] - a[k - 1]);
                sum[0] += (double)(b[0] - a[kTracePhases - 1]);
                ++n_it;
            }
            fprintf(stderr, "FE_TRACE mid-cta %d iterations, ns per phase:", n_it);
            for (int k = 0; k < kTracePhases; ++k) fprintf(stderr, " %d:%.0f", k, n_it ? sum[k] / n_it : 0.0);
            fprintf(stderr, "\n");
            // FE_TRACE_DUMP=<path>: raw stamps and per-CTA row counts
            // (header: n_cta, iterations, phases, stats per CTA, as int64)
            const char* dump = getenv("FE_TRACE_DUMP");
            if (dump && dump[0]) {
                if (FILE* f = fopen(dump, "wb")) {
                    const long long hdr[4] = {P.n_cta, kTraceIters, kTracePhases, kTraceStats};
                    fwrite(hdr, sizeof hdr, 1, f);
                    fwrite(tr.data(), sizeof(unsigned long long), (size_t)P.n_cta * kTraceIters * kTracePhases, f);
                    fwrite(tr.data() + (size_t)P.n_cta * kTraceIters * kTracePhases, sizeof(unsigned long long),
                           (size_t)P.n_cta * kTraceStats, f);
                    fclose(f);
                }
            }
        }
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

// ---------------------------------------------------------------------------
// Jobs (struct SolveJob in solve_kernels.cuh): independent solves that share one cooperative launch.  A job is one
// system with up to 32 right-hand sides, padded to a power-of-two tile width
// with zero columns (a zero right-hand side is converged at its first
// residual).  The server packs jobs of one width and precision into a launch.
// ---------------------------------------------------------------------------
fe_status job_create(fe_ctx* ctx, const fe_system* s, int nrhs, const double2* d_b, const fe_solve_opts& o,
                     SolveJob** out) {
    *out = nullptr;
    if (nrhs < 1 || nrhs > 32) {
        set_error("job: nrhs %d outside 1..32", nrhs);
        return FE_ERR_INVALID_ARG;
    }
    const int prec = o.precision;
    FE_TRY(check_system_precision(s, prec, "job"));
    if (o.preconditioner != FE_PRECOND_BLOCK_JACOBI) {
        set_error("job: multi-system launches use block Jacobi");
        return FE_ERR_INVALID_ARG;
    }
    SolveJob* j = new (std::nothrow) SolveJob();
    if (!j) {
        set_error("job: host allocation failed");
        return FE_ERR_OOM;
    }
    j->sys = s;
    j->nrhs = nrhs;
    j->R = pick_tile(nrhs, 0);
    j->prec = prec;
    j->n_dof = 3 * (int64_t)s->mesh->n_act;
    cudaStream_t st = ctx->stream;
    fe_status e = alloc_workspace(st, j->n_dof, j->R, prec, 2 * ctx->num_sms, j->w, packed_entries(s, prec, j->R));
    if (e != FE_OK) {
        delete j;
        return e;
    }
    if ((e = dev_alloc(st, j->w.state, sizeof(JobState))) != FE_OK ||
        cudaMemsetAsync(j->w.state.ptr, 0, sizeof(JobState), st) != cudaSuccess) {
        free_workspace(st, j->w);
        delete j;
        if (e == FE_OK) set_error("job: state reset failed");
        return e == FE_OK ? FE_ERR_CUDA : e;
    }
    const unsigned gb = (unsigned)((j->n_dof * j->R + 255) / 256);
    k_gather_cols<<<gb, 256, 0, st>>>(d_b, nrhs, 0, nrhs, (double2*)j->w.b.ptr, j->R, j->n_dof);
    count_launches(1);
    fill_params(j->P, s, j->w, j->R, prec, o, false);
    j->P.state = (JobState*)j->w.state.ptr;
    *out = j;
    return FE_OK;
}

int job_width(const SolveJob* j) { return j->R; }
int64_t job_rows(const SolveJob* j) { return j->P.n_rows; }

void job_destroy(fe_ctx* ctx, SolveJob* j) {
    if (!j) return;
    free_workspace(ctx->stream, j->w);
    delete j;
}

// Enqueues one cooperative launch of n jobs of one width and precision on
// `stream`; job i gets n_cta[i] CTAs (1..its row count) and runs at most
// seg_iters[i] iterations (seg_iters NULL or 0: to the end), resuming where
// its last launch stopped.  A job must keep its CTA count from launch to launch: the CTAs
// own its vector rows.
fe_status jobs_launch(fe_ctx* ctx, SolveJob* const* jobs, const int* n_cta, int n, cudaStream_t stream,
                      const int* seg_iters) {
    if (n < 1) return FE_OK;
    const int R = jobs[0]->R;
    const int prec = jobs[0]->prec;
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        if (jobs[i]->R != R || jobs[i]->prec != prec) {
            set_error("jobs: one launch takes one tile width and one precision");
            return FE_ERR_INVALID_ARG;
        }
        if (n_cta[i] < 1 || n_cta[i] > std::max(1, jobs[i]->P.n_rows)) {
            set_error("jobs: job %d asks for %d CTAs", i, n_cta[i]);
            return FE_ERR_INVALID_ARG;
        }
        total += n_cta[i];
    }
    if (total > ctx->num_sms) {
        set_error("jobs: %lld CTAs exceed one per SM", (long long)total);
        return FE_ERR_INVALID_ARG;
    }
    return with_inner_type(prec, [&](auto* tag) {
        return launch_jobs_w<std::remove_pointer_t<decltype(tag)>>(ctx, R, jobs, n_cta, n, stream, seg_iters);
    });
}

// A job's progress after a launch, from its state block: whether the solve
// has ended (every column done, or a device error), the iterations its last
// segment ran and their device time.  `stream` must have finished the job's
// last launch.
fe_status job_progress(SolveJob* j, cudaStream_t stream, bool* finished, int* seg_done, double* seg_ms) {
    struct {
        int started, finished, any_repl, any_refresh, seg_done, pad[3];
        unsigned long long seg_ns;
    } h{};
    static_assert(sizeof(h) == offsetof(JobState, seg_ns) + sizeof(unsigned long long), "state header layout");
    FE_CUDA(cudaMemcpyAsync(&h, j->w.state.ptr, sizeof(h), cudaMemcpyDeviceToHost, stream));
    FE_CUDA(cudaStreamSynchronize(stream));
    *finished = h.finished != 0;
    *seg_done = h.seg_done;
    *seg_ms = (double)h.seg_ns * 1e-6;
    return FE_OK;
}

// Copies a finished job's solution (the nrhs real columns, [n_dof][nrhs]) and
// reports to the host; waits for the context's stream.
fe_status job_collect(fe_ctx* ctx, SolveJob* j, fe_complex* x_host, fe_solve_report* rep) {
    cudaStream_t st = ctx->stream;
    const int R = j->R;
    std::vector<int> ri(3 * R);
    std::vector<double> rd(R);
    SyncState hs{};
    if (x_host)
        FE_CUDA(cudaMemcpy2DAsync(x_host, (size_t)j->nrhs * sizeof(double2), j->w.x.ptr, (size_t)R * sizeof(double2),
                                  (size_t)j->nrhs * sizeof(double2), (size_t)j->n_dof, cudaMemcpyDeviceToHost, st));
    FE_CUDA(cudaMemcpyAsync(ri.data(), j->P.rep_status, 3 * R * sizeof(int), cudaMemcpyDeviceToHost, st));
    FE_CUDA(cudaMemcpyAsync(rd.data(), j->P.rep_rel, R * sizeof(double), cudaMemcpyDeviceToHost, st));
    FE_CUDA(cudaMemcpyAsync(&hs, j->P.sync, sizeof(SyncState), cudaMemcpyDeviceToHost, st));
    FE_CUDA(cudaStreamSynchronize(st));
    fe_status worst = FE_OK;
    for (int c = 0; c < j->nrhs; ++c) {
        if (rep) {
            rep[c].status = ri[c];
            rep[c].iterations = ri[R + c];
            rep[c].outer = ri[2 * R + c];
            rep[c].reserved = 0;
            rep[c].rel_residual = rd[c];
        }
        if (ri[c] != FE_OK && worst == FE_OK) worst = (fe_status)ri[c];
    }
    if (hs.err) {
        set_error("job: a barrier wait expired (device status %d)", hs.err);
        return FE_ERR_TIMEOUT;
    }
    if (worst != FE_OK) set_error("job: at least one right-hand side did not reach the tolerance");
    return worst;
}

// ---------------------------------------------------------------------------
// Fixed scratch for callers that cannot allocate device memory.
//
// fe_solve_rhs_noalloc keeps its whole workspace (Krylov vectors, reduction
// partials, barrier state, reports) in this file-scope device array instead
// of allocating it per call.  Every GPU that loads the library holds the array
// until the process exits.  Host code must not use `g_solve_scratch` as a
// device address (it is a host-side stand-in); the address is looked up once
// per device with cudaGetSymbolAddress while that device is current.
// ---------------------------------------------------------------------------
constexpr size_t kStaticScratchBytes = (size_t)32 << 20;  // 32 MiB per device
static __device__ __align__(256) unsigned char g_solve_scratch[kStaticScratchBytes];
constexpr int kMaxDevices = 64;
static void* g_scratch_addr[kMaxDevices] = {nullptr};

// Forgets the cached address of a device whose context was destroyed (for
// example by cudaDeviceReset): the next call looks it up again.
static void forget_scratch_on(int device, cudaError_t e) {
    if (device >= 0 && device < kMaxDevices &&
        (e == cudaErrorContextIsDestroyed || e == cudaErrorDeviceUninitialized || e == cudaErrorInvalidResourceHandle))
        g_scratch_addr[device] = nullptr;
}

// A caller buffer must be device memory of the context's device (the call
// copies nothing: its kernel reads b and writes x in place).
static fe_status check_device_buffer(const void* p, int device, const char* what) {
    cudaPointerAttributes a{};
    const cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();  // clear the (non-sticky) error the query recorded
        set_error("fe_solve_rhs_noalloc: %s is not a device pointer (%s)", what, cudaGetErrorString(e));
        return FE_ERR_INVALID_ARG;
    }
    if ((a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != device) {
        set_error("fe_solve_rhs_noalloc: %s must be device memory of device %d (memory type %d, device %d)", what,
                  device, (int)a.type, a.device);
        return FE_ERR_INVALID_ARG;
    }
    return FE_OK;
}

static fe_status static_scratch(int device, char** out) {
    if (device < 0 || device >= kMaxDevices) {
        set_error("fe_solve_rhs_noalloc: device %d outside 0..%d", device, kMaxDevices - 1);
        return FE_ERR_INVALID_ARG;
    }
    if (!g_scratch_addr[device]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_solve_scratch);
        if (e != cudaSuccess || !ptr) {
            set_error("fe_solve_rhs_noalloc: cudaGetSymbolAddress of the static scratch failed: %s",
                      cudaGetErrorString(e));
            return FE_ERR_CUDA;
        }
        g_scratch_addr[device] = ptr;
    }
    *out = (char*)g_scratch_addr[device];
    return FE_OK;
}

static fe_status check_opts(const fe_solve_opts* o, fe_solve_opts& out) {
    fe_solve_opts_default(&out);
    if (o) out = *o;
    if (out.precision != FE_PREC_FP64 && out.precision != FE_PREC_MIXED && out.precision != FE_PREC_DF) {
        set_error("solve: precision must be FP64, MIXED or DF");
        return FE_ERR_INVALID_ARG;
    }
    if (!(out.tol > 0.0) || out.max_iter < 1 || out.max_outer < 1 || !(out.reliable >= 0.0 && out.reliable < 1.0) ||
        out.rhs_tile < 0 || out.max_pass_iter < 0 || out.wait_timeout_us < 0) {
        set_error("solve: bad tolerance or iteration limits");
        return FE_ERR_INVALID_ARG;
    }
    if (out.recurrence != FE_RECURRENCE_CG && out.recurrence != FE_RECURRENCE_EXPANDED) {
        set_error("solve: unknown recurrence %d", (int)out.recurrence);
        return FE_ERR_INVALID_ARG;
    }
    if (out.preconditioner != FE_PRECOND_BLOCK_JACOBI && out.preconditioner != FE_PRECOND_BICP) {
        set_error("solve: unknown preconditioner %d", (int)out.preconditioner);
        return FE_ERR_INVALID_ARG;
    }
    if (out.preconditioner == FE_PRECOND_BICP && out.precision != FE_PREC_FP64) {
        set_error("solve: the block incomplete Cholesky preconditioner runs with FE_PREC_FP64 only");
        return FE_ERR_INVALID_ARG;
    }
    return FE_OK;
}

// A block incomplete Cholesky solve needs a factor with one band per CTA of
// the solve grid (min(SMs, rows), the grid launch_solve uses).
static fe_status check_precond(const fe_ctx* ctx, const fe_system* s, const fe_solve_opts& o, const char* what) {
    if (o.preconditioner != FE_PRECOND_BICP) return FE_OK;
    const int grid = std::min(ctx->num_sms, std::max(1, s->mesh->n_act));
    if (s->bicp_n_sub < 1) {
        set_error("%s: no block incomplete Cholesky factor (call fe_system_factor_bicp first)", what);
        return FE_ERR_INVALID_ARG;
    }
    if (s->bicp_n_sub != grid) {
        set_error("%s: the factor has %d bands, the solve runs %d CTAs", what, s->bicp_n_sub, grid);
        return FE_ERR_INVALID_ARG;
    }
    return FE_OK;
}

}  // namespace fe

using namespace fe;

extern "C" {

void fe_solve_opts_default(fe_solve_opts* o) {
    if (!o) return;
    o->precision = FE_PREC_DF;
    o->tol = 1e-8;
    o->reliable = 1e-4;
    o->max_iter = 100000;
    o->max_outer = 200;
    o->rhs_tile = 0;
    o->max_pass_iter = 2000;
    o->wait_timeout_us = 4000000;
    o->preconditioner = FE_PRECOND_BLOCK_JACOBI;
    o->recurrence = FE_RECURRENCE_CG;
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


fe_status fe_solve_rhs_noalloc(fe_ctx* ctx, const fe_system* s, int32_t nrhs, const void* b_dev, void* x_dev,
                               int32_t use_x0, const fe_solve_opts* o, fe_solve_report* rep) {
    if (!ctx || !s || !b_dev || !x_dev) {
        set_error("fe_solve_rhs_noalloc: NULL argument");
        return FE_ERR_INVALID_ARG;
    }
    if (nrhs != 1 && nrhs != 2 && nrhs != 4 && nrhs != 8 && nrhs != 16 && nrhs != 32) {
        set_error("fe_solve_rhs_noalloc: nrhs must be 1, 2, 4, 8, 16 or 32 (got %d)", nrhs);
        return FE_ERR_INVALID_ARG;
    }
    fe_solve_opts opt;
    FE_TRY(check_opts(o, opt));
    const int prec = opt.precision;
    FE_TRY(check_system_precision(s, prec, "fe_solve_rhs_noalloc"));
    FE_TRY(check_precond(ctx, s, opt, "fe_solve_rhs_noalloc"));
    FE_CUDA(cudaSetDevice(ctx->device));
    FE_TRY(check_device_buffer(b_dev, ctx->device, "b_dev"));
    FE_TRY(check_device_buffer(x_dev, ctx->device, "x_dev"));
    char* base = nullptr;
    FE_TRY(static_scratch(ctx->device, &base));
    const fe_mesh* m = s->mesh;
    const int R = nrhs;
    const size_t nv = (size_t)3 * m->n_act * R;
    const size_t esz = inner_bytes(prec);
    const int max_cta = 2 * ctx->num_sms;
    // carve the workspace out of the static array, 256-byte aligned pieces;
    // b and x are the caller's buffers
    size_t off = 0;
    auto take = [&](DevBuf& b, size_t bytes) {
        b.ptr = base + off;
        b.bytes = bytes;
        off += (bytes + 255) & ~(size_t)255;
    };
    Workspace w;
    w.b.ptr = const_cast<void*>(b_dev);
    w.x.ptr = x_dev;
    take(w.r, nv * sizeof(double2));
    take(w.u, nv * sizeof(double2));
    take(w.p, nv * sizeof(double2));
    take(w.s, nv * sizeof(double2));
    take(w.w, nv * esz);
    if (!split_copies(prec, R)) {
        w.uM = w.u;
        w.pM = w.p;
    } else {
        take(w.uM, nv * esz);
        take(w.pM, nv * esz);
    }
    take(w.partial, (size_t)max_cta * kMaxNV * R * sizeof(double));
    take(w.result, (size_t)kMaxNV * R * sizeof(double));
    take(w.sync, sync_bytes(max_cta));
    take(w.rep, (size_t)R * (3 * sizeof(int) + sizeof(double)) + 64);
    if (off > kStaticScratchBytes) {
        set_error("fe_solve_rhs_noalloc: needs %zu bytes of scratch, the static array holds %zu (n_dof x nrhs too "
                  "large)",
                  off, kStaticScratchBytes);
        return FE_ERR_INVALID_ARG;
    }
    cudaStream_t st = ctx->stream;
    {
        const cudaError_t ce = cudaMemsetAsync(w.sync.ptr, 0, sync_bytes(ctx->num_sms), st);  // the array keeps old contents
        if (ce != cudaSuccess) {
            forget_scratch_on(ctx->device, ce);
            set_error("fe_solve_rhs_noalloc: %s", cudaGetErrorString(ce));
            return FE_ERR_CUDA;
        }
    }
    SolveParams P;
    fill_params(P, s, w, R, prec, opt, use_x0 != 0);
    P.trace = nullptr;
    SyncState* sync = P.sync;
    int* ri = P.rep_status;
    double* rrel = P.rep_rel;
    ctx->last_solve = fe_solve_stats{};
    FE_TRY(with_inner_type(prec, [&](auto* tag) { return dispatch<std::remove_pointer_t<decltype(tag)>>(ctx, R, P); }));
    SyncState hs{};
    int h_ri[3 * 32];
    double h_rel[32];
    FE_CUDA(cudaMemcpyAsync(&hs, sync, sizeof(SyncState), cudaMemcpyDeviceToHost, st));
    FE_CUDA(cudaMemcpyAsync(h_ri, ri, (size_t)3 * R * sizeof(int), cudaMemcpyDeviceToHost, st));
    FE_CUDA(cudaMemcpyAsync(h_rel, rrel, (size_t)R * sizeof(double), cudaMemcpyDeviceToHost, st));
    {
        const cudaError_t ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) {
            forget_scratch_on(ctx->device, ce);
            set_error("fe_solve_rhs_noalloc: %s", cudaGetErrorString(ce));
            return FE_ERR_CUDA;
        }
    }
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1) == cudaSuccess) ctx->last_solve.kernel_ms = ms;
    if (hs.err) {
        set_error("fe_solve_rhs_noalloc: a grid barrier wait expired (device status %d)", hs.err);
        return FE_ERR_TIMEOUT;
    }
    fe_status worst = FE_OK;
    for (int c = 0; c < R; ++c) {
        if (rep) {
            rep[c].status = h_ri[c];
            rep[c].iterations = h_ri[R + c];
            rep[c].outer = h_ri[2 * R + c];
            rep[c].reserved = 0;
            rep[c].rel_residual = h_rel[c];
        }
        ctx->last_solve.inner_iters += h_ri[R + c];
        if (h_ri[c] != FE_OK && worst == FE_OK) worst = (fe_status)h_ri[c];
    }
    if (worst != FE_OK) set_error("fe_solve_rhs_noalloc: at least one right-hand side did not reach the tolerance");
    return worst;
}

}  // extern "C"
