// Serving: a request queue solved with continuous batching.
//
// A worker thread owns an internal context (its own stream on the caller's
// device) and one more stream per right-hand-side tile width.  Solves run in
// segments: a persistent multi-system launch advances each of its requests
// by at most seg_iters iterations and saves their Krylov state on the device
// (solve_kernels.cuh, JobState).  Each loop turn the worker
//   1. admits queued requests in arrival order while the sum of their
//      estimated device bytes fits the budget, and builds each one's mesh,
//      system and right-hand sides (the same kernels as fe_mesh_create /
//      fe_assemble / fe_rhs);
//   2. plans the segment with fe_serve_plan over all active requests: every
//      request has a CTA count fixed by its own size, and requests run in
//      arrival order while their counts fit the device;
//   3. starts one cooperative launch per tile width, each on its own stream,
//      so that widths run side by side on disjoint SMs, and waits for them;
//   4. hands out the requests that finished and frees their memory.
// A request submitted meanwhile is admitted at the next turn, a few
// milliseconds later, and runs beside the requests already in flight.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>

#include "fe_internal.cuh"

namespace fe {
struct SolveJob;
fe_status job_create(fe_ctx* ctx, const fe_system* s, int nrhs, const double2* d_b, const fe_solve_opts& o,
                     SolveJob** out);
int job_width(const SolveJob* j);
int64_t job_rows(const SolveJob* j);
void job_destroy(fe_ctx* ctx, SolveJob* j);
fe_status jobs_launch(fe_ctx* ctx, SolveJob* const* jobs, const int* n_cta, int n, cudaStream_t stream,
                      const int* seg_iters);
fe_status job_progress(SolveJob* j, cudaStream_t stream, bool* finished, int* seg_done, double* seg_ms);
fe_status job_collect(fe_ctx* ctx, SolveJob* j, fe_complex* x_host, fe_solve_report* rep);
size_t workspace_bytes(int64_t n_dof, int R, int prec, int max_cta, int64_t pk_entries);
fe_status build_rhs(fe_ctx* ctx, const fe_system* s, int nrhs, const fe_planewave* waves, double2* d_B,
                    DevBuf& wave_buf);

namespace {

using Clock = std::chrono::steady_clock;

struct ServeReq {
    uint64_t ticket = 0;
    fe_mesh_desc desc{};
    std::vector<uint8_t> material;
    std::vector<fe_complex> eps, mu;
    double freq = 0.0;
    std::vector<fe_planewave> waves;
    int width = 1;  // power-of-two tile width >= nrhs
    int64_t est_bytes = 0;
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
    fe_mesh* mesh = nullptr;
    fe_system* sys = nullptr;
    SolveJob* job = nullptr;
    bool done = false;
    int status = FE_PENDING;
    std::string message;
    int64_t n_dof = 0;
    std::vector<fe_complex> x;
    std::vector<int32_t> node_id;
    std::vector<fe_solve_report> rep;
    int batch_jobs = 0, batch_ctas = 0;
    int segments = 0;         // segments the request has run in
    double ms_per_iter = 0.0;  // device time per iteration measured in its last segment (0: none yet)
};

// Segments last about kSegTargetMs: each request runs as many iterations as
// its own measured time per iteration allows, so that a small request
// launched beside a large one keeps its SMs busy for the whole segment.
constexpr double kSegTargetMs = 25.0;
constexpr int kSegFirst = 64;

int segment_iters(const fe_serve_opts& o, const ServeReq* q) {
    if (o.seg_iters > 0) return o.seg_iters;
    if (!(q->ms_per_iter > 0.0)) return kSegFirst;
    return (int)std::max(16.0, std::min(1e6, kSegTargetMs / q->ms_per_iter));
}

int width_slot(int width) {
    int k = 0;
    while ((1 << k) < width && k < 5) ++k;
    return k;
}

int tile_width(int nrhs) {
    int R = 1;
    while (R < nrhs) R <<= 1;
    return R;
}

// Upper bound of the device bytes a request holds while admitted: the mesh
// maps, the block values (complex128, plus complex64 in the mixed mode), the
// block-Jacobi inverses, the right-hand sides and the Krylov workspace, for
// the worst case of every grid node active with 27 neighbours.
int64_t estimate_bytes(const fe_mesh_desc& d, int nrhs, int width, int prec, int num_sms) {
    const int64_t n_el = (int64_t)d.nx * d.ny * d.nz;
    const int64_t nodes = (int64_t)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
    const int64_t nnzb = 27 * nodes;
    const int64_t stride = (nnzb + 63) / 64 * 64;
    const int64_t mesh = n_el + 8 * nodes + 4 * (nodes + 1) + 4 * nnzb + 256 * n_el + 24 * n_el;
    // complex128 values, plus the complex64 or FP32-pair copy
    const int64_t per_entry = prec == FE_PREC_FP64 ? 16 : (prec == FE_PREC_MIXED ? 24 : 32);
    const int64_t sys = 9 * stride * per_entry + 9 * nodes * 24 + nodes * 13 + 65536;
    const int64_t rhs = 3 * nodes * (int64_t)nrhs * 16;
    // the packed explicit rows of a single-column launch: at most every block
    const int64_t pk = (width == 1 && prec != FE_PREC_FP64) ? 9 * nnzb : 0;
    const int64_t ws = (int64_t)workspace_bytes(3 * nodes, width, prec, 2 * num_sms, pk);
    return (mesh + sys + rhs + ws) * 11 / 10 + (1 << 20);
}

}  // namespace
}  // namespace fe

using namespace fe;

struct fe_server {
    fe_ctx* ictx = nullptr;
    int device = 0;
    fe_serve_opts o{};
    fe_solve_opts so{};
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ServeReq*> queue;                  // submitted, not admitted
    std::vector<ServeReq*> ready;                 // admitted and built, in arrival order (worker only)
    cudaStream_t wstream[6] = {};                 // one launch stream per tile width 1..32
    std::unordered_map<uint64_t, ServeReq*> all;  // every unreleased ticket
    uint64_t next_ticket = 1;
    bool stop = false;
    int64_t used = 0;
    fe_serve_stats stats{};
    Clock::time_point t0;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// Frees a request's device objects (stream-ordered) and publishes its result.
void finish(fe_server* S, ServeReq* q, int status, const char* msg) {
    job_destroy(S->ictx, q->job);
    q->job = nullptr;
    if (q->sys) fe_system_destroy(q->sys);
    q->sys = nullptr;
    if (q->mesh) fe_mesh_destroy(q->mesh);
    q->mesh = nullptr;
    std::lock_guard<std::mutex> lk(S->mu);
    q->status = status;
    q->message = msg ? msg : "";
    q->t_done = S->now();
    q->done = true;
    S->used -= q->est_bytes;
    S->stats.completed += 1;
    if (status != FE_OK) S->stats.failed += 1;
    S->cv_done.notify_all();
}

// Builds mesh, system, right-hand sides and solve job of an admitted request.
fe_status build_request(fe_server* S, ServeReq* q) {
    fe_ctx* c = S->ictx;
    fe_mesh_desc d = q->desc;
    d.material = q->material.data();
    d.material_on_device = 0;
    d.eps_r = q->eps.data();
    d.mu_r = q->mu.data();
    FE_TRY(fe_mesh_create(c, &d, &q->mesh));
    q->n_dof = 3 * (int64_t)q->mesh->n_act;
    q->node_id.resize(q->mesh->n_act);
    if (q->mesh->n_act > 0)
        FE_CUDA(cudaMemcpyAsync(q->node_id.data(), q->mesh->node_id.ptr, q->node_id.size() * sizeof(int32_t),
                                cudaMemcpyDeviceToHost, c->stream));
    FE_TRY(fe_assemble(c, q->mesh, q->freq, S->so.precision, &q->sys));
    const int nrhs = (int)q->waves.size();
    DevBuf B, wave_buf;
    FE_TRY(dev_alloc(c->stream, B, (size_t)q->n_dof * nrhs * sizeof(double2)));
    fe_status e = build_rhs(c, q->sys, nrhs, q->waves.data(), (double2*)B.ptr, wave_buf);
    if (e == FE_OK) e = job_create(c, q->sys, nrhs, (const double2*)B.ptr, S->so, &q->job);
    dev_free(c->stream, wave_buf);
    dev_free(c->stream, B);
    return e;
}

// One turn of the worker: admit, build, run one segment.  Returns false to stop.
bool worker_turn(fe_server* S) {
    std::vector<ServeReq*> admitted;
    std::vector<std::pair<ServeReq*, std::string>> rejected;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty() || !S->ready.empty(); });
        if (S->stop) return false;
        while (!S->queue.empty()) {
            ServeReq* q = S->queue.front();
            if (q->est_bytes > S->stats.budget_bytes) {
                S->queue.pop_front();
                S->used += q->est_bytes;  // returned by finish()
                char buf[160];
                snprintf(buf, sizeof buf, "request needs about %lld device bytes, above the budget of %lld",
                         (long long)q->est_bytes, (long long)S->stats.budget_bytes);
                rejected.emplace_back(q, buf);
                continue;
            }
            if (S->used + q->est_bytes > S->stats.budget_bytes) break;  // wait for memory
            S->queue.pop_front();
            S->used += q->est_bytes;
            S->stats.peak_admitted_bytes = std::max(S->stats.peak_admitted_bytes, S->used);
            q->t_admit = S->now();
            admitted.push_back(q);
        }
    }
    for (auto& r : rejected) finish(S, r.first, FE_ERR_OOM, r.second.c_str());
    for (ServeReq* q : admitted) {
        const fe_status e = build_request(S, q);
        if (e != FE_OK) {
            const std::string msg = fe_last_error();
            finish(S, q, e, msg.c_str());
        } else {
            S->ready.push_back(q);
        }
    }
    if (S->ready.empty()) return true;
    // the builds ran on the internal stream; the launches use the width streams
    if (cudaStreamSynchronize(S->ictx->stream) != cudaSuccess) {
        const std::string msg = std::string("serve: build failed: ") + cudaGetErrorString(cudaGetLastError());
        for (ServeReq* q : S->ready) finish(S, q, FE_ERR_CUDA, msg.c_str());
        S->ready.clear();
        return true;
    }

    // plan the segment: fixed CTA counts, arrival order, later requests backfill
    const int n = (int)S->ready.size();
    std::vector<int64_t> rows(n);
    std::vector<int32_t> width(n), n_cta(n, 0);
    for (int i = 0; i < n; ++i) {
        rows[i] = job_rows(S->ready[i]->job);
        width[i] = job_width(S->ready[i]->job);
    }
    const int max_ctas = S->o.max_ctas > 0 ? std::min(S->o.max_ctas, S->ictx->num_sms) : S->ictx->num_sms;
    // default cap: three quarters of the device, so that requests arriving
    // while a large one runs find CTAs beside it
    const int max_job = S->o.max_job_ctas > 0 ? std::min(S->o.max_job_ctas, max_ctas) : std::max(1, max_ctas * 3 / 4);
    fe_serve_plan(n, rows.data(), width.data(), max_ctas, max_job, S->o.work_per_cta, n_cta.data());
    std::vector<SolveJob*> jobs[6];
    std::vector<int> ctas[6], iters[6];
    std::vector<ServeReq*> in_seg[6];
    int n_seg = 0;
    for (int i = 0; i < n; ++i) {
        if (n_cta[i] <= 0) continue;
        const int k = width_slot(width[i]);
        jobs[k].push_back(S->ready[i]->job);
        ctas[k].push_back(n_cta[i]);
        iters[k].push_back(segment_iters(S->o, S->ready[i]));
        in_seg[k].push_back(S->ready[i]);
        ++n_seg;
    }
    const auto t_seg0 = Clock::now();
    fe_status e = FE_OK;
    int launched = 0;
    for (int k = 0; k < 6 && e == FE_OK; ++k) {
        if (jobs[k].empty()) continue;
        e = jobs_launch(S->ictx, jobs[k].data(), ctas[k].data(), (int)jobs[k].size(), S->wstream[k],
                        iters[k].data());
        if (e == FE_OK) ++launched;
    }
    std::string launch_msg = e == FE_OK ? std::string() : std::string(fe_last_error());
    for (int k = 0; k < 6; ++k) {
        if (jobs[k].empty()) continue;
        const cudaError_t ce = cudaStreamSynchronize(S->wstream[k]);
        if (ce != cudaSuccess && e == FE_OK) {
            e = FE_ERR_CUDA;
            launch_msg = std::string("serve: solve launch failed: ") + cudaGetErrorString(ce);
        }
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stats.solve_device_s += std::chrono::duration<double>(Clock::now() - t_seg0).count();
        S->stats.launches += launched;
        S->stats.jobs_launched += n_seg;
    }
    // hand out what finished; the rest stays for the next segment
    std::vector<ServeReq*> keep;
    for (ServeReq* q : S->ready) {
        const int k = width_slot(job_width(q->job));
        bool ran = false;
        for (size_t i = 0; i < in_seg[k].size(); ++i)
            if (in_seg[k][i] == q) {
                ran = true;
                q->batch_jobs = std::max(q->batch_jobs, n_seg);
                q->batch_ctas = ctas[k][i];
            }
        if (!ran) {
            keep.push_back(q);
            continue;
        }
        q->segments += 1;
        if (e != FE_OK) {
            finish(S, q, e, launch_msg.c_str());
            continue;
        }
        bool fin = false;
        int done_it = 0;
        double seg_ms = 0.0;
        const fe_status ef = job_progress(q->job, S->wstream[k], &fin, &done_it, &seg_ms);
        if (done_it > 0) q->ms_per_iter = seg_ms / done_it;
        if (ef != FE_OK) {
            const std::string msg = fe_last_error();
            finish(S, q, ef, msg.c_str());
            continue;
        }
        if (!fin) {
            keep.push_back(q);
            continue;
        }
        q->x.resize((size_t)q->n_dof * q->waves.size());
        q->rep.resize(q->waves.size());
        const fe_status es = job_collect(S->ictx, q->job, q->x.data(), q->rep.data());
        const std::string msg = es == FE_OK ? std::string() : std::string(fe_last_error());
        finish(S, q, es, msg.c_str());
    }
    S->ready.swap(keep);
    return true;
}

void worker_main(fe_server* S) {
    cudaSetDevice(S->device);
    for (;;) {
        bool go = false;
        try {
            go = worker_turn(S);
        } catch (...) {  // host allocation failure: fail what is queued and ready, keep serving
            std::vector<ServeReq*> drop;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                drop.assign(S->queue.begin(), S->queue.end());
                S->queue.clear();
                for (ServeReq* q : drop) S->used += q->est_bytes;
            }
            drop.insert(drop.end(), S->ready.begin(), S->ready.end());
            S->ready.clear();
            for (ServeReq* q : drop) finish(S, q, FE_ERR_OOM, "host allocation failed in the server");
            go = true;
        }
        if (!go) return;
    }
}

void fill_result(const ServeReq* q, fe_result* out) {
    out->status = q->status;
    out->nrhs = (int32_t)q->waves.size();
    out->n_dof = q->n_dof;
    out->x = q->x.empty() ? nullptr : q->x.data();
    out->node_id = q->node_id.empty() ? nullptr : q->node_id.data();
    out->reports = q->rep.empty() ? nullptr : q->rep.data();
    out->t_submit = q->t_submit;
    out->t_admit = q->t_admit;
    out->t_done = q->t_done;
    out->batch_jobs = q->batch_jobs;
    out->batch_ctas = q->batch_ctas;
    out->message = q->message.c_str();
}

}  // namespace

extern "C" {

void fe_serve_opts_default(fe_serve_opts* o) {
    if (!o) return;
    o->precision = FE_PREC_DF;
    o->tol = 1e-8;
    o->reliable = 1e-4;
    o->max_iter = 100000;
    o->max_outer = 200;
    o->hbm_budget = 0;
    o->max_ctas = 0;
    o->work_per_cta = 2048;
    o->max_job_ctas = 0;
    o->seg_iters = 0;
    o->recurrence = FE_RECURRENCE_EXPANDED;  // the stream's large requests have long plateaus
}

int32_t fe_serve_plan(int32_t n, const int64_t* rows, const int32_t* width, int32_t max_ctas, int32_t max_job_ctas,
                      int32_t work_per_cta, int32_t* n_cta) {
    if (n <= 0 || !rows || !width || !n_cta || max_ctas < 1) return 0;
    if (work_per_cta < 1) work_per_cta = 2048;
    if (max_job_ctas < 1 || max_job_ctas > max_ctas) max_job_ctas = max_ctas;
    int32_t remaining = max_ctas, taken = 0;
    for (int i = 0; i < n; ++i) {
        n_cta[i] = 0;
        const int64_t r = std::max<int64_t>(rows[i], 1);
        int64_t want = (r * std::max(width[i], 1) + work_per_cta - 1) / work_per_cta;
        want = std::max<int64_t>(1, std::min<int64_t>(want, std::min<int64_t>(r, max_job_ctas)));
        if (want <= remaining) {
            n_cta[i] = (int32_t)want;
            remaining -= (int32_t)want;
            ++taken;
        }
    }
    return taken;
}

fe_status fe_serve_create(fe_ctx* ctx, const fe_serve_opts* opt, fe_server** out) {
    if (!ctx || !out) {
        set_error("fe_serve_create: NULL argument");
        return FE_ERR_INVALID_ARG;
    }
    *out = nullptr;
    fe_serve_opts o;
    fe_serve_opts_default(&o);
    if (opt) o = *opt;
    if (o.work_per_cta <= 0) o.work_per_cta = 2048;
    if ((o.precision != FE_PREC_FP64 && o.precision != FE_PREC_MIXED && o.precision != FE_PREC_DF) ||
        !(o.tol > 0.0) || o.max_iter < 1 ||
        o.max_outer < 1 || !(o.reliable >= 0.0 && o.reliable < 1.0) || o.hbm_budget < 0 || o.max_ctas < 0 ||
        o.max_job_ctas < 0 || o.seg_iters < 0 ||
        (o.recurrence != FE_RECURRENCE_CG && o.recurrence != FE_RECURRENCE_EXPANDED)) {
        set_error("fe_serve_create: option out of range");
        return FE_ERR_INVALID_ARG;
    }
    fe_server* S = new (std::nothrow) fe_server();
    if (!S) {
        set_error("fe_serve_create: host allocation failed");
        return FE_ERR_OOM;
    }
    S->device = ctx->device;
    S->o = o;
    fe_solve_opts_default(&S->so);
    S->so.precision = o.precision;
    S->so.tol = o.tol;
    S->so.reliable = o.reliable;
    S->so.max_iter = o.max_iter;
    S->so.max_outer = o.max_outer;
    S->so.recurrence = o.recurrence;
    fe_options io = ctx->opt;
    io.stream = nullptr;  // the server's own stream
    fe_status e = fe_ctx_create(&S->ictx, ctx->device, &io);
    if (e != FE_OK) {
        delete S;
        return e;
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        set_error("fe_serve_create: cudaMemGetInfo failed");
        fe_ctx_destroy(S->ictx);
        delete S;
        return FE_ERR_CUDA;
    }
    S->stats.budget_bytes = o.hbm_budget > 0 ? o.hbm_budget : (int64_t)(free_b / 10 * 8);
    for (int k = 0; k < 6; ++k)
        if (cudaStreamCreateWithFlags(&S->wstream[k], cudaStreamNonBlocking) != cudaSuccess) {
            set_error("fe_serve_create: stream creation failed");
            for (int q = 0; q < k; ++q) cudaStreamDestroy(S->wstream[q]);
            fe_ctx_destroy(S->ictx);
            delete S;
            return FE_ERR_CUDA;
        }
    S->t0 = Clock::now();
    try {
        S->worker = std::thread(worker_main, S);
    } catch (...) {
        set_error("fe_serve_create: could not start the worker thread");
        fe_ctx_destroy(S->ictx);
        delete S;
        return FE_ERR_OOM;
    }
    *out = S;
    return FE_OK;
}

fe_status fe_serve_submit(fe_server* S, const fe_request* r, uint64_t* ticket) {
    if (!S || !r || !ticket) {
        set_error("fe_serve_submit: NULL argument");
        return FE_ERR_INVALID_ARG;
    }
    const fe_mesh_desc& d = r->mesh;
    if (r->nrhs < 1 || r->nrhs > 32 || !r->waves || !(r->freq_hz > 0.0) || !d.material || d.material_on_device ||
        d.nx < 1 || d.ny < 1 || d.nz < 1 || d.n_materials < 1 || d.n_materials > 255 || !d.eps_r || !d.mu_r) {
        set_error("fe_serve_submit: bad request (nrhs 1..32, host material, sizes >= 1, 1..255 materials, f > 0)");
        return FE_ERR_INVALID_ARG;
    }
    const int64_t n_el = (int64_t)d.nx * d.ny * d.nz;
    if (n_el > ((int64_t)1 << 30)) {
        set_error("fe_serve_submit: %lld elements is too many", (long long)n_el);
        return FE_ERR_INVALID_ARG;
    }
    ServeReq* q = new (std::nothrow) ServeReq();
    if (!q) {
        set_error("fe_serve_submit: host allocation failed");
        return FE_ERR_OOM;
    }
    try {
        q->desc = d;
        q->material.assign(d.material, d.material + n_el);
        q->eps.assign(d.eps_r, d.eps_r + d.n_materials);
        q->mu.assign(d.mu_r, d.mu_r + d.n_materials);
        q->waves.assign(r->waves, r->waves + r->nrhs);
    } catch (...) {
        delete q;
        set_error("fe_serve_submit: host allocation failed");
        return FE_ERR_OOM;
    }
    q->freq = r->freq_hz;
    q->width = tile_width(r->nrhs);
    q->est_bytes = estimate_bytes(d, r->nrhs, q->width, S->o.precision, S->ictx->num_sms);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            delete q;
            set_error("fe_serve_submit: the server is stopping");
            return FE_ERR_INVALID_ARG;
        }
        q->ticket = S->next_ticket++;
        q->t_submit = S->now();
        S->all[q->ticket] = q;
        S->queue.push_back(q);
        S->stats.submitted += 1;
        *ticket = q->ticket;
    }
    S->cv_work.notify_one();
    return FE_OK;
}

fe_status fe_serve_poll(fe_server* S, uint64_t ticket, fe_result* out) {
    return fe_serve_wait(S, ticket, 0.0, out);
}

fe_status fe_serve_wait(fe_server* S, uint64_t ticket, double timeout_s, fe_result* out) {
    if (!S || !out) {
        set_error("fe_serve_wait: NULL argument");
        return FE_ERR_INVALID_ARG;
    }
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) {
        set_error("fe_serve_wait: unknown ticket %llu", (unsigned long long)ticket);
        return FE_ERR_INVALID_ARG;
    }
    ServeReq* q = it->second;
    if (!q->done && timeout_s > 0.0)
        S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return q->done; });
    if (!q->done) return FE_PENDING;
    fill_result(q, out);
    return FE_OK;
}

fe_status fe_serve_release(fe_server* S, uint64_t ticket) {
    if (!S) {
        set_error("fe_serve_release: NULL server");
        return FE_ERR_INVALID_ARG;
    }
    ServeReq* q = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->all.find(ticket);
        if (it == S->all.end()) {
            set_error("fe_serve_release: unknown ticket %llu", (unsigned long long)ticket);
            return FE_ERR_INVALID_ARG;
        }
        if (!it->second->done) return FE_PENDING;
        q = it->second;
        S->all.erase(it);
    }
    delete q;
    return FE_OK;
}

fe_status fe_serve_info(fe_server* S, fe_serve_stats* out) {
    if (!S || !out) {
        set_error("fe_serve_info: NULL argument");
        return FE_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    return FE_OK;
}

void fe_serve_destroy(fe_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (ServeReq* q : S->ready) {
        job_destroy(S->ictx, q->job);
        if (q->sys) fe_system_destroy(q->sys);
        if (q->mesh) fe_mesh_destroy(q->mesh);
        q->job = nullptr;
        q->sys = nullptr;
        q->mesh = nullptr;
    }
    for (auto& kv : S->all) delete kv.second;
    cudaStreamSynchronize(S->ictx->stream);
    for (int k = 0; k < 6; ++k)
        if (S->wstream[k]) cudaStreamDestroy(S->wstream[k]);
    fe_ctx_destroy(S->ictx);
    delete S;
}

}  // extern "C"
