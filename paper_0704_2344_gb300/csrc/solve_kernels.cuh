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
constexpr int kExplRows = 10;        // packed explicit rows: ten rows per warp, one lane per (row, component)
constexpr int kColsPerWarp = 272;    // >= 10 rows x 27 blocks
constexpr int kTracePhases = 8;

struct SyncState {
    unsigned count;
    unsigned gen;
    int err;
    int pad;
};
// Barrier state of one launch (zeroed before every launch).
inline size_t sync_bytes(int n_cta) {
    (void)n_cta;
    return sizeof(SyncState);
}

// Scalar state of a solve that runs in segments (serving): everything a
// persistent launch keeps in shared memory between iterations, saved by the
// job's first CTA when a segment ends and loaded by every CTA when the next
// one starts.  The vectors stay in the job's workspace, so a solve resumed
// this way performs exactly the operations of an uninterrupted one.
struct ColState {
    double bn, rr_ref, rel, gam_r, gam_i, al_r, al_i, be_r, be_i, igam_r, igam_i, ial_r, ial_i, pad;
    float4 a4, na4, b4;
    float4 gam4, igam4, ial4;  // FP32-pair solves: gamma, 1/gamma, 1/alpha as pairs
    long long xd[4];           // expanded recurrence: u^T s and p^T s of the last update (the raw 8-byte slots)
    int active, done, status, iters, outer, first, refresh, repl, pass_it, pad2[3];
};
struct JobState {
    int started;   // a segment has run (the next one resumes)
    int finished;  // every column is done: the solution is final (FP64) and the reports hold the results
    int any_repl, any_refresh;
    int seg_done;  // iterations the last segment ran
    int pad[3];
    unsigned long long seg_ns;  // device time of the last segment (its first CTA, start to end)
    ColState col[32];
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
    int seg_iters;     // iterations of this launch before the state is saved and the launch ends (0: to the end)
    int n_cta_req;     // CTAs of a single-system launch (0: one per SM)
    JobState* state;   // segmented solve state (NULL: one launch runs the whole solve)
    int halo;       // bound on |column rank - row rank|
    int stage;      // stage the CTA's uM halo in shared memory (1) or gather from L2 (0)
    int64_t halo_bytes;  // dynamic shared memory left for the halo (a CTA whose halo is larger gathers)
    int64_t part_half;   // doubles per parity buffer of the barrier partials (n_cta * kMaxNV * R)
    int red_bytes;  // dynamic shared memory used by the column sums
    int col_bytes;  // dynamic shared memory for the per-warp column-index staging (R = 1)
    // Resident product map (R = 1, complex64 and FP32-pair products): each
    // CTA sorts its product rows by cost once per launch and keeps them, their
    // block ranges and their columns resolved to positions in its staged halo
    // in shared memory; the halo is staged as up to three segments (the node
    // planes below, at and above the CTA's rows) instead of one window.
    int res;           // 1: the map is in use
    int res_rows_max;  // rows the map holds (a CTA with more rows uses the plain path)
    int res_tmid;      // |column - row| bound of same-plane neighbours (the middle segment)
    int res_bytes;     // dynamic shared memory of the map (a multiple of 16)
    // Packed explicit rows (with the map): each launch, every CTA copies the
    // values of its explicit rows into this buffer in the order its lanes read
    // them, so that each product step of a warp loads 30 consecutive entries
    // per block column instead of one scattered entry per lane; a CTA's part
    // starts at 9 * expl_prefix[first product row].  NULL: the lanes read the
    // planes.
    void* pk;                 // inner-precision entries [9 * explicit blocks]
    const int* expl_prefix;   // [n_rows + 1] stored blocks of explicit rows before each row
    // Block dictionary (with the map, when it fits): each CTA copies the
    // distinct blocks and its explicit rows' block indices into shared
    // memory, and explicit rows then read nothing from global memory but the
    // product input's halo.  NULL: packed rows or planes.
    const uint16_t* dict_idx;  // [nnzb] dictionary index of each stored block
    const void* dictM;         // [n_dict * 9] distinct blocks in the inner precision
    int n_dict;
    int* rep_status;
    int* rep_iters;
    int* rep_outer;
    double* rep_rel;
    unsigned long long* trace;  // optional [n_cta][kTraceIters][kTracePhases] timestamps
    unsigned long long timeout_ns;
    unsigned spin_ns;           // back-off between polls of the barrier generation
    int expand;                 // p^T A p of every iteration as u^T w + 2 beta u^T s + beta^2 p^T s (u^T s and
                                // p^T s taken in the update), not from the Chronopoulos-Gear recurrence
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
// Grid barrier with fused reduction.  Every CTA writes NV partial values,
// then one thread per CTA fences and arrives on a counter that only grows
// within a launch (barrier e of the launch completes when it reaches
// (e + 1) * n_cta).  After the wait, every CTA sums the partials of all CTAs
// itself, in CTA order (lane-strided, then a fixed butterfly), so all CTAs
// obtain bitwise the same results without a second round trip through a
// CTA that reduces and publishes.  Partials alternate between two buffers
// by barrier parity: a CTA can only write barrier e + 2's partials after
// every CTA has arrived at barrier e + 1, that is after every CTA has read
// barrier e's.  The CTA barrier before the fence makes the whole CTA's
// writes part of its release (fences are cumulative).  Waits are bounded by
// P.timeout_ns; on expiry the CTA records kDevTimeout and every CTA leaves
// at its next barrier.
// ---------------------------------------------------------------------------
static __shared__ unsigned g_bar_epoch;  // barriers this CTA has passed in this launch

// Arrival with release semantics at GPU scope (orders the CTA's earlier
// writes, which the preceding CTA barrier made this thread's, before it) and
// the matching acquire load of the counter.
__device__ __forceinline__ void arrive_release(unsigned* count) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(count), "r"(1u) : "memory");
}
__device__ __forceinline__ unsigned load_acquire(const unsigned* count) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
    return v;
}


__device__ __forceinline__ void grid_barrier_init() {
    if (threadIdx.x == 0) g_bar_epoch = 0u;
}

// kPair: s_in and s_out hold FP32 pairs (a float2 (h, l) in each 8-byte
// slot), and the partials travel and are summed as pairs (TwoSum additions)
// on the FP32 pipes.  On this GPU one FP64 instruction of a warp takes about
// 64 cycles, so sums that every CTA repeats are kept off the FP64 pipe.
template <int NV, bool kPair = false>
__device__ __noinline__ bool grid_reduce(const SolveParams& P, int cta, const double* s_in, double* s_out) {
    __shared__ int s_ok;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned ep = g_bar_epoch;
    double* part = P.partial + (size_t)(ep & 1u) * (size_t)P.part_half;
    for (int v = threadIdx.x; v < NV; v += kThreads) {
        if (kPair) {
            ((float2*)part)[(size_t)cta * NV + v] = ((const float2*)s_in)[v];
        } else {
            part[(size_t)cta * NV + v] = s_in[v];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int* verr = &P.sync->err;
        arrive_release(&P.sync->count);
        const unsigned target = (ep + 1u) * (unsigned)P.n_cta;
        int ok = 1;
        if ((int)(load_acquire(&P.sync->count) - target) < 0) {
            const unsigned long long t0 = globaltimer_ns();
            while ((int)(load_acquire(&P.sync->count) - target) < 0) {
                if (*verr) {
                    ok = 0;
                    break;
                }
                if (globaltimer_ns() - t0 > P.timeout_ns) {
                    atomicCAS(&P.sync->err, 0, kDevTimeout);
                    ok = 0;
                    break;
                }
                if (P.spin_ns) __nanosleep(P.spin_ns);
            }
        }
        s_ok = ok && *verr == 0;
        g_bar_epoch = ep + 1u;
    }
    __syncthreads();
    if (NV > 0 && s_ok) {
        for (int v = warp; v < NV; v += kWarps) {
            if (kPair) {
                float h = 0.f, l = 0.f;
                for (int c = lane; c < P.n_cta; c += 32) {
                    const float2 q = __ldcg((const float2*)part + (size_t)c * NV + v);
                    df_add(h, l, q.x, q.y);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
                    df_add(h, l, h2, l2);
                }
                if (lane == 0) {
                    df_norm(h, l);
                    ((float2*)s_out)[v] = make_float2(h, l);
                }
            } else {
                double acc = 0.0;
                for (int c = lane; c < P.n_cta; c += 32) acc += __ldcg(part + (size_t)c * NV + v);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) s_out[v] = acc;
            }
        }
        __syncthreads();
    }
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

// The same for FP32-pair values (f[2k] + f[2k + 1] is value k), with TwoSum
// additions; only the NV * R CTA totals are converted to FP64.
template <int R, int NV>
__device__ __forceinline__ void cta_colsum_df(const float (&f)[2 * NV], double* s_red, double* s_in) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2* s_redf = (float2*)s_red;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        float h = f[2 * k], l = f[2 * k + 1];
#pragma unroll
        for (int o = 16; o >= R; o >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
            df_add(h, l, h2, l2);
        }
        if (lane < R) s_redf[(k * kWarps + warp) * R + lane] = make_float2(h, l);
    }
    __syncthreads();
    for (int i = warp; i < NV * R; i += kWarps) {
        const int k = i / R, c = i % R;
        const float2 q = s_redf[(k * kWarps + lane) * R + c];  // kWarps == 32
        float h = q.x, l = q.y;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
            df_add(h, l, h2, l2);
        }
        if (lane == 0) {
            df_norm(h, l);
            ((float2*)s_in)[i] = make_float2(h, l);  // a pair, read as such by grid_reduce<NV, true>
        }
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

// ---------------------------------------------------------------------------
// Resident product map of an R = 1 launch.  Products cost very different
// amounts per row (an explicit row walks up to 27 stored 3x3 blocks, a
// diagonal-stencil row 27 real weights), and a warp lasts as long as its
// slowest lane; rows are therefore sorted by cost (explicit rows by block
// count, then general-stencil rows, then diagonal-stencil rows) so that a
// warp's ten rows cost alike, and the costly row groups spread over the
// CTA's warps and the SM's four schedulers.  The sort, the block ranges and
// the column map are built once per launch.  The halo of the product input
// is staged as up to three byte ranges (lexicographic node ranks put a
// row's neighbours one plane below, in its own plane and one plane above),
// which for the voxel grids here is about a third of the single window
// from the lowest to the highest neighbour.
// ---------------------------------------------------------------------------
struct ResMap {
    int n;                 // rows of the CTA's product range
    int nslot;             // sorted slots: explicit rows, padding to a multiple of 10, class rows
    int nexpl;             // explicit slots including their padding (row -1)
    long long pk_base;     // first entry of the CTA's packed explicit rows
    int staged;            // the segments fit the halo buffer
    int nseg;              // byte ranges staged per product
    unsigned total;        // their total bytes
    long long a0[3];       // first global byte of each range (16-byte aligned)
    unsigned bytes[3];     // its length (a multiple of 16)
    unsigned soff[3];      // its offset in the halo buffer
    int lo[3], hi[3];      // the node (column) range it covers
};

template <typename C>
__device__ __noinline__ void build_res_map(const SolveParams& P, int pr0, int pr1, int* rows, int2* meta, int* cols,
                                           int* goff, uint16_t* bidx, C* dict, ResMap& rm) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = pr1 - pr0;
    int* keys = cols;  // scratch until the column map is written
    __shared__ int s_lo[3], s_hi[3];
    for (int i = tid; i < n; i += kThreads) {
        const int row = pr0 + i;
        const int cls = P.row_class ? P.row_class[row] : -1;
        const int kind = cls >= 0 ? P.stencil->kind[cls] : 0;
        const int nb = P.rp[row + 1] - P.rp[row];
        // with the dictionary, general-stencil rows are read like explicit
        // ones (their blocks are in it too)
        keys[i] = kind == 2 ? 21 : ((kind == 1 && !bidx) ? 20 : max(0, min(19, 27 - nb)));
    }
    if (tid < 3) {
        s_lo[tid] = 0x7fffffff;
        s_hi[tid] = -1;
    }
    __syncthreads();
    // stable counting sort by key (one warp; deterministic); the explicit
    // rows are padded with empty slots (row -1) to a multiple of kExplRows,
    // so that every warp group holds rows of one kind
    if (warp == 0) {
        int base = 0;
        for (int b = 0; b < 22; ++b) {
            if (b == 20) {
                const int pad = (base + kExplRows - 1) / kExplRows * kExplRows;
                for (int i = base + lane; i < pad; i += 32) rows[i] = -1;
                if (lane == 0) rm.nexpl = pad;
                base = pad;
            }
            for (int c0 = 0; c0 < n; c0 += 32) {
                const int i = c0 + lane;
                const bool m = i < n && keys[i] == b;
                const unsigned bal = __ballot_sync(0xffffffffu, m);
                if (m) rows[base + __popc(bal & ((1u << lane) - 1u))] = pr0 + i;
                base += __popc(bal);
            }
        }
        if (lane == 0) rm.nslot = base;
    }
    __syncthreads();
    const int nslot = rm.nslot;
    // block ranges; column bounds of the three neighbour groups
    for (int i = warp; i < nslot; i += kWarps) {
        const int row = rows[i];
        if (row < 0) {
            if (lane == 0) meta[i] = make_int2(0, 0);
            continue;
        }
        const int s0 = __ldg(P.rp + row), nb = __ldg(P.rp + row + 1) - s0;
        if (lane == 0) {
            const int cls = P.row_class ? P.row_class[row] : -1;
            const int kind = cls >= 0 ? P.stencil->kind[cls] : 0;
            meta[i] = make_int2(s0, nb | (kind << 8) | ((cls & 0xff) << 16));
        }
        if (lane < nb) {
            const int c = __ldg(P.col + s0 + lane);
            const int d = c - row;
            const int g = d < -P.res_tmid ? 0 : (d > P.res_tmid ? 2 : 1);
            atomicMin(&s_lo[g], c);
            atomicMax(&s_hi[g], c);
        }
    }
    __syncthreads();
    if (tid == 0) {
        // packed explicit rows: offsets of the warp groups (entries)
        int acc = 0;
        for (int g = 0; g * kExplRows < rm.nexpl; ++g) {
            goff[g] = acc;
            for (int j = 0; j < kExplRows; ++j) acc += 9 * (meta[g * kExplRows + j].y & 0xff);
        }
        rm.pk_base = P.expl_prefix ? 9ll * P.expl_prefix[pr0] : 0ll;
        // non-empty ranges in ascending order, merged where they overlap or
        // nearly touch
        int lo[3], hi[3], m = 0;
        for (int g = 0; g < 3; ++g)
            if (s_hi[g] >= 0) {
                lo[m] = s_lo[g];
                hi[m] = s_hi[g];
                ++m;
            }
        for (int a = 0; a < m; ++a)
            for (int b = a + 1; b < m; ++b)
                if (lo[b] < lo[a]) {
                    const int tl = lo[a], th = hi[a];
                    lo[a] = lo[b];
                    hi[a] = hi[b];
                    lo[b] = tl;
                    hi[b] = th;
                }
        int k = 0;
        for (int a = 0; a < m; ++a) {
            if (k > 0 && lo[a] <= rm.hi[k - 1] + 8) {
                rm.hi[k - 1] = max(rm.hi[k - 1], hi[a]);
            } else {
                rm.lo[k] = lo[a];
                rm.hi[k] = hi[a];
                ++k;
            }
        }
        unsigned off = 0;
        for (int a = 0; a < k; ++a) {
            const long long b0 = 3ll * rm.lo[a] * (long long)sizeof(C), b1 = 3ll * (rm.hi[a] + 1) * (long long)sizeof(C);
            const long long a0 = b0 & ~15ll, a1 = (b1 + 15) & ~15ll;
            rm.a0[a] = a0;
            rm.bytes[a] = (unsigned)(a1 - a0);
            rm.soff[a] = off;
            off += (unsigned)(a1 - a0);
        }
        rm.nseg = k;
        rm.total = off;
        rm.n = n;
        rm.staged = (P.stage && k > 0 && (long long)off <= P.halo_bytes) ? 1 : 0;
    }
    __syncthreads();
    // column map: the position of the column's first vector entry in the
    // halo buffer (staged) or in the global vector
    for (int i = warp; i < nslot; i += kWarps) {
        const int2 mt = meta[i];
        const int nb = mt.y & 0xff;
        if (lane < nb) {
            const int c = __ldg(P.col + mt.x + lane);
            int e = 3 * c;
            if (rm.staged) {
                int a = 0;
                while (a + 1 < rm.nseg && c > rm.hi[a]) ++a;
                e = (int)(((long long)rm.soff[a] + 3ll * c * (long long)sizeof(C) - rm.a0[a]) / (long long)sizeof(C));
            }
            cols[i * 27 + lane] = e;
            if (bidx) bidx[i * 27 + lane] = __ldg(P.dict_idx + mt.x + lane);
        }
    }
    if (dict)
        for (int i = tid; i < 9 * P.n_dict; i += kThreads) dict[i] = __ldg((const C*)P.dictM + i);
    __syncthreads();
}

// Packs the values of the CTA's explicit rows for the product: in warp group
// g (kExplRows slots, rows sorted by block count, most first), step k takes
// the k-th block of the J_k rows that have one, stored as
// [beta][row j][alpha], so that entry (alpha, beta) of row j sits at
// beta * 3 J_k + 3j + alpha.  No entry is padding.  Values come from the
// planes (read-only); the product phase reads them back in the same launch
// through L2.
template <typename C>
__device__ __noinline__ void pack_explicit(const SolveParams& P, const int* rows, const int2* meta, const int* goff,
                                           const ResMap& rm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const C* valM = (const C*)P.valM;
    C* pk = (C*)P.pk + rm.pk_base;
    const int j = lane / 3, al = lane % 3;
    for (int g = warp; g * kExplRows < rm.nexpl; g += kWarps) {
        const int slot = g * kExplRows + j;
        const bool valid = lane < 3 * kExplRows && rows[slot] >= 0;
        const int2 mt = valid ? meta[slot] : make_int2(0, 0);
        const int nb = mt.y & 0xff;
        const int K = __shfl_sync(0xffffffffu, nb, 0);
        C* pg = pk + goff[g];
        int off = 0;
        for (int k = 0; k < K; ++k) {
            const int Jk = __popc(__ballot_sync(0xffffffffu, al == 0 && valid && k < nb));
            if (k < nb) {
#pragma unroll
                for (int be = 0; be < 3; ++be)
                    pg[off + be * 3 * Jk + 3 * j + al] = ld_ro(valM + (3 * al + be) * P.stride + mt.x + k);
            }
            off += 9 * Jk;
        }
    }
}

// Stages the map's byte ranges of v into the halo buffer with bulk (TMA)
// copies on one mbarrier.  Returns false when the bounded wait expired.
__device__ __forceinline__ bool stage_res(const SolveParams& P, const void* v, const ResMap& rm, char* halo_buf,
                                          uint64_t* mbar, unsigned& phase) {
    if (threadIdx.x == 0) {
        fence_proxy_async();
        mbar_expect_tx(mbar, rm.total);
        for (int a = 0; a < rm.nseg; ++a) bulk_g2s(halo_buf + rm.soff[a], (const char*)v + rm.a0[a], rm.bytes[a], mbar);
    }
    const bool ok = __syncthreads_and(mbar_wait_bounded(mbar, phase & 1u, P.timeout_ns)) != 0;
    if (!ok) {
        atomicCAS(&P.sync->err, 0, kDevTimeout);
        mbar_wait_bounded(mbar, phase & 1u, P.timeout_ns > 2000000000ull ? P.timeout_ns : 2000000000ull);
    }
    phase += 1;
    return ok;
}

// Views of the resident map in shared memory.
struct ResView {
    const int* rows;
    const int2* meta;
    const int* cols;
    const int* goff;  // packed entries before each explicit warp group
    const float2* dvw;  // diagonal-stencil weights [class][alpha][27] in shared memory (FP32 pair, or .x alone)
    const uint16_t* bidx;  // per slot, 27 dictionary indices of its blocks (shared memory; NULL: no dictionary)
    const void* dict;      // the dictionary in shared memory
    const ResMap* rm;
    unsigned long long* wtrace;  // diagnostics: per-warp stamps of one traced iteration (or NULL)
};

// Component alpha of a diagonal-stencil row (27 real weights, shared
// memory) times the vector; cols holds element indices.
template <typename C, bool kShared>
__device__ __forceinline__ C row_component_diag(const float2* dv, const int* cols, int al, const C* xs) {
    const float2* d = dv + al * 27;
  if constexpr (std::is_same<C, float4>::value) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 9
    for (int kk = 0; kk < 27; ++kk) {
        const int xi = cols[kk] + al;
        const float4 xv = kShared ? xs[xi] : ld_cg(xs + xi);
        const float2 dk = d[kk];
        df_mac(acc[0], acc[1], dk.x, dk.y, xv.x, xv.z);
        df_mac(acc[2], acc[3], dk.x, dk.y, xv.y, xv.w);
    }
    return df_result(acc);
  } else {
    using Tr = decltype(C{}.x);
    Tr ar = 0, ai = 0;
#pragma unroll 9
    for (int kk = 0; kk < 27; ++kk) {
        const int xi = cols[kk] + al;
        const C xv = kShared ? xs[xi] : ld_cg(xs + xi);
        const Tr dk = (Tr)d[kk].x;
        ar += dk * xv.x;
        ai += dk * xv.y;
    }
    return mk(ar, ai);
  }
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
                                              double (&acc)[NV], float (&facc)[2 * NV], const ResView* rv) {
    constexpr bool kRefresh = NV == 11;
    // FP32-pair vectors: dots accumulate as FP32 pairs in facc (facc[2k] +
    // facc[2k+1] is dot k), summed over the CTA as pairs as well
    constexpr bool kDFV = std::is_same<TM, DFloat>::value;
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
    if (R == 1 && kClassPath<C> && rv != nullptr) {
        // resident map: ten rows of like cost per warp (sorted slots); row
        // groups go to warps in snake order, so a warp that takes two groups
        // pairs a costly one with a cheap one
        const bool refresh = kRefresh && s_refresh[0] != 0;
        const int al = lane % 3;
        const int n = rv->rm->nslot;
        const int nexpl = rv->rm->nexpl;
        const int n_eg = nexpl / kExplRows;  // explicit groups (kExplRows rows), then class groups (ten rows)
        const int n_groups = n_eg + (n - nexpl + kRowsPerWarpR1 - 1) / kRowsPerWarpR1;
        const bool packed = P.pk != nullptr;
        int n_eg_done = 0, n_cg_done = 0;
        for (int k = 0; k * kWarps < n_groups; ++k) {
            const int g = k * kWarps + ((k & 1) ? kWarps - 1 - warp : warp);
            if (g >= n_groups) continue;
            if (g < n_eg) ++n_eg_done;
            else ++n_cg_done;
            if (g < n_eg && rv->bidx) {
                // explicit rows through the block dictionary: lane 3j + alpha
                // walks the blocks of row j, component alpha, reading the
                // block's index, its three entries and the three vector
                // entries from shared memory
                const int j = lane / 3;
                const int slot = g * kExplRows + j;
                const bool valid = lane < 3 * kExplRows && rv->rows[slot] >= 0;
                const int2 mt = valid ? rv->meta[slot] : make_int2(0, 0);
                const int nb = mt.y & 0xff;
                const int* rc = rv->cols + slot * 27;
                const uint16_t* rb = rv->bidx + slot * 27;
                const C* dct = (const C*)rv->dict + 3 * al;
                const C* xv = kStaged ? xs : uM;
                C y;
                if constexpr (std::is_same<C, float4>::value) {
                    float a4[4] = {0.f, 0.f, 0.f, 0.f};
                    for (int kk = 0; kk < nb; ++kk) {
                        const int e = rc[kk];
                        const C* m = dct + 9 * (int)rb[kk];
                        dfc_mac(a4, m[0], kStaged ? xv[e] : ld_cg(xv + e));
                        dfc_mac(a4, m[1], kStaged ? xv[e + 1] : ld_cg(xv + e + 1));
                        dfc_mac(a4, m[2], kStaged ? xv[e + 2] : ld_cg(xv + e + 2));
                    }
                    y = df_result(a4);
                } else {
                    using Tr = decltype(C{}.x);
                    Tr ar = 0, ai = 0;
                    for (int kk = 0; kk < nb; ++kk) {
                        const int e = rc[kk];
                        const C* m = dct + 9 * (int)rb[kk];
                        const C m0 = m[0], m1 = m[1], m2 = m[2];
                        const C x0 = kStaged ? xv[e] : ld_cg(xv + e), x1 = kStaged ? xv[e + 1] : ld_cg(xv + e + 1),
                                x2 = kStaged ? xv[e + 2] : ld_cg(xv + e + 2);
                        ar += m0.x * x0.x - m0.y * x0.y + m1.x * x1.x - m1.y * x1.y + m2.x * x2.x - m2.y * x2.y;
                        ai += m0.x * x0.y + m0.y * x0.x + m1.x * x1.y + m1.y * x1.x + m2.x * x2.y + m2.y * x2.x;
                    }
                    y = mk(ar, ai);
                }
                if (valid) {
                    const int row = rv->rows[slot];
                    const size_t o = (size_t)3 * row + al;
                    w[o] = y;
                    C sy = y;
                    if (refresh) sy = row_component<C, false>(valM, P.stride, P.col + mt.x, mt.x, mt.x + nb, al, pM, 0);
                    dots(o, y, refresh, sy);
                }
                continue;
            }
            if (g < n_eg && packed) {
                // explicit rows from the packed copy: lane 3j + alpha walks the
                // blocks of row j, component alpha; each step loads 3 J_k
                // consecutive entries per block column
                const int j = lane / 3;
                const int slot = g * kExplRows + j;
                const bool valid = lane < 3 * kExplRows && rv->rows[slot] >= 0;
                const int2 mt = valid ? rv->meta[slot] : make_int2(0, 0);
                const int nb = mt.y & 0xff;
                const int K = __shfl_sync(0xffffffffu, nb, 0);
                const C* pg = (const C*)P.pk + rv->rm->pk_base + rv->goff[g];
                const int* rc = rv->cols + slot * 27;
                const C* xv = kStaged ? xs : uM;
                const bool lead = al == 0 && valid;  // one lane per row counts the rows of a step
                int off = 0;
                C y;
                if constexpr (std::is_same<C, float4>::value) {
                    float a4[4] = {0.f, 0.f, 0.f, 0.f};
                    for (int kk = 0; kk < K; ++kk) {
                        const int Jk = __popc(__ballot_sync(0xffffffffu, lead && kk < nb));
                        if (kk < nb) {
                            const int e = rc[kk];
                            const C* pe = pg + off + 3 * j + al;
                            const C m0 = ld_cg(pe), m1 = ld_cg(pe + 3 * Jk), m2 = ld_cg(pe + 6 * Jk);
                            const C x0 = kStaged ? xv[e] : ld_cg(xv + e), x1 = kStaged ? xv[e + 1] : ld_cg(xv + e + 1),
                                    x2 = kStaged ? xv[e + 2] : ld_cg(xv + e + 2);
                            dfc_mac(a4, m0, x0);
                            dfc_mac(a4, m1, x1);
                            dfc_mac(a4, m2, x2);
                        }
                        off += 9 * Jk;
                    }
                    y = df_result(a4);
                } else {
                    using Tr = decltype(C{}.x);
                    Tr ar = 0, ai = 0;
                    for (int kk = 0; kk < K; ++kk) {
                        const int Jk = __popc(__ballot_sync(0xffffffffu, lead && kk < nb));
                        if (kk < nb) {
                            const int e = rc[kk];
                            const C* pe = pg + off + 3 * j + al;
                            const C m0 = ld_cg(pe), m1 = ld_cg(pe + 3 * Jk), m2 = ld_cg(pe + 6 * Jk);
                            const C x0 = kStaged ? xv[e] : ld_cg(xv + e), x1 = kStaged ? xv[e + 1] : ld_cg(xv + e + 1),
                                    x2 = kStaged ? xv[e + 2] : ld_cg(xv + e + 2);
                            ar += m0.x * x0.x - m0.y * x0.y + m1.x * x1.x - m1.y * x1.y + m2.x * x2.x - m2.y * x2.y;
                            ai += m0.x * x0.y + m0.y * x0.x + m1.x * x1.y + m1.y * x1.x + m2.x * x2.y + m2.y * x2.x;
                        }
                        off += 9 * Jk;
                    }
                    y = mk(ar, ai);
                }
                if (valid) {
                    const int row = rv->rows[slot];
                    const size_t o = (size_t)3 * row + al;
                    w[o] = y;
                    C sy = y;
                    if (refresh) sy = row_component<C, false>(valM, P.stride, P.col + mt.x, mt.x, mt.x + nb, al, pM, 0);
                    dots(o, y, refresh, sy);
                }
                continue;
            }
            // class rows (ten per warp), or explicit rows read from the planes
            // when no packed copy exists (kExplRows per warp)
            const int slot = g < n_eg ? g * kExplRows + lane / 3 : nexpl + (g - n_eg) * kRowsPerWarpR1 + lane / 3;
            const int lanes = g < n_eg ? 3 * kExplRows : 3 * kRowsPerWarpR1;
            if (lane < lanes && slot < n && rv->rows[slot] >= 0) {
                const int2 mt = rv->meta[slot];
                const int row = rv->rows[slot];
                const int s0 = mt.x, s1 = mt.x + (mt.y & 0xff);
                const int kind = (mt.y >> 8) & 0xff;
                const int cls = (int)(signed char)((mt.y >> 16) & 0xff);
                const int* rc = rv->cols + slot * 27;
                const C y = kind == 2 ? row_component_diag<C, kStaged>(rv->dvw + cls * 81, rc, al, kStaged ? xs : uM)
                            : kind ? row_component_class<C, kStaged, true>(P.stencil, cls, kind, rc, al, kStaged ? xs : uM, 0)
                                   : row_component<C, kStaged, true>(valM, P.stride, rc, s0, s1, al, kStaged ? xs : uM, 0);
                const size_t o = (size_t)3 * row + al;
                w[o] = y;
                C sy = y;
                if (refresh)
                    sy = kind ? row_component_class<C, false>(P.stencil, cls, kind, P.col + s0, al, pM, 0)
                              : row_component<C, false>(valM, P.stride, P.col + s0, s0, s1, al, pM, 0);
                dots(o, y, refresh, sy);
            }
        }
        if (rv->wtrace && lane == 0) {
            rv->wtrace[warp] = globaltimer_ns();
            rv->wtrace[kWarps + warp] = (unsigned long long)(1000 * n_eg_done + n_cg_done);
        }
    } else if (R == 1) {
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
    (void)any_refresh;
    return ok;
}

// Diagnostics (FE_TRACE=1): every CTA stamps the end of each phase of its
// first kTraceIters iterations, [cta][iteration][phase]; after those stamps
// come kTraceStats values per CTA describing its product rows.
constexpr int kTraceStats = 8 + 2 * kWarps;  // row counts, then per warp the end of its product rows and its groups
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
                                             bool any_refresh, int* s_cols, double (&acc)[NV],
                                             float (&facc)[2 * NV], int trace_it, const ResView* rv) {
    using C = typename CplxT<TM>::type;
    const int tid = threadIdx.x;
    bool ok;
    if (rv != nullptr) {
        if (rv->rm->staged) {
            if (!stage_res(P, uM, *rv->rm, halo_buf, mbar, mbar_phase)) return false;
            FE_TRACE_MARK(1);
            ok = product_phase<TM, R, true, NV>(P, (const C*)halo_buf, 0, pr0, pr1, s_refresh, any_refresh, s_cols,
                                                acc, facc, rv);
        } else {
            ok = product_phase<TM, R, false, NV>(P, nullptr, 0, pr0, pr1, s_refresh, any_refresh, s_cols, acc, facc,
                                                 rv);
        }
    } else if (stage_fits) {
        int shift = 0;
        if (!stage_halo<C, R>(P, uM, pr0, pr1, halo_buf, mbar, mbar_phase, shift)) return false;
        FE_TRACE_MARK(1);
        ok = product_phase<TM, R, true, NV>(P, (const C*)halo_buf, shift, pr0, pr1, s_refresh, any_refresh, s_cols,
                                            acc, facc, nullptr);
    } else {
        ok = product_phase<TM, R, false, NV>(P, nullptr, 0, pr0, pr1, s_refresh, any_refresh, s_cols, acc, facc,
                                             nullptr);
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
    // Krylov vectors: FP64, or FP32 pairs in the FE_PREC_DF mode (then the
    // products read u and p directly, and the updates, dots and reductions
    // run on the FP32 pipes: a warp's FP64 instruction holds the SM's FP64
    // pipe for about 16 cycles on this GPU, so FP64 vector work that every
    // thread repeats costs microseconds per iteration)
    constexpr bool kDFV = std::is_same<TM, DFloat>::value;
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
    // shared memory: [column sums][column staging][halo], or with the
    // resident map [column sums][map][halo], where the true-residual phase
    // stages its column indices at the start of the halo buffer (no bulk copy
    // is in flight outside the product phases)
    char* halo_buf = dyn + P.red_bytes + P.col_bytes + P.res_bytes;
    int* s_cols = P.res ? (int*)halo_buf : (int*)(dyn + P.red_bytes);
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ double s_in[kMaxNV * R], s_out[kMaxNV * R];
    __shared__ double s_bn[R], s_rr_ref[R], s_rel[R];
    __shared__ double s_gam_r[R], s_gam_i[R], s_al_r[R], s_al_i[R], s_be_r[R], s_be_i[R];
    __shared__ double s_igam_r[R], s_igam_i[R], s_ial_r[R], s_ial_i[R];  // 1/gamma, 1/alpha of the last iteration
    __shared__ float4 s_a4[R], s_na4[R], s_b4[R];  // alpha, -alpha, beta as FP32 pairs (FP32-pair updates)
    // FP32-pair solves keep gamma, 1/gamma and 1/alpha of the last iteration as
    // FP32 pairs, and 1/||b||^2 and 1/rr_ref in FP32 for the convergence tests
    // (s_scl_ok: both are normal FP32 numbers)
    __shared__ float4 s_gam4[kDFV ? R : 1], s_igam4[kDFV ? R : 1], s_ial4[kDFV ? R : 1];
    __shared__ float s_ibn2f[kDFV ? R : 1], s_irrf[kDFV ? R : 1];
    __shared__ int s_scl_ok[kDFV ? R : 1];
    // the expanded recurrence: u^T s and p^T s of the last update (u, p, s as
    // the update left them), summed over the grid at the barrier that ends it
    // (FP32 pairs in the 8-byte slots for FP32-pair solves)
    __shared__ double s_xd[4 * R];
    // FP32 forms of 1/||b||^2 and 1/rr_ref, set whenever those change (rare)
    auto set_scales = [&](int c) {
        if constexpr (kDFV) {
            const double b2 = s_bn[c] * s_bn[c];
            const double ib = b2 > 0.0 ? 1.0 / b2 : 0.0, ir = s_rr_ref[c] > 0.0 ? 1.0 / s_rr_ref[c] : 0.0;
            s_ibn2f[c] = (float)ib;
            s_irrf[c] = (float)ir;
            s_scl_ok[c] = ib > 1.0e-37 && ib < 1.0e37 && ir > 1.0e-37 && ir < 1.0e37;
        }
    };
    const float tol2f = (float)(P.tol * P.tol), rel2f = (float)(P.reliable * P.reliable);
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
    const bool stage_fits = P.stage && !P.res && [&] {
        const int h0 = max(0, pr0 - P.halo), h1 = min(P.n_rows, pr1 + P.halo);
        const size_t a0 = ((size_t)3 * h0 * R * sizeof(C)) & ~(size_t)15;
        const size_t a1 = ((size_t)3 * h1 * R * sizeof(C) + 15) & ~(size_t)15;
        return a1 - a0 <= (size_t)P.halo_bytes;
    }();
    // resident product map (R = 1 class-path products, when the host sized it)
    constexpr bool kRes = kClassPath<TM> && R == 1;
    __shared__ ResMap s_rm;
    __shared__ float2 s_dvw[kRes ? kMaxClasses * 81 : 1];
    ResView rv_local{nullptr, nullptr, nullptr, nullptr, s_dvw, nullptr, nullptr, &s_rm, nullptr};
    const ResView* rv = nullptr;
    if constexpr (kRes) {
        if (P.res && pr1 - pr0 + kRowsPerWarpR1 <= P.res_rows_max) {
            int* rrows = (int*)(dyn + P.red_bytes);
            int2* rmeta = (int2*)(rrows + P.res_rows_max);
            int* rcols = (int*)(rmeta + P.res_rows_max);
            int* rgoff = rcols + 27 * P.res_rows_max;
            uint16_t* rbidx = P.dictM ? (uint16_t*)(rgoff + (P.res_rows_max / kExplRows + 2)) : nullptr;
            C* rdict = P.dictM ? (C*)(((uintptr_t)(rbidx + 27 * P.res_rows_max) + 15) & ~(uintptr_t)15) : nullptr;
            for (int i = tid; i < kMaxClasses * 81; i += kThreads) {
                if constexpr (std::is_same<C, float4>::value) s_dvw[i] = (&P.stencil->dvaldf[0][0][0])[i];
                else s_dvw[i] = make_float2((&P.stencil->dval32[0][0][0])[i], 0.f);
            }
            build_res_map<C>(P, pr0, pr1, rrows, rmeta, rcols, rgoff, rbidx, rdict, s_rm);
            rv_local.bidx = rbidx;
            rv_local.dict = rdict;
            if (P.pk && !P.dictM) {
                pack_explicit<C>(P, rrows, rmeta, rgoff, s_rm);
                __syncthreads();
            }
            rv_local.rows = rrows;
            rv_local.meta = rmeta;
            rv_local.cols = rcols;
            rv_local.goff = rgoff;
            rv = &rv_local;
        }
    }
    const int n_items = (r1 - r0) * R;  // (node, column) pairs owned by this CTA
    const int my_c = tid % R;           // column of every item this thread handles
    const size_t base_o = (size_t)3 * r0 * R;
    unsigned mbar_phase = 0;
    int trace_it = 0;

    if (tid == 0) mbar_init(&s_mbar, 1);
    grid_barrier_init();
    int seg_it = 0;
    bool seg_end = false;
    const unsigned long long seg_t0 = (P.state && cta == 0 && tid == 0) ? globaltimer_ns() : 0ull;
    const bool resume = P.state && __ldcg(&P.state->started);
    if (resume) {
        if (tid < R) {
            const ColState& cs = P.state->col[tid];
            s_bn[tid] = cs.bn;
            s_rr_ref[tid] = cs.rr_ref;
            s_rel[tid] = cs.rel;
            s_gam_r[tid] = cs.gam_r;
            s_gam_i[tid] = cs.gam_i;
            s_al_r[tid] = cs.al_r;
            s_al_i[tid] = cs.al_i;
            s_be_r[tid] = cs.be_r;
            s_be_i[tid] = cs.be_i;
            s_igam_r[tid] = cs.igam_r;
            s_igam_i[tid] = cs.igam_i;
            s_ial_r[tid] = cs.ial_r;
            s_ial_i[tid] = cs.ial_i;
            s_a4[tid] = cs.a4;
            s_na4[tid] = cs.na4;
            s_b4[tid] = cs.b4;
            if constexpr (kDFV) {
                s_gam4[tid] = cs.gam4;
                s_igam4[tid] = cs.igam4;
                s_ial4[tid] = cs.ial4;
                set_scales(tid);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) s_xd[k * R + tid] = __longlong_as_double(cs.xd[k]);
            s_active[tid] = cs.active;
            s_done[tid] = cs.done;
            s_status[tid] = cs.status;
            s_iters[tid] = cs.iters;
            s_outer[tid] = cs.outer;
            s_first[tid] = cs.first;
            s_refresh[tid] = cs.refresh;
            s_repl[tid] = cs.repl;
            s_pass_it[tid] = cs.pass_it;
        }
        if (tid == 0) {
            s_any_repl = P.state->any_repl;
            s_any_refresh = P.state->any_refresh;
        }
        __syncthreads();
    } else {
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
    }

    for (;;) {
        // a segmented solve saves its state here, where every CTA has
        // finished the last iteration (or the replacement request before it)
        if (P.seg_iters > 0 && seg_it >= P.seg_iters) {
            seg_end = true;
            break;
        }
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
                        set_scales(c);
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
        // The CTA's last warp (the lightest product rows come last) takes the
        // reciprocals the next scalars need: 1/gamma = conj(gamma) / |gamma|^2
        // and 1/alpha = conj(alpha) / |alpha|^2 of the last iteration.
        if (tid >= kThreads - R) {
            const int c = kThreads - 1 - tid;
            if constexpr (kDFV) {  // the same in FP32-pair arithmetic
                if (s_active[c] && !s_first[c]) {
                    const DZ one = {make_float2(1.f, 0.f), make_float2(0.f, 0.f)};
                    s_igam4[c] = dz_f4(dz_div(one, dz_of(s_gam4[c])));
                    s_ial4[c] = dz_f4(dz_div(one, dz_of(s_a4[c])));
                }
            } else if (s_active[c] && !s_first[c]) {
                const double ig = rcp64(s_gam_r[c] * s_gam_r[c] + s_gam_i[c] * s_gam_i[c]);
                const double ia = rcp64(s_al_r[c] * s_al_r[c] + s_al_i[c] * s_al_i[c]);
                s_igam_r[c] = s_gam_r[c] * ig;
                s_igam_i[c] = -s_gam_i[c] * ig;
                s_ial_r[c] = s_al_r[c] * ia;
                s_ial_i[c] = -s_al_i[c] * ia;
            }
        }
        FE_TRACE_MARK(0);
        if (rv) rv_local.wtrace = (P.trace && trace_it == 20)
                                      ? P.trace + (size_t)P.n_cta * kTraceIters * kTracePhases + (size_t)cta * kTraceStats + 8
                                      : nullptr;
        if (s_any_refresh) {
            double acc[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
            float facc[22] = {};
            if (!product_step<TM, R, 11>(P, cta, stage_fits, uM, pr0, pr1, halo_buf, &s_mbar, mbar_phase, s_refresh,
                                         s_any_refresh, s_cols, acc, facc, trace_it, rv))
                goto out;
            FE_TRACE_MARK(2);
            if constexpr (kDFV) cta_colsum_df<R, 11>(facc, s_red, s_in);
            else cta_colsum<R, 11>(acc, s_red, s_in);
            FE_TRACE_MARK(3);
            if (!grid_reduce<11 * R, kDFV>(P, cta, s_in, s_out)) goto out;
        } else {
            double acc[5] = {0, 0, 0, 0, 0};
            float facc[10] = {};
            if (!product_step<TM, R, 5>(P, cta, stage_fits, uM, pr0, pr1, halo_buf, &s_mbar, mbar_phase, s_refresh,
                                        s_any_refresh, s_cols, acc, facc, trace_it, rv))
                goto out;
            FE_TRACE_MARK(2);
            if constexpr (kDFV) cta_colsum_df<R, 5>(facc, s_red, s_in);
            else cta_colsum<R, 5>(acc, s_red, s_in);
            FE_TRACE_MARK(3);
            if (!grid_reduce<5 * R, kDFV>(P, cta, s_in, s_out)) goto out;
        }
        FE_TRACE_MARK(4);
        // ---- [B] scalars ----
        // B1: does any column need its true residual first?  (No state of the
        // other columns changes in a replacement round: they redo the same
        // products next round.)
        if (tid < R) {
            const int c = tid;
            if (s_active[c]) {
                bool small, nan;
                if constexpr (kDFV) {  // |r|^2 as an FP32 pair; the tests scaled into FP32 range
                    const float2 q = ((const float2*)s_out)[4 * R + c];
                    const float rr = __fadd_rn(q.x, q.y);
                    nan = !(rr == rr);
                    if (s_scl_ok[c]) {
                        small = rr * s_ibn2f[c] <= tol2f || rr * s_irrf[c] < rel2f;
                    } else {
                        const double rd = (double)q.x + (double)q.y, tb = P.tol * s_bn[c];
                        small = rd <= tb * tb || rd < P.reliable * P.reliable * s_rr_ref[c];
                    }
                } else {
                    const double rr = s_out[4 * R + c];
                    const double tb = P.tol * s_bn[c];
                    small = rr <= tb * tb || rr < P.reliable * P.reliable * s_rr_ref[c];
                    nan = !(rr == rr);
                }
                const bool stalled = P.restart && P.max_pass > 0 && s_pass_it[c] >= P.max_pass;
                if (nan || s_iters[c] >= P.max_iter || (!s_first[c] && (small || stalled))) {
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
        // B2: Chronopoulos-Gear scalars (exact p^T A p after a replacement).
        // 1/gamma_old and 1/alpha_old come from the product phase (taken from
        // the gamma and the rounded alpha of the last iteration, the alpha
        // that updated x and r), so beta = gamma (1/gamma_old) and e = delta -
        // beta gamma (1/alpha_old) need no division: the one reciprocal on the
        // dependent chain is that of |e|^2.  FP64 operations of one thread
        // have a long latency on this GPU.
        if constexpr (kDFV) {  // the same recurrences in FP32-pair arithmetic
            if (tid < R) {
                const int c = tid;
                if (s_active[c]) {
                    const float2* so = (const float2*)s_out;
                    const float2 zero = make_float2(0.f, 0.f);
                    const DZ g = {so[c], so[R + c]}, d = {so[2 * R + c], so[3 * R + c]};
                    DZ b = {zero, zero}, e = d;
                    if (!s_first[c]) {
                        b = dz_mul(g, dz_of(s_igam4[c]));  // beta = gamma / gamma_old
                        if (s_refresh[c]) {
                            // p^T A p for p = u + beta p_old: u^T w + beta (u^T s + p^T w) + beta^2 p^T s
                            const DZ e12 = {dd_add(so[5 * R + c], so[7 * R + c]), dd_add(so[6 * R + c], so[8 * R + c])};
                            const DZ e3 = {so[9 * R + c], so[10 * R + c]};
                            e = dz_add(dz_add(d, dz_mul(b, e12)), dz_mul(dz_mul(b, b), e3));
                        } else if (P.expand) {
                            // u^T w + 2 beta u^T s + beta^2 p^T s, u^T s and p^T s from the last update
                            const float2* sx = (const float2*)s_xd;
                            const DZ us = {sx[c], sx[R + c]}, ps = {sx[2 * R + c], sx[3 * R + c]};
                            e = dz_add(dz_add(d, dz_mul(dz_add(b, b), us)), dz_mul(dz_mul(b, b), ps));
                        } else {
                            e = dz_sub(d, dz_mul(dz_mul(b, g), dz_of(s_ial4[c])));  // delta - beta gamma / alpha_old
                        }
                    }
                    s_b4[c] = dz_f4(b);
                    if (!dz_usable(e) || !dz_usable(g)) {
                        if (s_first[c]) {  // breakdown right after a (re)start
                            s_active[c] = 0;
                            s_done[c] = 1;
                            s_status[c] = FE_ERR_BREAKDOWN;
                        } else {  // restart from the true residual next round
                            s_repl[c] = 1;
                            s_first[c] = 1;
                        }
                    } else {
                        const float4 a4 = dz_f4(dz_div(g, e));
                        s_a4[c] = a4;
                        s_na4[c] = make_float4(-a4.x, -a4.y, -a4.z, -a4.w);
                        s_gam4[c] = dz_f4(g);
                        s_iters[c] += 1;
                        s_pass_it[c] += 1;
                        s_first[c] = 0;
                        s_refresh[c] = 0;
                    }
                }
            }
        } else if (tid < R) {
            const int c = tid;
            if (s_active[c]) {
                const double gr = s_out[c], gi = s_out[R + c];
                const double dr = s_out[2 * R + c], di = s_out[3 * R + c];
                double br = 0.0, bi = 0.0, er = dr, ei = di;
                if (!s_first[c]) {
                    // beta = gamma / gamma_old
                    br = gr * s_igam_r[c] - gi * s_igam_i[c];
                    bi = gr * s_igam_i[c] + gi * s_igam_r[c];
                    if (P.expand && !s_refresh[c]) {
                        // u^T w + 2 beta u^T s + beta^2 p^T s, u^T s and p^T s from the last update
                        const double b2r = br * br - bi * bi, b2i = 2.0 * br * bi;
                        const double usr = s_xd[c], usi = s_xd[R + c], psr = s_xd[2 * R + c], psi = s_xd[3 * R + c];
                        er = dr + 2.0 * (br * usr - bi * usi) + (b2r * psr - b2i * psi);
                        ei = di + 2.0 * (br * usi + bi * usr) + (b2r * psi + b2i * psr);
                    } else if (s_refresh[c]) {
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
                        er = dr - (tr * s_ial_r[c] - ti * s_ial_i[c]);
                        ei = di - (tr * s_ial_i[c] + ti * s_ial_r[c]);
                    }
                }
                const double ed = er * er + ei * ei;
                const double gg = gr * gr + gi * gi;
                if (!(ed > 0.0) || !(ed < 1e300) || !(gg > 0.0) || !(gg < 1e300)) {
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
                    const double ar = (gr * er + gi * ei) * ie, ai = (gi * er - gr * ei) * ie;
                    s_al_r[c] = ar;
                    s_al_i[c] = ai;
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
        // With the expanded recurrence the update also takes u^T s and p^T s of
        // the new u, p and s: with u^T w from the next product they give the
        // next p^T A p = u^T w + 2 beta u^T s + beta^2 p^T s (A symmetric, so
        // p^T A u = u^T A p, here u^T s).
        float xf[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        double xd[4] = {0.0, 0.0, 0.0, 0.0};
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
                const float4 a4 = s_a4[my_c], na4 = s_na4[my_c], b4 = s_b4[my_c];
                float4* ex = (float4*)s_exch;
                for (int base = 0; base < n3; base += kChunk) {
                    const int i = base + tid;
                    const bool valid = act && tid < kChunk && i < n3;
                    const size_t o = base_o + i;
                    float4 rn = make_float4(0.f, 0.f, 0.f, 0.f), pp = rn, ss = rn;
                    if (valid) {
                        pp = dfc_axpy(ld_cg(U + o), b4, ld_cg(Pv + o));
                        ss = dfc_axpy(ld_cg(wv + o), b4, ld_cg(Sv + o));
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
                        const float4 uu = df_result_norm(acc);
                        U[o] = uu;
                        if (P.expand) {
                            dfc_mac4(xf + 0, uu, ss);
                            dfc_mac4(xf + 4, pp, ss);
                        }
                    }
                    __syncthreads();
                }
            } else
            for (int base = 0; base < n3; base += kChunk) {
                const int i = base + tid;
                const bool valid = act && tid < kChunk && i < n3;
                const size_t o = base_o + i;
                double2 rn = make_double2(0.0, 0.0), pp = rn, ss = rn;
                if (valid) {
                    pp = cfma(beta, __ldcg(P.p + o), __ldcg(P.u + o));
                    ss = cfma(beta, __ldcg(P.s + o), to_c128(ld_cg(wv + o)));
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
                    if (P.expand) {
                        xd[0] += uu.x * ss.x - uu.y * ss.y;
                        xd[1] += uu.x * ss.y + uu.y * ss.x;
                        xd[2] += pp.x * ss.x - pp.y * ss.y;
                        xd[3] += pp.x * ss.y + pp.y * ss.x;
                    }
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
        if (P.expand) {
            if constexpr (kDFV) cta_colsum_df<R, 4>(xf, s_red, s_in);
            else cta_colsum<R, 4>(xd, s_red, s_in);
            if (!grid_reduce<4 * R, kDFV>(P, cta, s_in, s_xd)) goto out;
        } else if (!grid_reduce<0>(P, cta, s_in, s_out)) {
            goto out;
        }
        FE_TRACE_MARK(7);
        ++trace_it;
        ++seg_it;
    }
out:
    if (seg_end) {  // the job goes on in a later launch: keep x in its working form, save the scalars
        __syncthreads();
        if (cta == 0) {
            if (tid < R) {
                ColState& cs = P.state->col[tid];
                cs.bn = s_bn[tid];
                cs.rr_ref = s_rr_ref[tid];
                cs.rel = s_rel[tid];
                cs.gam_r = s_gam_r[tid];
                cs.gam_i = s_gam_i[tid];
                cs.al_r = s_al_r[tid];
                cs.al_i = s_al_i[tid];
                cs.be_r = s_be_r[tid];
                cs.be_i = s_be_i[tid];
                cs.igam_r = s_igam_r[tid];
                cs.igam_i = s_igam_i[tid];
                cs.ial_r = s_ial_r[tid];
                cs.ial_i = s_ial_i[tid];
                cs.a4 = s_a4[tid];
                cs.na4 = s_na4[tid];
                cs.b4 = s_b4[tid];
                if constexpr (kDFV) {
                    cs.gam4 = s_gam4[tid];
                    cs.igam4 = s_igam4[tid];
                    cs.ial4 = s_ial4[tid];
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) cs.xd[k] = __double_as_longlong(s_xd[k * R + tid]);
                cs.active = s_active[tid];
                cs.done = s_done[tid];
                cs.status = s_status[tid];
                cs.iters = s_iters[tid];
                cs.outer = s_outer[tid];
                cs.first = s_first[tid];
                cs.refresh = s_refresh[tid];
                cs.repl = s_repl[tid];
                cs.pass_it = s_pass_it[tid];
                P.rep_status[tid] = FE_PENDING;
                P.rep_iters[tid] = s_iters[tid];
                P.rep_outer[tid] = s_outer[tid];
                P.rep_rel[tid] = s_rel[tid];
            }
            if (tid == 0) {
                P.state->any_repl = s_any_repl;
                P.state->any_refresh = s_any_refresh;
                P.state->seg_done = seg_it;
                P.state->seg_ns = globaltimer_ns() - seg_t0;
                P.state->started = 1;
                P.state->finished = 0;
            }
        }
        return;
    }
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
    if (cta == 0 && tid == 0 && P.state) {
        P.state->seg_done = seg_it;
        P.state->seg_ns = globaltimer_ns() - seg_t0;
        P.state->started = 1;
        P.state->finished = 1;
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
    DevBuf b, x, r, u, p, s, uM, pM, w, partial, result, sync, rep, trace, pk, state;
};

constexpr size_t kSmemBudget = 200 * 1024;  // dynamic; static shared memory adds ~20 KB

// Sizes the resident product map of an R = 1 class-path launch (P.res and
// its shared memory); `rows_per_cta` bounds a CTA's product rows.  The halo
// buffer then takes the rest of the budget: three segments of at most
// rows + 2 * res_tmid nodes each fit it whenever the estimate below does.
template <typename C>
bool size_res_map_once(SolveParams& P, int64_t rows_per_cta, size_t& dyn) {
    P.res = 0;
    P.res_bytes = 0;
    if (!P.row_class || P.halo <= 0) return false;
    const int64_t m = (rows_per_cta + kRowsPerWarpR1 + 1) & ~1ll;  // rows plus the padding of the explicit slots
    int64_t res_bytes = m * (int64_t)(sizeof(int) + sizeof(int2) + 27 * sizeof(int)) +
                        (m / kExplRows + 2) * (int64_t)sizeof(int);
    if (P.dictM)  // per-slot block indices, then the dictionary (16-byte aligned)
        res_bytes = ((res_bytes + 27 * m * (int64_t)sizeof(uint16_t) + 15) & ~15ll) +
                    9 * (int64_t)P.n_dict * (int64_t)sizeof(C);
    res_bytes = (res_bytes + 15) & ~15ll;
    const int64_t fixed = (int64_t)P.red_bytes + res_bytes;
    // the halo also holds the true-residual phase's column staging; shared
    // memory is kept to what is needed, since the rest of the SM's 256 KB is
    // its L1 cache, which catches the register spills of 1024 threads
    const int64_t need = std::max<int64_t>(3 * (m + 2 * (int64_t)P.res_tmid + 24) * 3 * (int64_t)sizeof(C) + 3 * 32,
                                           (int64_t)kWarps * kColsPerWarp * (int64_t)sizeof(int));
    if (fixed + need > (int64_t)kSmemBudget || m > (1 << 20)) return false;
    P.res = 1;
    P.res_rows_max = (int)m;
    P.res_bytes = (int)res_bytes;
    P.col_bytes = 0;
    P.stage = 1;
    P.halo_bytes = (need + 15) & ~15ll;
    dyn = (size_t)(fixed + P.halo_bytes);
    return true;
}

template <typename C>
bool size_res_map(SolveParams& P, int64_t rows_per_cta, size_t& dyn) {
    if (size_res_map_once<C>(P, rows_per_cta, dyn)) return true;
    if (!P.dictM) return false;
    P.dictM = nullptr;  // without the dictionary, explicit rows read the planes
    P.dict_idx = nullptr;
    P.n_dict = 0;
    return size_res_map_once<C>(P, rows_per_cta, dyn);
}

template <typename T, int R>
fe_status launch_solve(fe_ctx* ctx, SolveParams& P) {
    static_assert(kWarps == 32, "cta_colsum assumes 32 warps");
    using C = typename CplxT<T>::type;
    // one CTA per SM; the reduction scratch and (when it fits) the CTA's
    // vector halo live in dynamic shared memory
    P.n_cta = std::min(P.n_cta_req > 0 ? std::min(P.n_cta_req, ctx->num_sms) : ctx->num_sms, std::max(1, P.n_rows));
    P.part_half = (int64_t)P.n_cta * kMaxNV * R;
    P.red_bytes = (int)(kMaxNV * kWarps * R * sizeof(double));
    P.col_bytes = R == 1 ? (int)(kWarps * kColsPerWarp * sizeof(int)) : 0;
    // product phases: a CTA's range costs at most total / n_cta plus one row
    const int64_t rows_per_cta =
        std::min<int64_t>(P.n_rows, (P.cost_total / P.n_cta + P.cost_max) / P.cost_min + 2);
    const int64_t halo_bytes = (rows_per_cta + 2 * (int64_t)P.halo + 2) * 3 * R * (int64_t)sizeof(C) + 64;
    P.stage = (P.halo > 0 && (size_t)P.red_bytes + P.col_bytes + (size_t)halo_bytes <= kSmemBudget) ? 1 : 0;
    P.halo_bytes = P.stage ? halo_bytes : 0;
    size_t dyn = (size_t)P.red_bytes + P.col_bytes + (P.stage ? (size_t)halo_bytes : 0);
    P.res = 0;
    P.res_bytes = 0;
    if constexpr (kClassPath<T> && R == 1) size_res_map<C>(P, rows_per_cta, dyn);
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
fe_status launch_jobs_t(fe_ctx* ctx, SolveJob* const* jobs, const int* n_cta, int n, cudaStream_t stream,
                        const int* seg_iters) {
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
        P.part_half = (int64_t)P.n_cta * kMaxNV * R;
        P.red_bytes = red_bytes;
        P.col_bytes = col_bytes;
        const int64_t rows_per_cta =
            std::min<int64_t>(P.n_rows, (P.cost_total / P.n_cta + P.cost_max) / P.cost_min + 2);
        const int64_t halo_bytes = (rows_per_cta + 2 * (int64_t)P.halo + 2) * 3 * R * (int64_t)sizeof(C) + 64;
        const size_t need = (size_t)red_bytes + col_bytes + (size_t)halo_bytes;
        P.stage = (P.halo > 0 && need <= kSmemBudget) ? 1 : 0;
        if (P.stage) dyn = std::max(dyn, need);
        P.res = 0;
        P.res_bytes = 0;
        if constexpr (kClassPath<T> && R == 1) {
            size_t dres = 0;
            if (size_res_map<C>(P, rows_per_cta, dres)) dyn = std::max(dyn, dres);
        }
        P.seg_iters = seg_iters ? seg_iters[i] : 0;
        cta0[i + 1] = cta0[i] + n_cta[i];
        FE_CUDA(cudaMemsetAsync(P.sync, 0, sync_bytes(P.n_cta), stream));
    }
    for (int i = 0; i < n; ++i) Ps[i].halo_bytes = (int64_t)dyn - red_bytes - Ps[i].col_bytes - Ps[i].res_bytes;
    const int grid = cta0[n];
    DevBuf dparams, dcta;
    FE_TRY(dev_alloc(stream, dparams, (size_t)n * sizeof(SolveParams)));
    fe_status e = dev_alloc(stream, dcta, (size_t)(n + 1) * sizeof(int));
    if (e != FE_OK) {
        dev_free(stream, dparams);
        return e;
    }
    auto done = [&](fe_status st) {
        dev_free(stream, dparams);
        dev_free(stream, dcta);
        return st;
    };
    if (cudaMemcpyAsync(dparams.ptr, Ps.data(), (size_t)n * sizeof(SolveParams), cudaMemcpyHostToDevice,
                        stream) != cudaSuccess ||
        cudaMemcpyAsync(dcta.ptr, cta0.data(), (size_t)(n + 1) * sizeof(int), cudaMemcpyHostToDevice,
                        stream) != cudaSuccess) {
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
    const cudaError_t le = cudaLaunchCooperativeKernel((void*)k_solve_jobs<T, R>, dim3(grid), dim3(kThreads), args,
                                                       dyn, stream);
    if (le != cudaSuccess) {
        set_error("jobs: launch failed: %s", cudaGetErrorString(le));
        return done(FE_ERR_CUDA);
    }
    count_launches(1);
    return done(FE_OK);
}

template <typename T>
fe_status launch_jobs_w(fe_ctx* ctx, int R, SolveJob* const* jobs, const int* n_cta, int n, cudaStream_t stream,
                        const int* seg_iters) {
    switch (R) {
        case 1: return launch_jobs_t<T, 1>(ctx, jobs, n_cta, n, stream, seg_iters);
        case 2: return launch_jobs_t<T, 2>(ctx, jobs, n_cta, n, stream, seg_iters);
        case 4: return launch_jobs_t<T, 4>(ctx, jobs, n_cta, n, stream, seg_iters);
        case 8: return launch_jobs_t<T, 8>(ctx, jobs, n_cta, n, stream, seg_iters);
        case 16: return launch_jobs_t<T, 16>(ctx, jobs, n_cta, n, stream, seg_iters);
        case 32: return launch_jobs_t<T, 32>(ctx, jobs, n_cta, n, stream, seg_iters);
        default: set_error("jobs: unsupported tile width %d", R); return FE_ERR_UNSUPPORTED;
    }
}

}  // namespace fe
