// Half (symmetric) storage of the block matrix and its sparse product
// (storage #1 of Section 4.2; the product of Section 4.2.5.1).
//
// The symmetrised matrix is kept by its lower part only: per block row the
// blocks (I, J <= I), which are the row's first slots in the sorted block
// pattern (diagonal last), compacted, the 9 entries of a block contiguous
// (row-major 3x3).  An upper block
// (I, J > I) is the transpose of the kept (J, I); a per-slot index gives
// its place in row J.  The product is a gather: a warp per block row, a
// lane per block of the full row, the upper lanes reading their block
// transposed from the neighbour's kept part.  Those reads come back within
// about one grid plane of rows, while the neighbour's own warp has just
// read the same block, so they are mostly served by L2, and the matrix
// bytes read from HBM are about those of the kept half (14 of 27 blocks of
// an interior row).  Keeping a block's entries together makes a
// transposed read three 32-byte sectors (complex64) instead of one sector
// per entry, as planes would.
//
// The storage belongs to a system: it is kept in a registry keyed by the
// system and released with it.
#include "krylov.cuh"

#include <algorithm>
#include <mutex>
#include <new>
#include <type_traits>
#include <unordered_map>

namespace fe {

struct HalfStore {
    int64_t nnzb = 0;              // kept blocks
    DevBuf ptr;                    // int [n_act + 1]: first kept slot of each row
    DevBuf up;                     // int [nnzb]: kept slot of (J, I) for a full slot (I, J > I), else -1
    DevBuf val64;                  // double2 [nnzb][9], row-major 3x3 per block
    DevBuf val32;                  // float2 [nnzb][9] (systems with a complex64 copy)
    cudaStream_t st = nullptr;
};

namespace {

std::mutex g_half_mu;
std::unordered_map<const fe_system*, HalfStore*> g_half;

HalfStore* half_of(const fe_system* s) {
    std::lock_guard<std::mutex> lk(g_half_mu);
    auto it = g_half.find(s);
    return it == g_half.end() ? nullptr : it->second;
}

void half_free(HalfStore* h) {
    for (DevBuf* b : {&h->ptr, &h->up, &h->val64, &h->val32}) dev_free(h->st, *b);
    delete h;
}

__global__ void k_half_count(int n, const int* __restrict__ rp, const int* __restrict__ col, int* __restrict__ cnt) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= n) return;
    int c = 0;
    for (int p = rp[I]; p < rp[I + 1]; ++p) c += col[p] <= I ? 1 : 0;
    cnt[I] = c;
}

// Kept slots: copy the row's first hp[I+1]-hp[I] blocks; upper slots: find
// (J, I) among row J's kept blocks.
template <typename C>
__global__ void k_half_fill(int n, const int* __restrict__ rp, const int* __restrict__ col, const int* __restrict__ hp,
                            const C* __restrict__ val, int64_t stride, C* __restrict__ hval,
                            int* __restrict__ up, int* __restrict__ status) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= n) return;
    const int p0 = rp[I], q0 = hp[I];
    for (int p = p0; p < rp[I + 1]; ++p) {
        const int J = col[p];
        if (J <= I) {
            const int q = q0 + (p - p0);
#pragma unroll
            for (int k = 0; k < 9; ++k) hval[(size_t)q * 9 + k] = val[k * stride + p];
            if (up) up[p] = -1;
        } else if (up) {
            int t = -1;
            for (int r = rp[J]; r < rp[J + 1]; ++r)
                if (col[r] == I) t = hp[J] + (r - rp[J]);
            up[p] = t;
            if (t < 0) atomicOr(status, kDevBadIndex);
        }
    }
}

// y = A x from the half storage, R = 1, 2, 4, ..., 32 columns: one warp per
// block row, its lanes split into 32/R block groups x R columns (as the
// full-storage product), a block read directly for J <= I and transposed
// from row J for J > I; the groups' partial sums meet in a fixed butterfly.
template <typename C, int R>
__global__ void __launch_bounds__(256) k_spmv_half(const C* __restrict__ hval, const int* __restrict__ hp, const int* __restrict__ up,
                                                   const int* __restrict__ col, const int* __restrict__ rp,
                                                   const C* __restrict__ x, C* __restrict__ y, int n_rows) {
    using Tr = decltype(C{}.x);
    const int lane = threadIdx.x & 31;
    constexpr int G = 32 / R;
    const int c = lane % R, g = lane / R;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n_rows; row += nw) {
        const int s0 = __ldg(rp + row), s1 = __ldg(rp + row + 1);
        const int q0 = __ldg(hp + row), kept = __ldg(hp + row + 1) - q0;
        Tr a[6] = {0, 0, 0, 0, 0, 0};
        for (int s = s0 + g; s < s1; s += G) {
            const bool low = s - s0 < kept;
            const int q = low ? q0 + (s - s0) : __ldg(up + s);
            const int cb = __ldg(col + s);
            C m[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) m[k] = __ldg(hval + (size_t)q * 9 + k);
            const int xb = 3 * cb * R + c;
            C xv[3];
#pragma unroll
            for (int be = 0; be < 3; ++be) xv[be] = __ldg(x + xb + be * R);
#pragma unroll
            for (int al = 0; al < 3; ++al)
#pragma unroll
                for (int be = 0; be < 3; ++be) {
                    const C e = low ? m[3 * al + be] : m[3 * be + al];
                    a[2 * al] += e.x * xv[be].x - e.y * xv[be].y;
                    a[2 * al + 1] += e.x * xv[be].y + e.y * xv[be].x;
                }
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

template <typename C>
void launch_half(int R, unsigned blocks, cudaStream_t st, const C* hval, const int* hp, const int* up,
                 const int* col, const int* rp, const C* x, C* y, int n) {
    switch (R) {
        case 1: k_spmv_half<C, 1><<<blocks, 256, 0, st>>>(hval, hp, up, col, rp, x, y, n); break;
        case 2: k_spmv_half<C, 2><<<blocks, 256, 0, st>>>(hval, hp, up, col, rp, x, y, n); break;
        case 4: k_spmv_half<C, 4><<<blocks, 256, 0, st>>>(hval, hp, up, col, rp, x, y, n); break;
        case 8: k_spmv_half<C, 8><<<blocks, 256, 0, st>>>(hval, hp, up, col, rp, x, y, n); break;
        case 16: k_spmv_half<C, 16><<<blocks, 256, 0, st>>>(hval, hp, up, col, rp, x, y, n); break;
        default: k_spmv_half<C, 32><<<blocks, 256, 0, st>>>(hval, hp, up, col, rp, x, y, n); break;
    }
}

unsigned blocks_for_n(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

void half_release(const fe_system* s) {
    HalfStore* h = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_half_mu);
        auto it = g_half.find(s);
        if (it == g_half.end()) return;
        h = it->second;
        g_half.erase(it);
    }
    half_free(h);
}

int64_t half_bytes(const fe_system* s) {
    const HalfStore* h = half_of(s);
    return h ? (int64_t)(h->ptr.bytes + h->up.bytes + h->val64.bytes + h->val32.bytes) : 0;
}

}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_system_pack_half(fe_ctx* ctx, fe_system* s, int64_t* kept_blocks) {
    if (!ctx || !s) {
        set_error("fe_system_pack_half: NULL argument");
        return FE_ERR_INVALID_ARG;
    }
    const fe_mesh* m = s->mesh;
    if (s->variant == FE_VARIANT_L || m->n_act < 1 || !s->val64.ptr) {
        set_error("fe_system_pack_half: needs a symmetric variant (S or P) with rows");
        return FE_ERR_INVALID_ARG;
    }
    FE_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    half_release(s);
    HalfStore* h = new (std::nothrow) HalfStore();
    if (!h) {
        set_error("fe_system_pack_half: host allocation failed");
        return FE_ERR_OOM;
    }
    h->st = st;
    const int n = m->n_act;
    const int* rp = (const int*)m->row_ptr.ptr;
    const int* col = (const int*)m->col_idx.ptr;
    DevBuf cnt, status;
    auto fail = [&](fe_status e) {
        dev_free(st, cnt);
        dev_free(st, status);
        half_free(h);
        return e;
    };
    fe_status e;
    if ((e = dev_alloc(st, h->ptr, ((size_t)n + 1) * sizeof(int))) != FE_OK) return fail(e);
    if ((e = dev_alloc(st, h->up, (size_t)m->nnzb * sizeof(int))) != FE_OK) return fail(e);
    if ((e = dev_alloc(st, cnt, (size_t)n * sizeof(int))) != FE_OK) return fail(e);
    if ((e = dev_alloc(st, status, sizeof(int))) != FE_OK) return fail(e);
    if (cudaMemsetAsync(status.ptr, 0, sizeof(int), st) != cudaSuccess) {
        set_error("fe_system_pack_half: memset failed");
        return fail(FE_ERR_CUDA);
    }
    k_half_count<<<blocks_for_n(n, 128), 128, 0, st>>>(n, rp, col, (int*)cnt.ptr);
    count_launches(1);
    int* hp = (int*)h->ptr.ptr;
    if ((e = scan_exclusive(st, (const int*)cnt.ptr, hp, n, hp + n, ctx->scan_tmp)) != FE_OK) return fail(e);
    int total = 0;
    cudaError_t ce = cudaMemcpyAsync(&total, hp + n, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) {
        set_error("fe_system_pack_half: %s", cudaGetErrorString(ce));
        return fail(FE_ERR_CUDA);
    }
    h->nnzb = total;
    if ((e = dev_alloc(st, h->val64, (size_t)total * 9 * sizeof(double2))) != FE_OK) return fail(e);
    k_half_fill<double2><<<blocks_for_n(n, 128), 128, 0, st>>>(n, rp, col, hp, (const double2*)s->val64.ptr,
                                                               s->stride, (double2*)h->val64.ptr, (int*)h->up.ptr,
                                                               (int*)status.ptr);
    count_launches(1);
    if (s->val32.ptr) {
        if ((e = dev_alloc(st, h->val32, (size_t)total * 9 * sizeof(float2))) != FE_OK) return fail(e);
        k_half_fill<float2><<<blocks_for_n(n, 128), 128, 0, st>>>(n, rp, col, hp, (const float2*)s->val32.ptr,
                                                                 s->stride, (float2*)h->val32.ptr, nullptr,
                                                                 (int*)status.ptr);
        count_launches(1);
    }
    int hs = 0;
    ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&hs, status.ptr, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) {
        set_error("fe_system_pack_half: %s", cudaGetErrorString(ce));
        return fail(FE_ERR_CUDA);
    }
    if (hs & kDevBadIndex) {
        set_error("fe_system_pack_half: the block pattern is not structurally symmetric");
        return fail(FE_ERR_CUDA);
    }
    dev_free(st, cnt);
    dev_free(st, status);
    {
        std::lock_guard<std::mutex> lk(g_half_mu);
        g_half[s] = h;
    }
    if (kept_blocks) *kept_blocks = h->nnzb;
    return FE_OK;
}

fe_status fe_spmv_half(fe_ctx* ctx, const fe_system* s, int32_t precision, int32_t nrhs, const void* x, void* y) {
    if (!ctx || !s || !x || !y || nrhs < 1 || nrhs > 32 || (nrhs & (nrhs - 1)) != 0) {
        set_error("fe_spmv_half: NULL argument, or nrhs not a power of two in [1, 32]");
        return FE_ERR_INVALID_ARG;
    }
    const HalfStore* h = half_of(s);
    if (!h) {
        set_error("fe_spmv_half: no half storage (call fe_system_pack_half first)");
        return FE_ERR_INVALID_ARG;
    }
    const fe_mesh* m = s->mesh;
    cudaStream_t st = ctx->stream;
    const int* rp = (const int*)m->row_ptr.ptr;
    const int* col = (const int*)m->col_idx.ptr;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)ctx->num_sms * 8,
                                                                             ((int64_t)m->n_act + 7) / 8));
    if (precision == FE_PREC_FP64) {
        launch_half<double2>(nrhs, blocks, st, (const double2*)h->val64.ptr, (const int*)h->ptr.ptr,
                             (const int*)h->up.ptr, col, rp, (const double2*)x, (double2*)y, m->n_act);
    } else if (precision == FE_PREC_MIXED) {
        if (!h->val32.ptr) {
            set_error("fe_spmv_half: no complex64 copy (system assembled in FP64)");
            return FE_ERR_INVALID_ARG;
        }
        launch_half<float2>(nrhs, blocks, st, (const float2*)h->val32.ptr, (const int*)h->ptr.ptr,
                            (const int*)h->up.ptr, col, rp, (const float2*)x, (float2*)y, m->n_act);
    } else {
        set_error("fe_spmv_half: precision must be FE_PREC_FP64 or FE_PREC_MIXED");
        return FE_ERR_INVALID_ARG;
    }
    FE_LAUNCHED();
    return FE_OK;
}

}  // extern "C"
