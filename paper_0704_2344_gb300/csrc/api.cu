// Context, error reporting, device buffers and the prefix-sum primitive.
#include "fe_internal.cuh"

#include <cstring>
#include <new>

namespace fe {

static thread_local char g_err[1024] = "";
static std::atomic<int64_t> g_launches{0};

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

fe_status dev_alloc(cudaStream_t st, DevBuf& b, size_t bytes) {
    if (b.ptr && b.bytes >= bytes) return FE_OK;
    dev_free(st, b);
    if (bytes == 0) bytes = 16;
    // 16 bytes of slack so that 16-byte vector loads near the end stay inside.
    cudaError_t e = cudaMallocAsync(&b.ptr, bytes + 16, st);
    if (e != cudaSuccess) {
        b.ptr = nullptr;
        b.bytes = 0;
        set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return FE_ERR_OOM;
    }
    b.bytes = bytes;
    return FE_OK;
}

void dev_free(cudaStream_t st, DevBuf& b) {
    if (b.ptr) cudaFreeAsync(b.ptr, st);
    b.ptr = nullptr;
    b.bytes = 0;
}

// ---------------------------------------------------------------------------
// Exclusive scan: tiles of kScanTile items per CTA, a one-CTA scan of the
// tile sums, then a fix-up pass.  Integer only, so the result is exact.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int block_exclusive_scan(int v, int* total, int* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        int w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) s_warp[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    const int before = warp > 0 ? s_warp[warp - 1] : 0;
    *total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void k_scan_tiles(const int* __restrict__ in, int* __restrict__ out, int* __restrict__ tile_sums,
                             int64_t n) {
    __shared__ int s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        sum += v[i];
    }
    int total;
    int run = block_exclusive_scan(sum, &total, s_warp);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void k_scan_sums(int* sums, int n_tiles, int* d_total) {
    __shared__ int s_warp[32];
    int carry = 0;
    for (int b = 0; b < n_tiles; b += blockDim.x) {
        const int i = b + threadIdx.x;
        int v = i < n_tiles ? sums[i] : 0;
        int total;
        int ex = block_exclusive_scan(v, &total, s_warp);
        if (i < n_tiles) sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) *d_total = carry;
}

__global__ void k_scan_fix(int* __restrict__ out, const int* __restrict__ tile_sums, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_sums[i / kScanTile];
}

fe_status scan_exclusive(cudaStream_t st, const int* in, int* out, int64_t n, int* d_total, DevBuf& tmp) {
    if (n <= 0) {
        FE_CUDA(cudaMemsetAsync(d_total, 0, sizeof(int), st));
        return FE_OK;
    }
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    FE_TRY(dev_alloc(st, tmp, tiles * sizeof(int)));
    int* sums = (int*)tmp.ptr;
    k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, out, sums, n);
    FE_LAUNCHED();
    k_scan_sums<<<1, 1024, 0, st>>>(sums, (int)tiles, d_total);
    FE_LAUNCHED();
    k_scan_fix<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, sums, n);
    FE_LAUNCHED();
    return FE_OK;
}

}  // namespace fe

using namespace fe;

extern "C" {

void fe_options_default(fe_options* opt) {
    if (!opt) return;
    opt->stream = nullptr;
    opt->variant = FE_VARIANT_S;
    opt->abc_sigma = 1.0;
    opt->penalty_s = 1.0;
    opt->formulation = FE_FORMULATION_H;
}

const char* fe_last_error(void) { return g_err; }

int64_t fe_launch_count(void) { return g_launches.load(); }

fe_status fe_ctx_create(fe_ctx** out, int cuda_device, const fe_options* opt) {
    if (!out) {
        set_error("fe_ctx_create: out is NULL");
        return FE_ERR_INVALID_ARG;
    }
    *out = nullptr;
    fe_options o;
    fe_options_default(&o);
    if (opt) o = *opt;
    if (o.variant < FE_VARIANT_S || o.variant > FE_VARIANT_P) {
        set_error("fe_ctx_create: unknown variant %d", o.variant);
        return FE_ERR_INVALID_ARG;
    }
    if (o.formulation != FE_FORMULATION_H && o.formulation != FE_FORMULATION_E) {
        set_error("fe_ctx_create: unknown formulation %d", o.formulation);
        return FE_ERR_INVALID_ARG;
    }
    int ndev = 0;
    FE_CUDA(cudaGetDeviceCount(&ndev));
    if (cuda_device < 0 || cuda_device >= ndev) {
        set_error("fe_ctx_create: device %d out of range (%d devices)", cuda_device, ndev);
        return FE_ERR_INVALID_ARG;
    }
    FE_CUDA(cudaSetDevice(cuda_device));
    fe_ctx* c = new (std::nothrow) fe_ctx();
    if (!c) {
        set_error("fe_ctx_create: host allocation failed");
        return FE_ERR_OOM;
    }
    c->device = cuda_device;
    c->opt = o;
    if (o.stream) {
        c->stream = (cudaStream_t)o.stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            set_error("cudaStreamCreate: %s", cudaGetErrorString(e));
            return FE_ERR_CUDA;
        }
        c->own_stream = true;
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, cuda_device);
    // Meshes, systems and solve workspaces are created and freed per request:
    // keep freed blocks in the stream-ordered pool instead of returning them
    // to the driver at every synchronisation.
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, cuda_device) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) {
        set_error("cudaEventCreate failed");
        fe_ctx_destroy(c);
        return FE_ERR_CUDA;
    }
    fe_status s = dev_alloc(c->stream, c->small, 64 * sizeof(int));
    if (s == FE_OK && cudaMallocHost((void**)&c->h_small, 64 * sizeof(int)) != cudaSuccess) {
        set_error("pinned host allocation failed");
        s = FE_ERR_OOM;
    }
    if (s != FE_OK) {
        fe_ctx_destroy(c);
        return s;
    }
    *out = c;
    return FE_OK;
}

fe_status fe_ctx_synchronize(fe_ctx* c) {
    if (!c) {
        set_error("fe_ctx_synchronize: NULL context");
        return FE_ERR_INVALID_ARG;
    }
    FE_CUDA(cudaStreamSynchronize(c->stream));
    return FE_OK;
}

fe_status fe_last_solve_stats(const fe_ctx* c, fe_solve_stats* out) {
    if (!c || !out) {
        set_error("fe_last_solve_stats: NULL argument");
        return FE_ERR_INVALID_ARG;
    }
    *out = c->last_solve;
    return FE_OK;
}

void fe_ctx_destroy(fe_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    dev_free(c->stream, c->scan_tmp);
    dev_free(c->stream, c->small);
    cudaStreamSynchronize(c->stream);
    if (c->h_small) cudaFreeHost(c->h_small);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"
