// Block dictionary of an assembled system.
//
// On a voxel mesh the 3x3 blocks of Eq. 4's matrix are sums of a few element
// and face tables chosen by the local configuration (materials of the
// elements around two nodes, absorbing or PEC faces among them), and the
// gather assembly adds them in a fixed order, so equal configurations give
// bitwise equal blocks: the 748 658 blocks of the 3-wavelength cube take about
// four hundred distinct values.  The dictionary lists the distinct blocks once
// (in the inner precision of the products) and gives every stored block its
// index, so that a product can read an explicit row's blocks from a table of a
// few tens of KB held in shared memory instead of streaming 9 values per
// block from L2.
//
// Construction: a 64-bit hash of each block's 18 FP64 words; an
// open-addressing table (bounded probing) keyed by the hash, whose entry keeps
// the lowest block slot with that hash; ids numbered by that representative
// slot (deterministic); and a check that every block equals its
// representative bit for bit.  A hash collision between different blocks, a
// table overflow or more than kMaxDict distinct blocks leaves the system
// without a dictionary (the products then read the planes).
#include "fe_internal.cuh"

#include <algorithm>
#include <vector>

namespace fe {

constexpr int kDictTableBits = 17;
constexpr int kDictTable = 1 << kDictTableBits;
constexpr int kDictProbes = 64;

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    // the finaliser of the SplitMix64 generator (Steele, Lea and Flood, 2014)
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long block_hash(const double2* __restrict__ val, int64_t stride, int64_t s) {
    unsigned long long h = 0x9e3779b97f4a7c15ull;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const double2 v = val[q * stride + s];
        h = mix64(h ^ (unsigned long long)__double_as_longlong(v.x));
        h = mix64(h ^ (unsigned long long)__double_as_longlong(v.y));
    }
    return h | 1ull;  // 0 marks an empty table entry
}

// Inserts every block's hash; slot_of[s] = its table entry (-1: overflow).
__global__ void k_dict_insert(const double2* __restrict__ val, int64_t stride, int nnzb,
                              unsigned long long* __restrict__ keys, int* __restrict__ rep, int* __restrict__ slot_of,
                              int* __restrict__ d_new, int* __restrict__ d_overflow) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nnzb) return;
    const unsigned long long h = block_hash(val, stride, s);
    unsigned t = (unsigned)(h >> (64 - kDictTableBits));
    for (int probe = 0; probe < kDictProbes; ++probe, t = (t + 1) & (kDictTable - 1)) {
        const unsigned long long prev = atomicCAS(keys + t, 0ull, h);
        if (prev == 0ull || prev == h) {
            if (prev == 0ull) atomicAdd(d_new, 1);
            atomicMin(rep + t, s);
            slot_of[s] = (int)t;
            return;
        }
    }
    slot_of[s] = -1;
    atomicExch(d_overflow, 1);
}

// Block s gets its value's id; blocks that differ from their representative
// (a hash collision) are counted.
__global__ void k_dict_index(const double2* __restrict__ val, int64_t stride, int nnzb, const int* __restrict__ slot_of,
                             const int* __restrict__ rep, const int* __restrict__ id_of_slot,
                             uint16_t* __restrict__ dict_idx, int* __restrict__ d_mismatch) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nnzb) return;
    const int t = slot_of[s];
    if (t < 0) return;
    const int r = rep[t];
    bool same = true;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const double2 a = val[q * stride + s], b = val[q * stride + r];
        same = same && __double_as_longlong(a.x) == __double_as_longlong(b.x) &&
               __double_as_longlong(a.y) == __double_as_longlong(b.y);
    }
    if (!same) atomicAdd(d_mismatch, 1);
    dict_idx[s] = (uint16_t)id_of_slot[t];
}

// Entry q = 3 alpha + beta of dictionary block d, in the inner precisions.
__global__ void k_dict_fill(const int* __restrict__ rep_of_id, int n_dict, int64_t stride,
                            const float2* __restrict__ val32, const float4* __restrict__ valdf,
                            float2* __restrict__ d32, float4* __restrict__ ddf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 9 * n_dict) return;
    const int d = i / 9, q = i % 9;
    const int64_t src = q * stride + rep_of_id[d];
    if (d32) d32[i] = val32[src];
    if (ddf) ddf[i] = valdf[src];
}

fe_status build_block_dict(fe_ctx* ctx, fe_system* s) {
    const fe_mesh* m = s->mesh;
    cudaStream_t st = ctx->stream;
    s->n_dict = 0;
    const bool df = s->precision == FE_PREC_DF, mixed = s->precision == FE_PREC_MIXED;
    if ((!df && !mixed) || m->nnzb < 1) return FE_OK;
    DevBuf keys, rep, slot_of, idmap, flags, reps;
    auto done = [&](fe_status e) {
        for (DevBuf* b : {&keys, &rep, &slot_of, &idmap, &flags, &reps}) dev_free(st, *b);
        return e;
    };
    fe_status e;
    if ((e = dev_alloc(st, keys, (size_t)kDictTable * sizeof(unsigned long long))) != FE_OK) return done(e);
    if ((e = dev_alloc(st, rep, (size_t)kDictTable * sizeof(int))) != FE_OK) return done(e);
    if ((e = dev_alloc(st, slot_of, (size_t)m->nnzb * sizeof(int))) != FE_OK) return done(e);
    if ((e = dev_alloc(st, flags, 4 * sizeof(int))) != FE_OK) return done(e);
    FE_CUDA(cudaMemsetAsync(keys.ptr, 0, (size_t)kDictTable * sizeof(unsigned long long), st));
    FE_CUDA(cudaMemsetAsync(rep.ptr, 0x7f, (size_t)kDictTable * sizeof(int), st));
    FE_CUDA(cudaMemsetAsync(flags.ptr, 0, 4 * sizeof(int), st));
    int* d_flags = (int*)flags.ptr;  // new entries, overflow, mismatches
    const unsigned grid = (unsigned)((m->nnzb + 255) / 256);
    k_dict_insert<<<grid, 256, 0, st>>>((const double2*)s->val64.ptr, s->stride, m->nnzb,
                                        (unsigned long long*)keys.ptr, (int*)rep.ptr, (int*)slot_of.ptr, d_flags,
                                        d_flags + 1);
    FE_LAUNCHED();
    int h_flags[2] = {0, 0};
    FE_CUDA(cudaMemcpyAsync(h_flags, d_flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    FE_CUDA(cudaStreamSynchronize(st));
    const int n_dict = h_flags[0];
    if (h_flags[1] || n_dict < 1 || n_dict > kMaxDict) return done(FE_OK);
    // deterministic ids: occupied entries ordered by their representative slot
    std::vector<unsigned long long> h_keys(kDictTable);
    std::vector<int> h_rep(kDictTable);
    FE_CUDA(cudaMemcpyAsync(h_keys.data(), keys.ptr, h_keys.size() * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, st));
    FE_CUDA(cudaMemcpyAsync(h_rep.data(), rep.ptr, h_rep.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
    FE_CUDA(cudaStreamSynchronize(st));
    std::vector<std::pair<int, int>> occ;  // (representative slot, table entry)
    for (int t = 0; t < kDictTable; ++t)
        if (h_keys[t]) occ.emplace_back(h_rep[t], t);
    std::sort(occ.begin(), occ.end());
    std::vector<int> id_of_slot(kDictTable, 0), rep_of_id(occ.size());
    for (size_t i = 0; i < occ.size(); ++i) {
        id_of_slot[occ[i].second] = (int)i;
        rep_of_id[i] = occ[i].first;
    }
    if ((e = dev_alloc(st, idmap, (size_t)kDictTable * sizeof(int))) != FE_OK) return done(e);
    if ((e = dev_alloc(st, reps, rep_of_id.size() * sizeof(int))) != FE_OK) return done(e);
    if ((e = dev_alloc(st, s->dict_idx, (size_t)m->nnzb * sizeof(uint16_t))) != FE_OK) return done(e);
    FE_CUDA(cudaMemcpyAsync(idmap.ptr, id_of_slot.data(), (size_t)kDictTable * sizeof(int), cudaMemcpyHostToDevice,
                            st));
    FE_CUDA(cudaMemcpyAsync(reps.ptr, rep_of_id.data(), rep_of_id.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    k_dict_index<<<grid, 256, 0, st>>>((const double2*)s->val64.ptr, s->stride, m->nnzb, (const int*)slot_of.ptr,
                                       (const int*)rep.ptr, (const int*)idmap.ptr, (uint16_t*)s->dict_idx.ptr,
                                       d_flags + 2);
    FE_LAUNCHED();
    const size_t esz = df ? sizeof(float4) : sizeof(float2);
    if ((e = dev_alloc(st, s->dict_vals, (size_t)n_dict * 9 * esz)) != FE_OK) {
        dev_free(st, s->dict_idx);
        return done(e);
    }
    k_dict_fill<<<(unsigned)((9 * n_dict + 255) / 256), 256, 0, st>>>(
        (const int*)reps.ptr, n_dict, s->stride, (const float2*)s->val32.ptr, (const float4*)s->valdf.ptr,
        mixed ? (float2*)s->dict_vals.ptr : nullptr, df ? (float4*)s->dict_vals.ptr : nullptr);
    FE_LAUNCHED();
    int mismatch = 0;
    FE_CUDA(cudaMemcpyAsync(&mismatch, d_flags + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
    FE_CUDA(cudaStreamSynchronize(st));  // the host vectors must outlive the copies
    if (mismatch) {  // a hash collision between different blocks: no dictionary
        dev_free(st, s->dict_idx);
        dev_free(st, s->dict_vals);
        return done(FE_OK);
    }
    s->n_dict = n_dict;
    return done(FE_OK);
}

}  // namespace fe
