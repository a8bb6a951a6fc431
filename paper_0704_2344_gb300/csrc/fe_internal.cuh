// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../include/fe.h"

namespace fe {

constexpr uint8_t kPEC = 255;
constexpr double kC0 = 299792458.0;
constexpr double kPi = 3.14159265358979323846;

// Device-side error codes written to the context's status word.
enum : int { kDevOk = 0, kDevTimeout = 1, kDevBadIndex = 2, kDevSingular = 4 };

void set_error(const char* fmt, ...);
void count_launches(int64_t n);

#define FE_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            ::fe::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
            return e_ == cudaErrorMemoryAllocation ? FE_ERR_OOM : FE_ERR_CUDA;             \
        }                                                                                  \
    } while (0)

#define FE_LAUNCHED()                                                                      \
    do {                                                                                   \
        ::fe::count_launches(1);                                                           \
        cudaError_t e_ = cudaGetLastError();                                               \
        if (e_ != cudaSuccess) {                                                           \
            ::fe::set_error("%s:%d launch: %s", __FILE__, __LINE__, cudaGetErrorString(e_)); \
            return FE_ERR_CUDA;                                                            \
        }                                                                                  \
    } while (0)

#define FE_TRY(expr)                  \
    do {                              \
        fe_status s_ = (expr);        \
        if (s_ != FE_OK) return s_;   \
    } while (0)

// Stream-ordered device buffer owned by the library.
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};
fe_status dev_alloc(cudaStream_t st, DevBuf& b, size_t bytes);
void dev_free(cudaStream_t st, DevBuf& b);

// Box faces -x, +x, -y, +y, -z, +z: kinds packed 2 bits per face, and the
// mask of absorbing faces.
inline unsigned pack_planes(const int* b) {
    unsigned p = 0;
    for (int f = 0; f < 6; ++f) p |= (unsigned)(b[f] & 3) << (2 * f);
    return p;
}
inline unsigned abc_faces(const int* b) {
    unsigned m = 0;
    for (int f = 0; f < 6; ++f) m |= (b[f] == FE_BOUNDARY_ABC ? 1u : 0u) << f;
    return m;
}

// Bit c set when component c of grid node (i, j, k) is held at zero by a
// plane face: the normal component on a symmetry plane (Eq. 6a), the two
// tangential ones on an antisymmetry plane (Eq. 6b).
__host__ __device__ inline unsigned fixed_components(int i, int j, int k, int nx, int ny, int nz, unsigned planes) {
    unsigned m = 0;
    const int c[3] = {i, j, k}, d[3] = {nx, ny, nz};
    for (int f = 0; f < 6; ++f) {
        const unsigned kind = (planes >> (2 * f)) & 3u;
        if (!kind) continue;
        const int axis = f >> 1;
        if (c[axis] != ((f & 1) ? d[axis] : 0)) continue;
        m |= kind == 1u ? (1u << axis) : (7u & ~(1u << axis));
    }
    return m;
}

// E formulation: bit c set when component c of grid node (i, j, k) is held at
// zero on a conductor surface (n x E = 0).  Axis a is a surface normal at
// the node when two of its (up to) eight elements that differ only along a
// are one PEC and one active; every component but a is then tangential.
__device__ inline unsigned pec_held(const uint8_t* __restrict__ mat, int nx, int ny, int nz, int i, int j, int k) {
    unsigned pec = 0, act = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int a = i - 1 + (b & 1), c = j - 1 + ((b >> 1) & 1), d = k - 1 + ((b >> 2) & 1);
        if (a < 0 || a >= nx || c < 0 || c >= ny || d < 0 || d >= nz) continue;
        if (mat[a + (int64_t)nx * (c + (int64_t)ny * d)] == kPEC) pec |= 1u << b;
        else act |= 1u << b;
    }
    unsigned held = 0;
#pragma unroll
    for (int axis = 0; axis < 3; ++axis) {
        const unsigned bit = 1u << axis;
        bool normal = false;
#pragma unroll
        for (unsigned b = 0; b < 8; ++b)
            if (!(b & bit) && ((((pec >> b) & 1u) && ((act >> (b | bit)) & 1u)) ||
                               (((act >> b) & 1u) && ((pec >> (b | bit)) & 1u))))
                normal = true;
        if (normal) held |= 7u & ~bit;
    }
    return held;
}

// Exclusive prefix sum of n int32 values (in may alias out); writes the total
// to *d_total (device).  Uses `tmp` (grown as needed) for block sums.
fe_status scan_exclusive(cudaStream_t st, const int* in, int* out, int64_t n, int* d_total, DevBuf& tmp);

}  // namespace fe

struct fe_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    fe_options opt{};
    int num_sms = 0;
    fe::DevBuf scan_tmp;
    fe::DevBuf small;  // small device scratch: totals, status words
    int* h_small = nullptr;  // pinned host mirror of `small` (64 ints)
    fe_solve_stats last_solve{};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

struct fe_mesh {
    fe_ctx* ctx = nullptr;
    int nx = 0, ny = 0, nz = 0;
    double h[3]{}, origin[3]{};
    int64_t n_el = 0, n_nodes_total = 0;
    int n_act = 0, nnzb = 0, n_ext = 0, n_pec = 0, n_act_el = 0;
    int n_mat = 0;
    int boundary[6] = {0, 0, 0, 0, 0, 0};  // fe_boundary per face
    std::vector<fe_complex> eps, mu;
    fe::DevBuf material, node_rank, node_id, row_ptr, col_idx, elem_slot, faces_ext, faces_pec;
    int64_t bytes = 0;
};

struct fe_system {
    fe_ctx* ctx = nullptr;
    const fe_mesh* mesh = nullptr;
    double freq = 0, k0 = 0;
    int precision = FE_PREC_MIXED;
    int variant = FE_VARIANT_S;
    int formulation = FE_FORMULATION_H;
    double sigma = -1, s_pen = 1;
    fe::DevBuf tables;               // double2 [(n_mat + 12) * 576], block-major
    // Block values are stored as 9 planes, one per block entry (alpha, beta):
    // value (alpha, beta) of block s at [(3*alpha + beta) * stride + s], so a
    // warp reading one entry of consecutive blocks reads consecutive memory.
    int64_t stride = 0;              // plane stride: nnzb rounded up to a multiple of 64
    fe::DevBuf val64, val32;         // double2 / float2 [9 * stride]
    fe::DevBuf valdf;                // float4 [9 * stride]: FP32 pairs (re_hi, im_hi, re_lo, im_lo), FE_PREC_DF
    fe::DevBuf dinv64, dinv32;       // double2 / float2 [n_act * 9]
    fe::DevBuf dinvdf;               // float4 [n_act * 9]: FP32 pairs of dinv64, FE_PREC_DF
    // Regular rows: interior nodes whose 8 elements are active, of one
    // material and have no outer or PEC face.  All regular rows of a material
    // carry the same 27 blocks (same element tables, same summation order), so
    // the products read them from a per-class stencil instead of the planes.
    fe::DevBuf row_class;            // int8 [n_act]: class (material < kMaxClasses) or -1
    fe::DevBuf stencil;              // StencilSet (device)
    // prefix sum of a per-row cost of the complex64 sparse product (see
    // fe_assemble for the weights): the product phases split rows across
    // CTAs by equal cost
    fe::DevBuf cost_prefix;          // int [n_act + 1]
    int64_t cost_total = 0;
    // the same with the weights of the FP32-pair products
    fe::DevBuf cost_prefix_alu;      // int [n_act + 1]
    int64_t cost_total_alu = 0;
    // prefix sum of the stored blocks of explicit rows (rows of no class)
    fe::DevBuf expl_prefix;          // int [n_act + 1]; expl_prefix[n_act] = blocks_explicit
    // Block dictionary (complex64 and FP32-pair systems): the distinct 3x3
    // blocks once, in the inner precision, entry (alpha, beta) of block d at
    // [9 d + 3 alpha + beta], and each stored block's index.  n_dict = 0: none.
    fe::DevBuf dict_idx;             // uint16 [nnzb]
    fe::DevBuf dict_vals;            // float2 or float4 [n_dict * 9]
    int n_dict = 0;
    int cost_min[2] = {1, 1}, cost_max[2] = {1, 1};  // bounds of one row's cost (complex64, FP32 pairs)
    int64_t rows_general = 0, rows_diagonal = 0, blocks_explicit = 0;  // rows per product path
    // Block incomplete Cholesky factor (Section 3.1.5.3): node rows split into
    // bicp_n_sub contiguous bands, floor(b n / S) <= I < floor((b + 1) n / S),
    // one per CTA of the solve; L L^T reproduces A on the lower node-block
    // pattern of each band.
    int bicp_n_sub = 0;
    fe::DevBuf bicp_l;               // double2 [nnzb * 9]: L_IJ at block slot (I, J), row-major 3x3
                                     //   (J < I in I's band; L_II lower triangular; zero elsewhere)
    fe::DevBuf bicp_linv;            // double2 [n_act * 9]: L_II^{-1} (lower triangular)
    fe::DevBuf bicp_tpos;            // int [nnzb]: slot of block (J, I) for the block (I, J)
    fe::DevBuf bicp_tab;             // int4 [n_act]: each band's nodes sorted by level, in the band's range:
                                     //   (node, first slot in the band, diagonal slot, end of the band's slots)
    fe::DevBuf bicp_lev;             // int [n_act + n_sub]: band b's level offsets at [first node + b, ...]
    fe::DevBuf bicp_nlev;            // int [n_sub]: levels per band
};

namespace fe {
constexpr int kMaxClasses = 4;
constexpr int kMaxDict = 4096;  // distinct blocks a dictionary may hold
fe_status build_block_dict(fe_ctx* ctx, fe_system* s);
// Per-class stencils of regular rows, indexed [class][alpha][block k][beta];
// kind: 0 = no regular row, 1 = general complex blocks, 2 = real diagonal
// blocks (the homogeneous interior with eps_r = 1 and s = 1); dval holds the
// diagonal of kind 2.
struct StencilSet {
    int kind[kMaxClasses];
    int pad[kMaxClasses];
    double2 s64[kMaxClasses][3][27][3];
    float2 s32[kMaxClasses][3][27][3];
    double dval[kMaxClasses][3][27];
    float dval32[kMaxClasses][3][27];
    float4 sdf[kMaxClasses][3][27][3];   // FP32 pairs of s64
    float2 dvaldf[kMaxClasses][3][27];   // FP32 pairs (hi, lo) of dval
};
}  // namespace fe
