// Mesh validation and the integer maps of the block matrix, built on the
// device: active nodes and their lexicographic ranks, the 3x3-block row
// pattern (the paper's storage of the three rows of a node with only the
// couplings that exist, Section 3.1.2; the matrix structure of Section 4.2.1),
// the element-to-slot map and the outer / PEC face lists.
#include "fe_internal.cuh"

#include <cstring>
#include <new>

namespace fe {

struct Grid {
    int nx, ny, nz;
    __device__ __forceinline__ int64_t elem(int i, int j, int k) const {
        return (int64_t)i + (int64_t)nx * ((int64_t)j + (int64_t)ny * k);
    }
    __device__ __forceinline__ int64_t node(int i, int j, int k) const {
        return (int64_t)i + (int64_t)(nx + 1) * ((int64_t)j + (int64_t)(ny + 1) * k);
    }
};

// Bit (ex + 2 ey + 4 ez) set when element (i-1+ex, j-1+ey, k-1+ez) exists and
// is not PEC: the up to eight elements around node (i, j, k).
__device__ __forceinline__ unsigned node_elem_mask(const uint8_t* __restrict__ mat, Grid g, int i, int j, int k) {
    unsigned m = 0;
#pragma unroll
    for (int ez = 0; ez < 2; ++ez)
#pragma unroll
        for (int ey = 0; ey < 2; ++ey)
#pragma unroll
            for (int ex = 0; ex < 2; ++ex) {
                const int a = i - 1 + ex, b = j - 1 + ey, c = k - 1 + ez;
                if (a >= 0 && a < g.nx && b >= 0 && b < g.ny && c >= 0 && c < g.nz &&
                    mat[g.elem(a, b, c)] != kPEC)
                    m |= 1u << (ex + 2 * ey + 4 * ez);
            }
    return m;
}

// Elements around a node that also contain the neighbour at offset d (per
// axis -1, 0, +1): along an axis, offset -1 keeps only the lower element,
// +1 only the upper, 0 both.
__device__ __forceinline__ unsigned shared_elem_bits(int dx, int dy, int dz) {
    const unsigned ax = dx < 0 ? 0x55u : dx > 0 ? 0xAAu : 0xFFu;  // ex = 0 / 1
    const unsigned ay = dy < 0 ? 0x33u : dy > 0 ? 0xCCu : 0xFFu;  // ey = 0 / 1
    const unsigned az = dz < 0 ? 0x0Fu : dz > 0 ? 0xF0u : 0xFFu;  // ez = 0 / 1
    return ax & ay & az;
}

// 27-bit mask of existing blocks in the row of a node; bit l is the neighbour
// at offset (l % 3 - 1, (l / 3) % 3 - 1, l / 9 - 1): ascending l is ascending
// neighbour id, hence ascending column rank.
__device__ __forceinline__ unsigned row_mask(unsigned emask) {
    unsigned m = 0;
#pragma unroll
    for (int l = 0; l < 27; ++l)
        if (emask & shared_elem_bits(l % 3 - 1, (l / 3) % 3 - 1, l / 9 - 1)) m |= 1u << l;
    return m;
}

__global__ void k_validate(const uint8_t* __restrict__ mat, Grid g, int n_mat, uint32_t vac0, uint32_t vac1,
                           uint32_t vac2, uint32_t vac3, unsigned abc, int* flags) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool inside = e < (int64_t)g.nx * g.ny * g.nz;
    const unsigned act = __ballot_sync(0xffffffffu, inside && mat[inside ? e : 0] != kPEC);
    if ((threadIdx.x & 31) == 0 && act) atomicAdd(&flags[5], __popc(act));
    if (!inside) return;
    const int i = (int)(e % g.nx), j = (int)((e / g.nx) % g.ny), k = (int)(e / ((int64_t)g.nx * g.ny));
    const unsigned m = mat[e];
    if (m != kPEC && (int)m >= n_mat) atomicOr(&flags[0], 1);
    // elements on an absorbing face (symmetry-plane faces have no vacuum rule)
    const bool shell = (i == 0 && (abc & 1u)) || (i == g.nx - 1 && (abc & 2u)) || (j == 0 && (abc & 4u)) ||
                       (j == g.ny - 1 && (abc & 8u)) || (k == 0 && (abc & 16u)) || (k == g.nz - 1 && (abc & 32u));
    if (shell) {
        if (m == kPEC) {
            atomicOr(&flags[0], 2);
        } else if ((int)m < n_mat) {
            const uint32_t w = m < 32 ? vac0 : m < 64 ? vac1 : m < 96 ? vac2 : vac3;
            if (m >= 128 || !((w >> (m & 31)) & 1u)) atomicOr(&flags[0], 4);
        }
    }
}

__global__ void k_node_flags(const uint8_t* __restrict__ mat, Grid g, int* __restrict__ flag) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nn = (int64_t)(g.nx + 1) * (g.ny + 1) * (g.nz + 1);
    if (id >= nn) return;
    const int i = (int)(id % (g.nx + 1)), j = (int)((id / (g.nx + 1)) % (g.ny + 1));
    const int k = (int)(id / ((int64_t)(g.nx + 1) * (g.ny + 1)));
    flag[id] = node_elem_mask(mat, g, i, j, k) != 0;
}

__global__ void k_node_rank(const int* __restrict__ flag, int* __restrict__ rank, int* __restrict__ node_id,
                            int64_t nn) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= nn) return;
    // `rank` holds the exclusive scan of the flags on entry.
    const int r = rank[id];
    if (flag[id]) {
        node_id[r] = (int)id;
    } else {
        rank[id] = -1;
    }
}

__device__ __forceinline__ void node_ijk(Grid g, int id, int& i, int& j, int& k) {
    i = id % (g.nx + 1);
    j = (id / (g.nx + 1)) % (g.ny + 1);
    k = id / ((g.nx + 1) * (g.ny + 1));
}

__global__ void k_row_count(const uint8_t* __restrict__ mat, Grid g, const int* __restrict__ node_id,
                            int* __restrict__ cnt, int n_act) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_act) return;
    int i, j, k;
    node_ijk(g, node_id[r], i, j, k);
    cnt[r] = __popc(row_mask(node_elem_mask(mat, g, i, j, k)));
}

__global__ void k_col_fill(const uint8_t* __restrict__ mat, Grid g, const int* __restrict__ node_id,
                           const int* __restrict__ rank, const int* __restrict__ row_ptr, int* __restrict__ col,
                           int n_act) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_act) return;
    const int id = node_id[r];
    int i, j, k;
    node_ijk(g, id, i, j, k);
    unsigned m = row_mask(node_elem_mask(mat, g, i, j, k));
    int s = row_ptr[r];
    while (m) {
        const int l = __ffs(m) - 1;
        m &= m - 1;
        col[s++] = rank[g.node(i + l % 3 - 1, j + (l / 3) % 3 - 1, k + l / 9 - 1)];
    }
}

__global__ void k_elem_slot(const uint8_t* __restrict__ mat, Grid g, const int* __restrict__ rank,
                            const int* __restrict__ row_ptr, int* __restrict__ slot, int64_t n_el) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // (element, local a)
    if (t >= n_el * 8) return;
    const int64_t e = t >> 3;
    const int a = (int)(t & 7);
    int* out = slot + e * 64 + a * 8;
    if (mat[e] == kPEC) {
#pragma unroll
        for (int b = 0; b < 8; ++b) out[b] = -1;
        return;
    }
    const int ei = (int)(e % g.nx), ej = (int)((e / g.nx) % g.ny), ek = (int)(e / ((int64_t)g.nx * g.ny));
    const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
    const int i = ei + ax, j = ej + ay, k = ek + az;
    const unsigned m = row_mask(node_elem_mask(mat, g, i, j, k));
    const int base = row_ptr[rank[g.node(i, j, k)]];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int dx = (b & 1) - ax, dy = ((b >> 1) & 1) - ay, dz = ((b >> 2) & 1) - az;
        const int l = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
        out[b] = base + __popc(m & ((1u << l) - 1u));
    }
}

// Outer (Sext) face: a face of an active element on the outer box.  PEC face:
// a face of an active element whose neighbour across it is PEC.
__global__ void k_face_flags(const uint8_t* __restrict__ mat, Grid g, unsigned abc, int* __restrict__ fext,
                             int* __restrict__ fpec, int64_t n_el) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_el * 6) return;
    const int64_t e = t / 6;
    const int f = (int)(t - e * 6);
    const int axis = f >> 1, side = f & 1;
    const int c[3] = {(int)(e % g.nx), (int)((e / g.nx) % g.ny), (int)(e / ((int64_t)g.nx * g.ny))};
    const int dim[3] = {g.nx, g.ny, g.nz};
    const bool active = mat[e] != kPEC;
    const bool on_box = side == 0 ? c[axis] == 0 : c[axis] == dim[axis] - 1;
    int isext = active && on_box && ((abc >> f) & 1u);  // plane faces are not Sext
    int ispec = 0;
    if (active && !on_box) {
        int n[3] = {c[0], c[1], c[2]};
        n[axis] += side ? 1 : -1;
        ispec = mat[g.elem(n[0], n[1], n[2])] == kPEC;
    }
    fext[t] = isext;
    fpec[t] = ispec;
}

__global__ void k_face_compact(const int* __restrict__ flag, const int* __restrict__ pos, int* __restrict__ out,
                               int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    if (flag[t]) out[pos[t]] = (int)t;
}

static unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

static fe_status build(fe_ctx* ctx, fe_mesh* m) {
    cudaStream_t st = ctx->stream;
    const Grid g{m->nx, m->ny, m->nz};
    const int64_t nn = m->n_nodes_total, ne = m->n_el;
    int* d_small = (int*)ctx->small.ptr;
    int* h_small = ctx->h_small;

    // Vacuum materials (eps_r = mu_r = 1), as a 128-bit mask.
    uint32_t vac[4] = {0, 0, 0, 0};
    for (int q = 0; q < m->n_mat && q < 128; ++q)
        if (m->eps[q].re == 1.0 && m->eps[q].im == 0.0 && m->mu[q].re == 1.0 && m->mu[q].im == 0.0)
            vac[q >> 5] |= 1u << (q & 31);
    FE_CUDA(cudaMemsetAsync(d_small, 0, 16 * sizeof(int), st));
    k_validate<<<blocks_for(ne, 256), 256, 0, st>>>((const uint8_t*)m->material.ptr, g, m->n_mat, vac[0], vac[1],
                                                    vac[2], vac[3], abc_faces(m->boundary), d_small);
    FE_LAUNCHED();

    // Active nodes and ranks.
    DevBuf flags;
    FE_TRY(dev_alloc(st, flags, (size_t)std::max<int64_t>(nn, 6 * ne) * sizeof(int)));
    FE_TRY(dev_alloc(st, m->node_rank, nn * sizeof(int)));
    FE_TRY(dev_alloc(st, m->node_id, nn * sizeof(int)));
    int* fl = (int*)flags.ptr;
    k_node_flags<<<blocks_for(nn, 256), 256, 0, st>>>((const uint8_t*)m->material.ptr, g, fl);
    FE_LAUNCHED();
    FE_TRY(scan_exclusive(st, fl, (int*)m->node_rank.ptr, nn, d_small + 1, ctx->scan_tmp));
    k_node_rank<<<blocks_for(nn, 256), 256, 0, st>>>(fl, (int*)m->node_rank.ptr, (int*)m->node_id.ptr, nn);
    FE_LAUNCHED();
    FE_CUDA(cudaMemcpyAsync(h_small, d_small, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    FE_CUDA(cudaStreamSynchronize(st));
    if (h_small[0]) {
        dev_free(st, flags);
        if (h_small[0] & 1) {
            set_error("fe_mesh_create: material byte outside the table (and not 255)");
            return FE_ERR_INVALID_ARG;
        }
        set_error("fe_mesh_create: %s in the outer layer of elements (outer faces must be in vacuum)",
                  (h_small[0] & 2) ? "PEC" : "non-vacuum material");
        return FE_ERR_MESH;
    }
    m->n_act = h_small[1];
    FE_CUDA(cudaMemcpyAsync(h_small + 5, d_small + 5, sizeof(int), cudaMemcpyDeviceToHost, st));
    FE_CUDA(cudaStreamSynchronize(st));
    m->n_act_el = h_small[5];
    if (m->n_act == 0) {
        dev_free(st, flags);
        set_error("fe_mesh_create: no active element");
        return FE_ERR_MESH;
    }

    // Row pattern.
    FE_TRY(dev_alloc(st, m->row_ptr, (size_t)(m->n_act + 1) * sizeof(int)));
    int* rp = (int*)m->row_ptr.ptr;
    k_row_count<<<blocks_for(m->n_act, 256), 256, 0, st>>>((const uint8_t*)m->material.ptr, g,
                                                           (const int*)m->node_id.ptr, rp, m->n_act);
    FE_LAUNCHED();
    FE_TRY(scan_exclusive(st, rp, rp, m->n_act, d_small + 2, ctx->scan_tmp));
    FE_CUDA(cudaMemcpyAsync(rp + m->n_act, d_small + 2, sizeof(int), cudaMemcpyDeviceToDevice, st));

    // Faces.
    int* fext = fl;
    DevBuf fpec_flags, pos;
    FE_TRY(dev_alloc(st, fpec_flags, (size_t)(6 * ne) * sizeof(int)));
    FE_TRY(dev_alloc(st, pos, (size_t)(6 * ne) * sizeof(int)));
    k_face_flags<<<blocks_for(6 * ne, 256), 256, 0, st>>>((const uint8_t*)m->material.ptr, g,
                                                          abc_faces(m->boundary), fext, (int*)fpec_flags.ptr, ne);
    FE_LAUNCHED();
    FE_TRY(scan_exclusive(st, fext, (int*)pos.ptr, 6 * ne, d_small + 3, ctx->scan_tmp));
    FE_CUDA(cudaMemcpyAsync(h_small + 2, d_small + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    FE_CUDA(cudaStreamSynchronize(st));
    m->nnzb = h_small[2];
    m->n_ext = h_small[3];
    FE_TRY(dev_alloc(st, m->faces_ext, (size_t)m->n_ext * sizeof(int)));
    k_face_compact<<<blocks_for(6 * ne, 256), 256, 0, st>>>(fext, (const int*)pos.ptr, (int*)m->faces_ext.ptr,
                                                            6 * ne);
    FE_LAUNCHED();
    FE_TRY(scan_exclusive(st, (const int*)fpec_flags.ptr, (int*)pos.ptr, 6 * ne, d_small + 4, ctx->scan_tmp));
    FE_CUDA(cudaMemcpyAsync(h_small + 4, d_small + 4, sizeof(int), cudaMemcpyDeviceToHost, st));
    FE_CUDA(cudaStreamSynchronize(st));
    m->n_pec = h_small[4];
    FE_TRY(dev_alloc(st, m->faces_pec, (size_t)m->n_pec * sizeof(int)));
    k_face_compact<<<blocks_for(6 * ne, 256), 256, 0, st>>>((const int*)fpec_flags.ptr, (const int*)pos.ptr,
                                                            (int*)m->faces_pec.ptr, 6 * ne);
    FE_LAUNCHED();

    FE_TRY(dev_alloc(st, m->col_idx, (size_t)m->nnzb * sizeof(int)));
    k_col_fill<<<blocks_for(m->n_act, 128), 128, 0, st>>>((const uint8_t*)m->material.ptr, g,
                                                          (const int*)m->node_id.ptr, (const int*)m->node_rank.ptr,
                                                          rp, (int*)m->col_idx.ptr, m->n_act);
    FE_LAUNCHED();
    FE_TRY(dev_alloc(st, m->elem_slot, (size_t)ne * 64 * sizeof(int)));
    k_elem_slot<<<blocks_for(ne * 8, 256), 256, 0, st>>>((const uint8_t*)m->material.ptr, g,
                                                         (const int*)m->node_rank.ptr, rp,
                                                         (int*)m->elem_slot.ptr, ne);
    FE_LAUNCHED();
    dev_free(st, flags);
    dev_free(st, fpec_flags);
    dev_free(st, pos);
    m->bytes = (int64_t)(m->material.bytes + m->node_rank.bytes + m->node_id.bytes + m->row_ptr.bytes +
                         m->col_idx.bytes + m->elem_slot.bytes + m->faces_ext.bytes + m->faces_pec.bytes);
    return FE_OK;
}

static void mesh_free(fe_mesh* m) {
    cudaStream_t st = m->ctx->stream;
    for (DevBuf* b : {&m->material, &m->node_rank, &m->node_id, &m->row_ptr, &m->col_idx, &m->elem_slot,
                      &m->faces_ext, &m->faces_pec})
        dev_free(st, *b);
}

}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_mesh_create(fe_ctx* ctx, const fe_mesh_desc* d, fe_mesh** out) {
    if (!ctx || !d || !out) {
        set_error("fe_mesh_create: NULL argument");
        return FE_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || !d->material || d->n_materials < 1 || d->n_materials > 255 ||
        !d->eps_r || !d->mu_r) {
        set_error("fe_mesh_create: bad sizes, material table or NULL pointer");
        return FE_ERR_INVALID_ARG;
    }
    for (int a = 0; a < 3; ++a)
        if (!(d->h[a] > 0.0)) {
            set_error("fe_mesh_create: element size h[%d] must be > 0", a);
            return FE_ERR_INVALID_ARG;
        }
    const int64_t ne = (int64_t)d->nx * d->ny * d->nz;
    const int64_t nn = (int64_t)(d->nx + 1) * (d->ny + 1) * (d->nz + 1);
    if (ne > (int64_t)1 << 24 || nn >= (int64_t)1 << 30) {
        set_error("fe_mesh_create: grid too large (at most 2^24 elements)");
        return FE_ERR_INVALID_ARG;
    }
    for (int f = 0; f < 6; ++f)
        if (d->boundary[f] < FE_BOUNDARY_ABC || d->boundary[f] > FE_BOUNDARY_ANTISYMMETRY) {
            set_error("fe_mesh_create: boundary[%d] = %d is not a face kind (0..2)", f, d->boundary[f]);
            return FE_ERR_INVALID_ARG;
        }
    for (int q = 0; q < d->n_materials; ++q) {
        if (d->eps_r[q].re == 0.0 && d->eps_r[q].im == 0.0) {
            set_error("fe_mesh_create: eps_r[%d] is zero", q);
            return FE_ERR_INVALID_ARG;
        }
    }
    cudaSetDevice(ctx->device);
    fe_mesh* m = new (std::nothrow) fe_mesh();
    if (!m) {
        set_error("fe_mesh_create: host allocation failed");
        return FE_ERR_OOM;
    }
    m->ctx = ctx;
    m->nx = d->nx;
    m->ny = d->ny;
    m->nz = d->nz;
    for (int a = 0; a < 3; ++a) {
        m->h[a] = d->h[a];
        m->origin[a] = d->origin[a];
    }
    m->n_el = ne;
    m->n_nodes_total = nn;
    m->n_mat = d->n_materials;
    for (int f = 0; f < 6; ++f) m->boundary[f] = d->boundary[f];
    m->eps.assign(d->eps_r, d->eps_r + d->n_materials);
    m->mu.assign(d->mu_r, d->mu_r + d->n_materials);
    fe_status s = dev_alloc(ctx->stream, m->material, (size_t)ne);
    if (s == FE_OK) {
        cudaError_t e = cudaMemcpyAsync(m->material.ptr, d->material, (size_t)ne,
                                        d->material_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                        ctx->stream);
        if (e != cudaSuccess) {
            set_error("fe_mesh_create: material copy: %s", cudaGetErrorString(e));
            s = FE_ERR_CUDA;
        }
    }
    if (s == FE_OK) s = build(ctx, m);
    if (s != FE_OK) {
        mesh_free(m);
        delete m;
        return s;
    }
    *out = m;
    return FE_OK;
}

fe_status fe_mesh_info(const fe_mesh* m, fe_mesh_stats* o) {
    if (!m || !o) {
        set_error("fe_mesh_info: NULL argument");
        return FE_ERR_INVALID_ARG;
    }
    o->n_elements = m->n_el;
    o->n_nodes_total = m->n_nodes_total;
    o->n_nodes = m->n_act;
    o->n_dof = 3 * (int64_t)m->n_act;
    o->nnzb = m->nnzb;
    o->n_faces_ext = m->n_ext;
    o->n_faces_pec = m->n_pec;
    o->device_bytes = m->bytes;
    o->n_active_elements = m->n_act_el;
    return FE_OK;
}

fe_status fe_mesh_export_maps(fe_ctx* ctx, const fe_mesh* m, int32_t* node_rank, int32_t* row_ptr,
                              int32_t* col_idx, int32_t* elem_slot, int32_t* faces_ext, int32_t* faces_pec) {
    if (!ctx || !m) {
        set_error("fe_mesh_export_maps: NULL argument");
        return FE_ERR_INVALID_ARG;
    }
    cudaStream_t st = ctx->stream;
    struct Item {
        void* dst;
        const void* src;
        size_t bytes;
    } items[] = {
        {node_rank, m->node_rank.ptr, (size_t)m->n_nodes_total * 4},
        {row_ptr, m->row_ptr.ptr, (size_t)(m->n_act + 1) * 4},
        {col_idx, m->col_idx.ptr, (size_t)m->nnzb * 4},
        {elem_slot, m->elem_slot.ptr, (size_t)m->n_el * 64 * 4},
        {faces_ext, m->faces_ext.ptr, (size_t)m->n_ext * 4},
        {faces_pec, m->faces_pec.ptr, (size_t)m->n_pec * 4},
    };
    for (auto& it : items)
        if (it.dst && it.bytes) FE_CUDA(cudaMemcpyAsync(it.dst, it.src, it.bytes, cudaMemcpyDeviceToHost, st));
    FE_CUDA(cudaStreamSynchronize(st));
    return FE_OK;
}

void fe_mesh_destroy(fe_mesh* m) {
    if (!m) return;
    cudaSetDevice(m->ctx->device);
    mesh_free(m);
    delete m;
}

}  // extern "C"
