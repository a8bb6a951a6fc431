// Assembly of Eq. 4's left-hand side into 3x3-block rows.
//
// Element matrices (Eq. 1 with the Eq. 2 volume penalty) of an axis-aligned
// brick are sums of Kronecker products of three 1-D matrices,
//     M1 = h/6 [[2,1],[1,2]],  K1 = 1/h [[1,-1],[-1,1]],
//     D1[p][q] = int phi_p' phi_q = (p == 0 ? -1/2 : +1/2),
// so every entry has a closed form.  Per material one 24x24 table is built
// (k_tables), plus per face orientation the absorbing-boundary form G of
// Eq. 3 and the penalty surface term of Eq. 4.  The assembly kernel then
// follows the paper's assembly by degree of freedom (Section 3.1.2): one warp
// per node gathers, for each of the node's up to 27 blocks, the contributions
// of the elements and faces shared with the neighbour, with no atomics.  The
// symmetrisation by the transpose (Section 3.1.4, variant P) is applied to
// each face table, since (sum_e A_e)^T = sum_e A_e^T.  The same warp inverts
// the diagonal block for the block-Jacobi preconditioner.
#include "fe_internal.cuh"

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

namespace fe {

// FP32 pair of a complex128 value: hi = RN32(v), lo = RN32(v - hi) per part.
__device__ __forceinline__ float4 df_pair(double2 v) {
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    return make_float4(rh, ih, __double2float_rn(v.x - (double)rh), __double2float_rn(v.y - (double)ih));
}

struct Cx {
    double re, im;
};
__device__ __forceinline__ Cx cx(double r, double i) { return Cx{r, i}; }
__device__ __forceinline__ Cx operator+(Cx a, Cx b) { return Cx{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ Cx operator-(Cx a, Cx b) { return Cx{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ Cx operator*(Cx a, Cx b) {
    return Cx{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ Cx operator*(double s, Cx a) { return Cx{s * a.re, s * a.im}; }
__device__ __forceinline__ Cx cdiv(Cx a, Cx b) {
    const double d = b.re * b.re + b.im * b.im;
    return Cx{(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

struct TableParams {
    double h[3];
    double k0, sigma, s_pen;
    int variant;
    int n_mat;
    Cx eps[64], mu[64];
};

__device__ __forceinline__ double m1(double h, int p, int q) { return h * (p == q ? 2.0 : 1.0) / 6.0; }
__device__ __forceinline__ double k1(double h, int p, int q) { return (p == q ? 1.0 : -1.0) / h; }
__device__ __forceinline__ double d1(int p) { return p == 0 ? -0.5 : 0.5; }

// int d_g N_a d_d N_b over the brick (a, b local node indices 0..7).
__device__ double cterm(const double* h, int g, int d, int a, int b) {
    const int ac[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
    const int bc[3] = {b & 1, (b >> 1) & 1, (b >> 2) & 1};
    if (g == d) {
        double v = k1(h[g], ac[g], bc[g]);
        for (int t = 0; t < 3; ++t)
            if (t != g) v *= m1(h[t], ac[t], bc[t]);
        return v;
    }
    const int t = 3 - g - d;
    return d1(ac[g]) * d1(bc[d]) * m1(h[t], ac[t], bc[t]);
}

__device__ double mterm(const double* h, int a, int b) {
    return m1(h[0], a & 1, b & 1) * m1(h[1], (a >> 1) & 1, (b >> 1) & 1) * m1(h[2], (a >> 2) & 1, (b >> 2) & 1);
}

// Volume entry (a, al; b, be) of Eq. 1 + Eq. 2:
//   (1/eps)(delta_ab G_ab - C^{be,al}_ab) + s C^{al,be}_ab - k0^2 mu delta M_ab
__device__ Cx vol_entry(const TableParams& P, Cx inv_eps, Cx mu, int a, int al, int b, int be) {
    double cc = -cterm(P.h, be, al, a, b);
    if (al == be) cc += cterm(P.h, 0, 0, a, b) + cterm(P.h, 1, 1, a, b) + cterm(P.h, 2, 2, a, b);
    const double dd = P.s_pen * cterm(P.h, al, be, a, b);
    Cx v = cc * inv_eps + cx(dd, 0.0);
    if (al == be) v = v - (P.k0 * P.k0 * mterm(P.h, a, b)) * mu;
    return v;
}

// Absorbing boundary form of Eq. 3 on face f (weak form, transverse
// Laplacian integrated by parts):  j k0 int W_t.H_t + sigma j/(2k0) int
// grad_t W_t : grad_t H_t, only tangential components, only face nodes.
__device__ Cx abc_entry(const TableParams& P, int f, int a, int al, int b, int be) {
    const int nu = f >> 1, side = f & 1;
    const int ac[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
    const int bc[3] = {b & 1, (b >> 1) & 1, (b >> 2) & 1};
    if (al != be || al == nu || ac[nu] != side || bc[nu] != side) return cx(0, 0);
    const int t1 = nu == 0 ? 1 : 0, t2 = nu == 2 ? 1 : 2;
    const double m_1 = m1(P.h[t1], ac[t1], bc[t1]), m_2 = m1(P.h[t2], ac[t2], bc[t2]);
    const double mf = m_1 * m_2;
    const double kf = k1(P.h[t1], ac[t1], bc[t1]) * m_2 + m_1 * k1(P.h[t2], ac[t2], bc[t2]);
    return cx(0.0, P.k0 * mf + P.sigma * kf / (2.0 * P.k0));
}

// Penalty surface term of Eq. 4 on face f: -s n_al int N_a d_be N_b ds.
__device__ double pen_entry(const TableParams& P, int f, int a, int al, int b, int be) {
    const int nu = f >> 1, side = f & 1;
    const int ac[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
    const int bc[3] = {b & 1, (b >> 1) & 1, (b >> 2) & 1};
    if (al != nu || ac[nu] != side) return 0.0;
    double v = (be == nu) ? (bc[nu] == 1 ? 1.0 : -1.0) / P.h[nu] : (bc[nu] == side ? 1.0 : 0.0);
    for (int t = 0; t < 3; ++t) {
        if (t == nu) continue;
        v *= (be == t) ? d1(bc[t]) : m1(P.h[t], ac[t], bc[t]);
    }
    return -P.s_pen * (side ? 1.0 : -1.0) * v;
}

// Tables, block-major: table[(a*8 + b)*9 + al*3 + be].  Table t < n_mat is
// the volume matrix of material t; n_mat + f is the outer-face table of
// orientation f; n_mat + 6 + f the PEC-face table.
__global__ void k_tables(TableParams P, double2* __restrict__ tab) {
    const int t = blockIdx.x;
    const int idx = threadIdx.x;  // 0..575, block-major
    const int blk = idx / 9, w = idx % 9;
    const int a = blk >> 3, b = blk & 7, al = w / 3, be = w % 3;
    Cx v = cx(0, 0);
    if (t < P.n_mat) {
        v = vol_entry(P, cdiv(cx(1, 0), P.eps[t]), P.mu[t], a, al, b, be);
    } else {
        const int f = (t - P.n_mat) % 6;
        const bool ext = (t - P.n_mat) < 6;
        double pen = 0.0;
        if (P.variant == FE_VARIANT_L) {
            pen = pen_entry(P, f, a, al, b, be);
        } else if (P.variant == FE_VARIANT_P) {
            pen = 0.5 * (pen_entry(P, f, a, al, b, be) + pen_entry(P, f, b, be, a, al));
        }
        v = cx(pen, 0.0);
        if (ext) v = v + abc_entry(P, f, a, al, b, be);
    }
    tab[(size_t)t * 576 + idx] = make_double2(v.re, v.im);
}

// One warp per block row; lane l < 27 owns the block at neighbour offset
// (l % 3 - 1, (l / 3) % 3 - 1, l / 9 - 1).
__global__ void __launch_bounds__(256) k_assemble(const uint8_t* __restrict__ mat, int nx, int ny, int nz,
                                                  int n_mat, const int* __restrict__ node_id,
                                                  const int* __restrict__ row_ptr,
                                                  const double2* __restrict__ tab, double2* __restrict__ val64,
                                                  float2* __restrict__ val32, float4* __restrict__ valdf,
                                                  double2* __restrict__ dinv64, float2* __restrict__ dinv32,
                                                  float4* __restrict__ dinvdf, int n_act, int64_t stride,
                                                  unsigned abc, unsigned planes, int form_e,
                                                  int* __restrict__ status) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_act) return;
    const int id = node_id[warp];
    const int i = id % (nx + 1), j = (id / (nx + 1)) % (ny + 1), k = id / ((nx + 1) * (ny + 1));
    // elements around the node (bit ex + 2ey + 4ez: element (i-1+ex, j-1+ey, k-1+ez))
    unsigned emask = 0;
    if (lane < 8) {
        const int ex = lane & 1, ey = (lane >> 1) & 1, ez = (lane >> 2) & 1;
        const int a = i - 1 + ex, b = j - 1 + ey, c = k - 1 + ez;
        if (a >= 0 && a < nx && b >= 0 && b < ny && c >= 0 && c < nz &&
            mat[a + (int64_t)nx * (b + (int64_t)ny * c)] != kPEC)
            emask = 1;
    }
    emask = __ballot_sync(0xffffffffu, emask) & 0xFFu;
    const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
    const unsigned ax = dx < 0 ? 0x55u : dx > 0 ? 0xAAu : 0xFFu;
    const unsigned ay = dy < 0 ? 0x33u : dy > 0 ? 0xCCu : 0xFFu;
    const unsigned az = dz < 0 ? 0x0Fu : dz > 0 ? 0xF0u : 0xFFu;
    const unsigned shared = lane < 27 ? (emask & ax & ay & az) : 0u;
    const unsigned exists = __ballot_sync(0xffffffffu, shared != 0);
    if (!shared) return;
    const int slot = row_ptr[warp] + __popc(exists & ((1u << lane) - 1u));

    double2 acc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q] = make_double2(0.0, 0.0);
    unsigned sm = shared;
    while (sm) {
        const int p = __ffs(sm) - 1;
        sm &= sm - 1;
        const int ex = p & 1, ey = (p >> 1) & 1, ez = (p >> 2) & 1;
        const int ei = i - 1 + ex, ej = j - 1 + ey, ek = k - 1 + ez;
        // local indices of the row node (a) and the neighbour (b) in this element
        const int a = (1 - ex) + 2 * (1 - ey) + 4 * (1 - ez);
        const int b = (1 - ex + dx) + 2 * (1 - ey + dy) + 4 * (1 - ez + dz);
        const int64_t e = ei + (int64_t)nx * (ej + (int64_t)ny * ek);
        const int m = mat[e];
        const double2* tv = tab + (size_t)m * 576 + (a * 8 + b) * 9;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const double2 v = __ldg(tv + q);
            acc[q].x += v.x;
            acc[q].y += v.y;
        }
        // faces of this element on the outer box or against a PEC element
        const int ec[3] = {ei, ej, ek};
        const int dim[3] = {nx, ny, nz};
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            const int axis = f >> 1, side = f & 1;
            const bool on_box = side ? ec[axis] == dim[axis] - 1 : ec[axis] == 0;
            int tsel = -1;
            if (on_box) {
                if ((abc >> f) & 1u) tsel = n_mat + f;  // symmetry-plane faces carry no surface term
            } else {
                int nb[3] = {ei, ej, ek};
                nb[axis] += side ? 1 : -1;
                if (mat[nb[0] + (int64_t)nx * (nb[1] + (int64_t)ny * nb[2])] == kPEC) tsel = n_mat + 6 + f;
            }
            if (tsel >= 0) {
                const double2* fv = tab + (size_t)tsel * 576 + (a * 8 + b) * 9;
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    const double2 v = __ldg(fv + q);
                    acc[q].x += v.x;
                    acc[q].y += v.y;
                }
            }
        }
    }
    // unknowns held at zero by symmetry planes: identity rows and columns
    // (and, for E, the tangential components on conductor surfaces)
    unsigned rfix = fixed_components(i, j, k, nx, ny, nz, planes);
    unsigned cfix = fixed_components(i + dx, j + dy, k + dz, nx, ny, nz, planes);
    if (form_e) {
        rfix |= pec_held(mat, nx, ny, nz, i, j, k);
        cfix |= pec_held(mat, nx, ny, nz, i + dx, j + dy, k + dz);
    }
    if (rfix | cfix) {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const int al = q / 3, be = q % 3;
            if (((rfix >> al) & 1u) || ((cfix >> be) & 1u))
                acc[q] = make_double2(lane == 13 && al == be ? 1.0 : 0.0, 0.0);
        }
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) val64[q * stride + slot] = acc[q];
    if (val32) {
#pragma unroll
        for (int q = 0; q < 9; ++q)
            val32[q * stride + slot] = make_float2(__double2float_rn(acc[q].x), __double2float_rn(acc[q].y));
    }
    if (valdf) {
#pragma unroll
        for (int q = 0; q < 9; ++q) valdf[q * stride + slot] = df_pair(acc[q]);
    }
    if (lane == 13) {  // diagonal block: 3x3 complex inverse by cofactors
        Cx A[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) A[r][c] = cx(acc[3 * r + c].x, acc[3 * r + c].y);
        Cx C[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                C[r][c] = A[(r + 1) % 3][(c + 1) % 3] * A[(r + 2) % 3][(c + 2) % 3] -
                          A[(r + 1) % 3][(c + 2) % 3] * A[(r + 2) % 3][(c + 1) % 3];
        const Cx det = A[0][0] * C[0][0] + A[0][1] * C[0][1] + A[0][2] * C[0][2];
        if (det.re == 0.0 && det.im == 0.0) {
            atomicOr(status, kDevSingular);
            return;
        }
        const Cx inv_det = cdiv(cx(1, 0), det);
        double2* d64 = dinv64 + (size_t)warp * 9;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const Cx v = C[c][r] * inv_det;  // inverse = adjugate / det, adjugate = cofactor^T
                d64[3 * r + c] = make_double2(v.re, v.im);
                if (dinv32)
                    dinv32[(size_t)warp * 9 + 3 * r + c] =
                        make_float2(__double2float_rn(v.re), __double2float_rn(v.im));
                if (dinvdf) dinvdf[(size_t)warp * 9 + 3 * r + c] = df_pair(make_double2(v.re, v.im));
            }
    }
}

// Regular-row classes.  A row is regular when its node is interior and all
// 8 elements around it are active, of one material, and have no outer face
// and no PEC neighbour (so no face term reaches the row in any variant).
__global__ void k_row_class(const uint8_t* __restrict__ mat, int nx, int ny, int nz, const int* __restrict__ node_id,
                            int n_act, int form_e, signed char* __restrict__ cls, int* __restrict__ rep) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_act) return;
    const int id = node_id[r];
    const int i = id % (nx + 1), j = (id / (nx + 1)) % (ny + 1), k = id / ((nx + 1) * (ny + 1));
    int c = -1;
    if (i >= 2 && i <= nx - 2 && j >= 2 && j <= ny - 2 && k >= 2 && k <= nz - 2) {
        // the 8 elements and their face neighbours lie inside the box
        const int m = mat[(i - 1) + (int64_t)nx * ((j - 1) + (int64_t)ny * (k - 1))];
        bool ok = m != kPEC && m < kMaxClasses;
        for (int ez = 0; ez < 2 && ok; ++ez)
            for (int ey = 0; ey < 2 && ok; ++ey)
                for (int ex = 0; ex < 2 && ok; ++ex) {
                    const int a = i - 1 + ex, b = j - 1 + ey, cc = k - 1 + ez;
                    if (mat[a + (int64_t)nx * (b + (int64_t)ny * cc)] != m) ok = false;
                    const int nb[6][3] = {{a - 1, b, cc}, {a + 1, b, cc}, {a, b - 1, cc},
                                          {a, b + 1, cc}, {a, b, cc - 1}, {a, b, cc + 1}};
                    for (int f = 0; f < 6 && ok; ++f)
                        if (mat[nb[f][0] + (int64_t)nx * (nb[f][1] + (int64_t)ny * nb[f][2])] == kPEC) ok = false;
                }
        // E: no neighbour on a conductor surface either (its held columns would
        // differ from the class stencil): no PEC in the 4 x 4 x 4 elements around
        for (int ez = -2; ez < 2 && ok && form_e; ++ez)
            for (int ey = -2; ey < 2 && ok; ++ey)
                for (int ex = -2; ex < 2 && ok; ++ex)
                    if (mat[(i + ex) + (int64_t)nx * ((j + ey) + (int64_t)ny * (k + ez))] == kPEC) ok = false;
        if (ok) c = m;
    }
    cls[r] = (signed char)c;
    if (c >= 0) atomicMin(&rep[c], r);
}

// One warp per class: copies the 27 blocks of the class's first regular row
// (bitwise the values every regular row of the class carries) and classifies
// them.  Entries below 1e-15 of the largest are treated as zero.
__global__ void k_class_stencil(const double2* __restrict__ val64, int64_t stride, const int* __restrict__ row_ptr,
                                const int* __restrict__ rep, StencilSet* __restrict__ S) {
    const int c = blockIdx.x, lane = threadIdx.x;
    const int r = rep[c];
    const bool has = r != 0x7fffffff;
    double2 v[9];
    double amax = 0.0;
    if (has && lane < 27) {
        const int slot = row_ptr[r] + lane;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            v[q] = val64[q * stride + slot];
            amax = fmax(amax, fmax(fabs(v[q].x), fabs(v[q].y)));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    const double tiny = 1e-15 * amax;
    int diag_real = 1;
    if (has && lane < 27) {
#pragma unroll
        for (int al = 0; al < 3; ++al)
#pragma unroll
            for (int be = 0; be < 3; ++be) {
                const double2 e = v[3 * al + be];
                if (fabs(e.y) > tiny || (al != be && fabs(e.x) > tiny)) diag_real = 0;
            }
    }
    diag_real = __all_sync(0xffffffffu, diag_real);
    if (has && lane < 27) {
#pragma unroll
        for (int al = 0; al < 3; ++al) {
#pragma unroll
            for (int be = 0; be < 3; ++be) {
                const double2 e = v[3 * al + be];
                S->s64[c][al][lane][be] = e;
                S->s32[c][al][lane][be] = make_float2(__double2float_rn(e.x), __double2float_rn(e.y));
                S->sdf[c][al][lane][be] = df_pair(e);
            }
            S->dval[c][al][lane] = v[4 * al].x;
            S->dval32[c][al][lane] = __double2float_rn(v[4 * al].x);
            const float dh = __double2float_rn(v[4 * al].x);
            S->dvaldf[c][al][lane] = make_float2(dh, __double2float_rn(v[4 * al].x - (double)dh));
        }
    }
    if (lane == 0) S->kind[c] = has ? (diag_real ? 2 : 1) : 0;
}

// Rows on each product path: counts[0] general-stencil rows, counts[1] real
// diagonal stencil rows, counts[2] blocks of the explicit rows.
__global__ void k_class_counts(const signed char* __restrict__ cls, const StencilSet* __restrict__ S,
                               const int* __restrict__ row_ptr, int n_act, unsigned long long* __restrict__ counts) {
    unsigned long long c1 = 0, c2 = 0, cb = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_act; r += gridDim.x * blockDim.x) {
        const int c = cls[r];
        const int kind = c >= 0 ? S->kind[c] : 0;
        c1 += kind == 1;
        c2 += kind == 2;
        cb += kind == 0 ? (unsigned long long)(row_ptr[r + 1] - row_ptr[r]) : 0ull;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c1 += __shfl_xor_sync(0xffffffffu, c1, o);
        c2 += __shfl_xor_sync(0xffffffffu, c2, o);
        cb += __shfl_xor_sync(0xffffffffu, cb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(counts, c1);
        atomicAdd(counts + 1, c2);
        atomicAdd(counts + 2, cb);
    }
}

// Per-row product cost: w_block per stored block of an explicit row,
// w_general for a general-stencil row, w_diagonal for a diagonal-stencil row.
__global__ void k_row_cost(const signed char* __restrict__ cls, const StencilSet* __restrict__ S,
                           const int* __restrict__ row_ptr, int n_act, int w_block, int w_general, int w_diagonal,
                           int* __restrict__ cost) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_act) return;
    const int c = cls[r];
    const int kind = c >= 0 ? S->kind[c] : 0;
    cost[r] = kind == 2 ? w_diagonal : (kind == 1 ? w_general : w_block * (row_ptr[r + 1] - row_ptr[r]));
}

// the half storage (half.cu) lives beside the system and goes with it
void half_release(const fe_system* s);
int64_t half_bytes(const fe_system* s);

static void system_free(fe_system* s) {
    half_release(s);
    cudaStream_t st = s->ctx->stream;
    for (DevBuf* b : {&s->tables, &s->val64, &s->val32, &s->valdf, &s->dinv64, &s->dinv32, &s->dinvdf,
                      &s->row_class, &s->stencil, &s->cost_prefix, &s->cost_prefix_alu, &s->expl_prefix, &s->dict_idx,
                      &s->dict_vals, &s->bicp_l,
                      &s->bicp_linv, &s->bicp_tpos, &s->bicp_tab, &s->bicp_lev, &s->bicp_nlev})
        dev_free(st, *b);
    s->bicp_n_sub = 0;
    s->n_dict = 0;
}

}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_assemble(fe_ctx* ctx, const fe_mesh* m, double freq_hz, int32_t precision, fe_system** out) {
    if (!ctx || !m || !out) {
        set_error("fe_assemble: NULL argument");
        return FE_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!(freq_hz > 0.0) || (precision != FE_PREC_FP64 && precision != FE_PREC_MIXED && precision != FE_PREC_DF)) {
        set_error("fe_assemble: frequency must be > 0 and precision FP64, MIXED or DF");
        return FE_ERR_INVALID_ARG;
    }
    if (m->n_mat > 64) {
        set_error("fe_assemble: at most 64 materials are supported");
        return FE_ERR_UNSUPPORTED;
    }
    cudaSetDevice(ctx->device);
    fe_system* s = new (std::nothrow) fe_system();
    if (!s) {
        set_error("fe_assemble: host allocation failed");
        return FE_ERR_OOM;
    }
    s->ctx = ctx;
    s->mesh = m;
    s->freq = freq_hz;
    s->k0 = 2.0 * kPi * freq_hz / kC0;
    s->precision = precision;
    s->variant = ctx->opt.variant;
    s->formulation = ctx->opt.formulation;
    s->sigma = ctx->opt.abc_sigma;
    s->s_pen = ctx->opt.penalty_s;
    cudaStream_t st = ctx->stream;
    auto fail = [&](fe_status e) {
        system_free(s);
        delete s;
        return e;
    };
    fe_status e;
    const int n_tab = m->n_mat + 12;
    if ((e = dev_alloc(st, s->tables, (size_t)n_tab * 576 * sizeof(double2))) != FE_OK) return fail(e);
    s->stride = ((int64_t)m->nnzb + 63) / 64 * 64;
    if ((e = dev_alloc(st, s->val64, (size_t)s->stride * 9 * sizeof(double2))) != FE_OK) return fail(e);
    if ((e = dev_alloc(st, s->dinv64, (size_t)m->n_act * 9 * sizeof(double2))) != FE_OK) return fail(e);
    if (precision == FE_PREC_MIXED) {
        if ((e = dev_alloc(st, s->val32, (size_t)s->stride * 9 * sizeof(float2))) != FE_OK) return fail(e);
        if ((e = dev_alloc(st, s->dinv32, (size_t)m->n_act * 9 * sizeof(float2))) != FE_OK) return fail(e);
    }
    if (precision == FE_PREC_DF) {
        if ((e = dev_alloc(st, s->valdf, (size_t)s->stride * 9 * sizeof(float4))) != FE_OK) return fail(e);
        if ((e = dev_alloc(st, s->dinvdf, (size_t)m->n_act * 9 * sizeof(float4))) != FE_OK) return fail(e);
    }
    TableParams P{};
    for (int a = 0; a < 3; ++a) P.h[a] = m->h[a];
    P.k0 = s->k0;
    P.sigma = s->sigma;
    P.s_pen = s->s_pen;
    P.variant = s->variant;
    P.n_mat = m->n_mat;
    for (int q = 0; q < m->n_mat; ++q) {
        // the E formulation is the H formulation with the material roles exchanged
        const fe_complex& ce = s->formulation == FE_FORMULATION_E ? m->mu[q] : m->eps[q];
        const fe_complex& cm = s->formulation == FE_FORMULATION_E ? m->eps[q] : m->mu[q];
        P.eps[q] = Cx{ce.re, ce.im};
        P.mu[q] = Cx{cm.re, cm.im};
    }
    int* d_status = (int*)ctx->small.ptr + 8;
    cudaMemsetAsync(d_status, 0, sizeof(int), st);
    k_tables<<<n_tab, 576, 0, st>>>(P, (double2*)s->tables.ptr);
    {
        count_launches(1);
        cudaError_t ce = cudaGetLastError();
        if (ce != cudaSuccess) {
            set_error("k_tables launch: %s", cudaGetErrorString(ce));
            return fail(FE_ERR_CUDA);
        }
    }
    const int threads = 256;
    const unsigned blocks = (unsigned)(((int64_t)m->n_act * 32 + threads - 1) / threads);
    k_assemble<<<blocks, threads, 0, st>>>((const uint8_t*)m->material.ptr, m->nx, m->ny, m->nz, m->n_mat,
                                           (const int*)m->node_id.ptr, (const int*)m->row_ptr.ptr,
                                           (const double2*)s->tables.ptr, (double2*)s->val64.ptr,
                                           (float2*)s->val32.ptr, (float4*)s->valdf.ptr, (double2*)s->dinv64.ptr,
                                           (float2*)s->dinv32.ptr, (float4*)s->dinvdf.ptr, m->n_act, s->stride,
                                           abc_faces(m->boundary), pack_planes(m->boundary),
                                           s->formulation == FE_FORMULATION_E ? 1 : 0, d_status);
    {
        count_launches(1);
        cudaError_t ce = cudaGetLastError();
        if (ce != cudaSuccess) {
            set_error("k_assemble launch: %s", cudaGetErrorString(ce));
            return fail(FE_ERR_CUDA);
        }
    }
    // regular-row classes and their stencils
    if ((e = dev_alloc(st, s->row_class, (size_t)m->n_act)) != FE_OK) return fail(e);
    if ((e = dev_alloc(st, s->stencil, sizeof(StencilSet))) != FE_OK) return fail(e);
    int* d_rep = (int*)ctx->small.ptr + 16;  // kMaxClasses ints
    {
        std::vector<int> big(kMaxClasses, 0x7fffffff);
        cudaMemcpyAsync(d_rep, big.data(), kMaxClasses * sizeof(int), cudaMemcpyHostToDevice, st);
        k_row_class<<<(unsigned)((m->n_act + 255) / 256), 256, 0, st>>>(
            (const uint8_t*)m->material.ptr, m->nx, m->ny, m->nz, (const int*)m->node_id.ptr, m->n_act,
            s->formulation == FE_FORMULATION_E ? 1 : 0, (signed char*)s->row_class.ptr, d_rep);
        count_launches(1);
        k_class_stencil<<<kMaxClasses, 32, 0, st>>>((const double2*)s->val64.ptr, s->stride,
                                                    (const int*)m->row_ptr.ptr, d_rep, (StencilSet*)s->stencil.ptr);
        count_launches(1);
        // product cost prefixes, in units of one stored block of an explicit
        // row: a general-stencil row costs 18 (complex64) or 27 (FP32 pairs,
        // read through the block dictionary like an explicit row) such
        // blocks, a diagonal-stencil row 10 or 9 (per-CTA product times
        // measured on GB300 and fitted to these three row kinds)
        // The third prefix counts the stored blocks of explicit rows only: a
        // solve CTA packs its explicit rows' values at 9 times that prefix.
        const int weights[3][3] = {{1, 18, 10}, {1, 27, 9}, {1, 0, 0}};
        DevBuf* bufs[3] = {&s->cost_prefix, &s->cost_prefix_alu, &s->expl_prefix};
        int* d_total = (int*)ctx->small.ptr + 24;
        for (int k = 0; k < 3; ++k) {
            if ((e = dev_alloc(st, *bufs[k], (size_t)(m->n_act + 1) * sizeof(int))) != FE_OK) return fail(e);
            int* cp = (int*)bufs[k]->ptr;
            k_row_cost<<<(unsigned)((m->n_act + 255) / 256), 256, 0, st>>>(
                (const signed char*)s->row_class.ptr, (const StencilSet*)s->stencil.ptr, (const int*)m->row_ptr.ptr,
                m->n_act, weights[k][0], weights[k][1], weights[k][2], cp);
            count_launches(1);
            if ((e = scan_exclusive(st, cp, cp, m->n_act, d_total + k, ctx->scan_tmp)) != FE_OK) return fail(e);
            cudaMemcpyAsync(cp + m->n_act, d_total + k, sizeof(int), cudaMemcpyDeviceToDevice, st);
        }
        unsigned long long* d_counts = (unsigned long long*)((int*)ctx->small.ptr + 32);
        cudaMemsetAsync(d_counts, 0, 3 * sizeof(unsigned long long), st);
        k_class_counts<<<std::max(1, std::min(1024, (m->n_act + 255) / 256)), 256, 0, st>>>(
            (const signed char*)s->row_class.ptr, (const StencilSet*)s->stencil.ptr, (const int*)m->row_ptr.ptr,
            m->n_act, d_counts);
        count_launches(1);
        cudaMemcpyAsync(ctx->h_small + 24, d_total, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(ctx->h_small + 32, d_counts, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
        cudaError_t ce = cudaStreamSynchronize(st);  // `big` must outlive the copy
        if (ce != cudaSuccess) {
            set_error("regular-row classes: %s", cudaGetErrorString(ce));
            return fail(FE_ERR_CUDA);
        }
        s->cost_total = ctx->h_small[24];
        s->cost_total_alu = ctx->h_small[25];
        // bounds of one row's cost (an explicit row has 8 to 27 blocks)
        for (int k = 0; k < 2; ++k) {
            s->cost_min[k] = std::min({8 * weights[k][0], weights[k][1], weights[k][2]});
            s->cost_max[k] = std::max({27 * weights[k][0], weights[k][1], weights[k][2]});
        }
        const unsigned long long* hc = (const unsigned long long*)(ctx->h_small + 32);
        s->rows_general = (int64_t)hc[0];
        s->rows_diagonal = (int64_t)hc[1];
        s->blocks_explicit = (int64_t)hc[2];
    }
    if ((e = build_block_dict(ctx, s)) != FE_OK) return fail(e);
    *out = s;
    return FE_OK;
}

fe_status fe_system_info(const fe_system* s, fe_system_stats* out) {
    if (!s || !out) {
        set_error("fe_system_info: NULL argument");
        return FE_ERR_INVALID_ARG;
    }
    const fe_mesh* m = s->mesh;
    out->precision = s->precision;
    out->dict_blocks = s->n_dict;
    out->n_rows = m->n_act;
    out->nnzb = m->nnzb;
    out->rows_general = s->rows_general;
    out->rows_diagonal = s->rows_diagonal;
    out->blocks_explicit = s->blocks_explicit;
    int64_t bytes = 0;
    for (const DevBuf* b : {&s->tables, &s->val64, &s->val32, &s->valdf, &s->dinv64, &s->dinv32, &s->dinvdf,
                            &s->row_class, &s->stencil, &s->cost_prefix, &s->cost_prefix_alu, &s->expl_prefix,
                            &s->dict_idx, &s->dict_vals, &s->bicp_l,
                            &s->bicp_linv, &s->bicp_tpos, &s->bicp_tab, &s->bicp_lev, &s->bicp_nlev})
        bytes += (int64_t)b->bytes;
    out->device_bytes = bytes + half_bytes(s);
    return FE_OK;
}

fe_status fe_system_export_df(fe_ctx* ctx, const fe_system* s, void* vals_df) {
    if (!ctx || !s || !vals_df) {
        set_error("fe_system_export_df: NULL argument");
        return FE_ERR_INVALID_ARG;
    }
    if (!s->valdf.ptr) {
        set_error("fe_system_export_df: no FP32-pair copy (system not assembled with FE_PREC_DF)");
        return FE_ERR_INVALID_ARG;
    }
    cudaStream_t st = ctx->stream;
    const fe_mesh* m = s->mesh;
    std::vector<float4> tmp((size_t)s->stride * 9);
    FE_CUDA(cudaMemcpyAsync(tmp.data(), s->valdf.ptr, tmp.size() * sizeof(float4), cudaMemcpyDeviceToHost, st));
    FE_CUDA(cudaStreamSynchronize(st));
    float4* out = (float4*)vals_df;
    for (int64_t b = 0; b < m->nnzb; ++b)
        for (int q = 0; q < 9; ++q) out[(size_t)b * 9 + q] = tmp[(size_t)q * s->stride + b];
    return FE_OK;
}

fe_status fe_system_export(fe_ctx* ctx, const fe_system* s, void* vals_c128, void* vals_c64, void* dinv_c128) {
    if (!ctx || !s) {
        set_error("fe_system_export: NULL argument");
        return FE_ERR_INVALID_ARG;
    }
    if (vals_c64 && !s->val32.ptr) {
        set_error("fe_system_export: no complex64 copy (system assembled in FP64)");
        return FE_ERR_INVALID_ARG;
    }
    cudaStream_t st = ctx->stream;
    const fe_mesh* m = s->mesh;
    // planes -> [nnzb][9] (host-side reorder; export is for checks, not the hot path)
    auto export_planes = [&](void* dst, const void* src, size_t elem) -> fe_status {
        std::vector<char> tmp((size_t)s->stride * 9 * elem);
        FE_CUDA(cudaMemcpyAsync(tmp.data(), src, tmp.size(), cudaMemcpyDeviceToHost, st));
        FE_CUDA(cudaStreamSynchronize(st));
        char* out = (char*)dst;
        for (int64_t b = 0; b < m->nnzb; ++b)
            for (int q = 0; q < 9; ++q)
                memcpy(out + ((size_t)b * 9 + q) * elem, tmp.data() + ((size_t)q * s->stride + b) * elem, elem);
        return FE_OK;
    };
    if (vals_c128) FE_TRY(export_planes(vals_c128, s->val64.ptr, sizeof(double2)));
    if (vals_c64) FE_TRY(export_planes(vals_c64, s->val32.ptr, sizeof(float2)));
    if (dinv_c128)
        FE_CUDA(cudaMemcpyAsync(dinv_c128, s->dinv64.ptr, (size_t)m->n_act * 9 * sizeof(double2),
                                cudaMemcpyDeviceToHost, st));
    FE_CUDA(cudaStreamSynchronize(st));
    return FE_OK;
}

void fe_system_destroy(fe_system* s) {
    if (!s) return;
    cudaSetDevice(s->ctx->device);
    system_free(s);
    delete s;
}

}  // extern "C"
