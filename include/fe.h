/*
 * fe.h - C ABI of the GB300 nodal finite-element H-field scattering solver.
 *
 * The library assembles and solves the time-harmonic total-field H
 * formulation of Vollaire, Nicolas & Nicolas, "Parallel computing for the
 * finite element method" (Section 2, Eqs. 1-4): curl-curl with 1/eps_r, the
 * grad-div penalty (Eq. 2), the -k0^2 mu_r mass term, the second-order
 * Engquist-Majda absorbing condition on the rectangular outer faces (Eq. 3),
 * PEC surfaces, and the incident plane-wave right-hand side of Eq. 4.
 * Geometry is a voxel box of first-order (trilinear) hexahedra.  Unknowns are
 * the three Cartesian H components at every active node ("three lines per
 * node", Section 3.1.2), stored as a 3x3-block sparse row matrix.  A box face
 * may instead be a symmetry or antisymmetry plane (Section 3.1.3, Eqs.
 * 6a/6b), and a context may solve for the total E field instead of H
 * (Section 2; n x E = 0 held on conductors).
 *
 * Conventions used by every call
 *   - Units SI, time dependence e^{j omega t}, c0 = 299 792 458 m/s,
 *     k0 = 2 pi f / c0.
 *   - Element (i,j,k) id = i + nx*(j + ny*k); node (i,j,k) id =
 *     i + (nx+1)*(j + (ny+1)*k); local node a = ix + 2*iy + 4*iz.
 *   - Active element: material byte != 255 (255 = PEC, not meshed).
 *     Active node: touches at least one active element.  Active nodes are
 *     ranked by increasing node id; dof = 3*rank + component (x, y, z).
 *   - Block pattern: block (n, m) exists iff nodes n and m share an active
 *     element; col_idx ascending within each block row, diagonal included.
 *   - Faces are encoded 6*element + face, face 0..5 = -x, +x, -y, +y, -z, +z,
 *     listed in ascending order.
 *   - Complex numbers are interleaved (re, im) pairs: complex128 = two
 *     doubles, complex64 = two floats.  A block is stored row-major:
 *     value (alpha, beta) of block s at [9*s + 3*alpha + beta].
 *   - Multi-right-hand-side vectors are laid out [n_dof][nrhs] (the nrhs
 *     values of one dof are contiguous).
 *
 * Ownership and errors
 *   - Every opaque handle and every device buffer the library allocates is
 *     owned by the library and freed by the matching *_destroy call.
 *   - Caller buffers (host or device) are only read or written during the
 *     call that receives them; the call returns once they are no longer used
 *     (device outputs are complete on the context's stream).
 *   - Every call returns an fe_status.  No exception or abort crosses the
 *     ABI.  fe_last_error() returns a thread-local message for the last
 *     failing call of the calling thread.
 *   - All GPU work of a context runs on the CUDA stream given in fe_options
 *     (NULL: a stream the context creates).  Calls on one context must not
 *     overlap in time from different host threads.
 */
#ifndef FE_H
#define FE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fe_status {
    FE_OK = 0,
    FE_PENDING = 1,            /* fe_serve_poll: request not finished yet */
    FE_ERR_INVALID_ARG = -1,   /* a NULL handle, a size out of range, ... */
    FE_ERR_MESH = -2,          /* mesh rules broken (PEC or a non-vacuum material on the outer box) */
    FE_ERR_OOM = -3,           /* a device or host allocation failed, or admission budget exceeded */
    FE_ERR_BREAKDOWN = -4,     /* Krylov breakdown (p^T A p or r^T z vanished) */
    FE_ERR_NOT_CONVERGED = -5, /* iteration limits reached above tolerance */
    FE_ERR_TIMEOUT = -6,       /* a bounded device-side wait (grid barrier) expired */
    FE_ERR_CUDA = -7,          /* a CUDA runtime call failed */
    FE_ERR_UNSUPPORTED = -8    /* option combination not built */
} fe_status;

typedef struct fe_complex {
    double re, im;
} fe_complex;

typedef enum fe_variant {
    FE_VARIANT_S = 0, /* a + G: volume terms + ABC; complex symmetric (default) */
    FE_VARIANT_L = 1, /* a + L + G: the literal Eq. 4 with the penalty surface term; non-symmetric */
    FE_VARIANT_P = 2  /* (A_L + A_L^T)/2: the paper's symmetrisation by the transpose (Section 3.1.4) */
} fe_variant;

typedef enum fe_precision {
    FE_PREC_FP64 = 0,  /* plain method: complex128 matrix, complex128 Krylov loop */
    FE_PREC_MIXED = 1, /* complex64 Krylov loop inside FP64 iterative refinement */
    FE_PREC_DF = 2     /* the Krylov loop on FP32 pairs ("double-float", about 48 significant bits:
                          hi = RN32(v), lo = RN32(v - hi), products and sums by error-free
                          transformations on the FP32 pipes): products, vectors, inner products and
                          the recurrence scalars; the true residual, the refinement and the solution
                          FP64.  Converges like FE_PREC_FP64 on well-behaved systems (a few percent
                          more iterations) */
} fe_precision;

/* The field solved for (Section 2: every step of the H formulation applies
 * to E as well).  FE_FORMULATION_E puts 1/mu_r in the curl-curl term and
 * eps_r in the mass term, and holds n x E = 0 on conductor surfaces
 * (Section 3.1.3): the tangential E components at nodes on PEC surfaces are
 * fixed at zero (at PEC edges and corners all three).  Plane waves then give
 * the incident E (p_hat its polarisation), the solution is the total E, and
 * the symmetry-plane kinds refer to E. */
typedef enum fe_formulation {
    FE_FORMULATION_H = 0,
    FE_FORMULATION_E = 1
} fe_formulation;

typedef struct fe_options {
    void* stream;      /* cudaStream_t for all work of the context; NULL = context-owned stream */
    int32_t variant;   /* fe_variant; default FE_VARIANT_S */
    double abc_sigma;  /* weight of the transverse ABC term: +1 Eq. 3 as printed (default, absorbing for every mode), -1 Taylor sign, 0 first order */
    double penalty_s;  /* grad-div penalty coefficient s (Eq. 2); default 1 */
    int32_t formulation; /* fe_formulation; default FE_FORMULATION_H */
} fe_options;

/* Fills *opt with the defaults above. */
void fe_options_default(fe_options* opt);

typedef struct fe_ctx fe_ctx;
typedef struct fe_mesh fe_mesh;
typedef struct fe_system fe_system;
typedef struct fe_server fe_server;

/* Creates a context on CUDA device `cuda_device`.  opt may be NULL (defaults).
 * Errors: FE_ERR_INVALID_ARG (out == NULL, bad option), FE_ERR_CUDA. */
fe_status fe_ctx_create(fe_ctx** out, int cuda_device, const fe_options* opt);
void fe_ctx_destroy(fe_ctx* ctx);
/* Blocks until all work queued on the context's stream has finished.
 * Errors: FE_ERR_INVALID_ARG (NULL), FE_ERR_CUDA (an earlier kernel failed). */
fe_status fe_ctx_synchronize(fe_ctx* ctx);

/* ------------------------------------------------------------------------
 * Mesh and block pattern (Section 3.1.2 storage by node rows; Section 4.2.1
 * structure of the global matrix).  Built on the device by the library's
 * kernels; the caller's description is copied.
 * ---------------------------------------------------------------------- */
/* Kind of a box face (Section 3.1.3).  A symmetry or antisymmetry plane
 * replaces the absorbing condition on that face and lets the box hold one half
 * (or quarter, eighth) of a mirror-symmetric problem: the face carries no
 * surface term, may cut through the scatterer, and the held components at its
 * nodes are fixed at zero (identity rows, zero right-hand side). */
typedef enum fe_boundary {
    FE_BOUNDARY_ABC = 0,          /* second-order absorbing condition (Eq. 3); the face's elements must be vacuum */
    FE_BOUNDARY_SYMMETRY = 1,     /* symmetry plane: n . H = 0 (Eq. 6a), the normal component is held */
    FE_BOUNDARY_ANTISYMMETRY = 2  /* antisymmetry plane: n x H = 0 (Eq. 6b), the tangential components are held */
} fe_boundary;

typedef struct fe_mesh_desc {
    int32_t nx, ny, nz;          /* elements per axis, each >= 1 */
    double h[3];                 /* element edge lengths (m), > 0 */
    double origin[3];            /* world position of node (0,0,0) (m) */
    const uint8_t* material;     /* nx*ny*nz bytes indexed by element id; < n_materials or 255 (PEC) */
    int32_t material_on_device;  /* 0: host pointer; 1: device pointer (read on the context stream) */
    int32_t n_materials;         /* 1..255 entries in eps_r / mu_r */
    const fe_complex* eps_r;     /* host, n_materials relative permittivities (eps' - j eps'' for losses) */
    const fe_complex* mu_r;      /* host, n_materials relative permeabilities */
    int32_t boundary[6];         /* fe_boundary of the faces -x, +x, -y, +y, -z, +z (all zero: absorbing box) */
} fe_mesh_desc;

typedef struct fe_mesh_stats {
    int64_t n_elements, n_active_elements;
    int64_t n_nodes_total, n_nodes; /* all grid nodes / active nodes (block rows) */
    int64_t n_dof;                  /* 3 * n_nodes */
    int64_t nnzb;                   /* number of 3x3 blocks */
    int64_t n_faces_ext, n_faces_pec;
    int64_t device_bytes;           /* device memory held by the mesh */
} fe_mesh_stats;

/* Validates the description and builds every integer map on the device.
 * Errors: FE_ERR_INVALID_ARG (sizes, NULL pointers, material byte outside
 * the table, boundary kind outside 0..2), FE_ERR_MESH (PEC or non-vacuum
 * material in the outer layer of elements of an absorbing face, i.e. an
 * absorbing face not in free space), FE_ERR_OOM, FE_ERR_CUDA. */
fe_status fe_mesh_create(fe_ctx* ctx, const fe_mesh_desc* d, fe_mesh** out);
fe_status fe_mesh_info(const fe_mesh* m, fe_mesh_stats* out);
/* Copies the integer maps to caller-allocated HOST buffers; any pointer may
 * be NULL to skip that map.  Sizes: node_rank[n_nodes_total] (-1 = inactive),
 * row_ptr[n_nodes + 1], col_idx[nnzb], elem_slot[n_elements*64] (slot of block
 * (local a, local b) of element e at [64e + 8a + b], -1 for PEC elements),
 * faces_ext[n_faces_ext], faces_pec[n_faces_pec]. */
fe_status fe_mesh_export_maps(fe_ctx* ctx, const fe_mesh* m, int32_t* node_rank, int32_t* row_ptr,
                              int32_t* col_idx, int32_t* elem_slot, int32_t* faces_ext,
                              int32_t* faces_pec);
void fe_mesh_destroy(fe_mesh* m);

/* ------------------------------------------------------------------------
 * Assembly (Section 3.1.2, assembly by degree of freedom: each block row
 * gathers the contributions of the elements and faces around its node; the
 * variant's symmetrisation, Section 3.1.4, is applied element by element).
 * Also builds the 3x3 block-Jacobi inverse (the block form of the diagonal
 * preconditioning of Section 3.1.5.1) and, for FE_PREC_MIXED, the
 * round-to-nearest complex64 copies of the matrix and of the inverse; for
 * FE_PREC_DF, the FP32-pair copy of the matrix.
 * ---------------------------------------------------------------------- */
/* Errors: FE_ERR_INVALID_ARG (freq_hz <= 0, bad precision), FE_ERR_OOM, FE_ERR_CUDA. */
fe_status fe_assemble(fe_ctx* ctx, const fe_mesh* m, double freq_hz, int32_t precision, fe_system** out);
/* Copies values to caller-allocated HOST buffers (any may be NULL):
 * vals_c128[nnzb*9*2 doubles], vals_c64[nnzb*9*2 floats] (FE_PREC_MIXED only,
 * else FE_ERR_INVALID_ARG), dinv_c128[n_nodes*9*2 doubles]. */
fe_status fe_system_export(fe_ctx* ctx, const fe_system* s, void* vals_c128, void* vals_c64, void* dinv_c128);
/* Block dictionary (complex64 and FP32-pair systems): equal local
 * configurations of the voxel mesh give bitwise equal 3x3 blocks, so the
 * system also keeps each distinct block once (at most 4096 of them) with an
 * index per stored block; single-column solves read explicit rows through it
 * when it fits in shared memory.  dict_blocks counts the distinct blocks, 0
 * when there are too many (the products then read the stored values).
 *
 * Regular rows (interior nodes whose eight elements are active, of one
 * material, with no outer or PEC face) all carry the same 27 blocks per
 * material; the Krylov products read them from a per-material stencil instead
 * of the stored blocks.  The counts say how many rows take each path. */
typedef struct fe_system_stats {
    int32_t precision;         /* as assembled */
    int32_t dict_blocks;       /* distinct 3x3 blocks in the block dictionary (0: none) */
    int64_t n_rows, nnzb;      /* block rows, stored blocks */
    int64_t rows_general;      /* regular rows with a general 3x3-block stencil */
    int64_t rows_diagonal;     /* regular rows whose stencil blocks are real multiples of I3 */
    int64_t blocks_explicit;   /* stored blocks of the other (explicit) rows */
    int64_t device_bytes;      /* device memory held by the system */
} fe_system_stats;
fe_status fe_system_info(const fe_system* s, fe_system_stats* out);
/* Copies the FP32-pair values of a system assembled with FE_PREC_DF to a
 * caller-allocated HOST buffer vals_df[nnzb*9*4 floats]: per entry
 * (re_hi, im_hi, re_lo, im_lo), block-major as vals_c128.  Errors:
 * FE_ERR_INVALID_ARG (NULL, or the system has no FP32-pair copy). */
fe_status fe_system_export_df(fe_ctx* ctx, const fe_system* s, void* vals_df);

/* Block incomplete Cholesky preconditioner, BICP (Section 3.1.5.3; the
 * factor of Section 3.1.5.2, Eq. 5; its application by the forward and back
 * substitutions of Eq. 6).  The node rows are split into n_sub contiguous
 * bands, band b holding nodes floor(b n / n_sub) <= I < floor((b+1) n / n_sub)
 * (n = active nodes); each band gets the incomplete Cholesky factor of its
 * own diagonal block on the lower 3x3-block pattern of A, unconjugated
 * (A ~ L L^T, L L^T = A on every stored block of the band), and couplings
 * between bands are dropped.  The persistent solve runs one CTA per band, so
 * a solve with fe_solve_opts.preconditioner = FE_PRECOND_BICP needs a factor
 * with as many bands as its grid: n_sub = 0 picks that number, min(SMs, n).
 * The factor is FP64 and is used by FE_PREC_FP64 solves.  It is built on the
 * device (one thread per band) and kept with the system (16 B x 9 per stored
 * block, plus index arrays); a new call replaces it.
 * Errors: FE_ERR_INVALID_ARG (NULL, no rows, variant L, which is not
 * symmetric, n_sub outside [0, n]),
 * FE_ERR_BREAKDOWN (a pivot is zero or not finite; no factor is kept),
 * FE_ERR_OOM, FE_ERR_CUDA. */
fe_status fe_system_factor_bicp(fe_ctx* ctx, fe_system* s, int32_t n_sub);

/* Copies the factor to the host: l_c128 (optional) complex128 [nnzb][3][3]
 * in block-slot order: L_IJ at the slot of block (I, J) for J < I in I's
 * band, the lower triangular L_II at the diagonal slot, zeros elsewhere;
 * n_sub (optional) receives the number of bands.  Errors:
 * FE_ERR_INVALID_ARG (NULL, or no factor), FE_ERR_CUDA. */
fe_status fe_system_export_bicp(fe_ctx* ctx, const fe_system* s, void* l_c128, int32_t* n_sub);
void fe_system_destroy(fe_system* s);

/* ------------------------------------------------------------------------
 * Right-hand side (Eq. 4): b(W) = G(W, H_i) - int_Sext W.(n x curl H_i) ds
 * with H_i = p_hat * amplitude * exp(-j k0 k_hat . r).
 * ---------------------------------------------------------------------- */
typedef struct fe_planewave {
    double k_hat[3];      /* unit propagation direction */
    double p_hat[3];      /* unit H polarisation, orthogonal to k_hat */
    fe_complex amplitude; /* H0 (A/m) */
} fe_planewave;

/* b_out: complex128 [n_dof][nrhs]; host buffer, or device when on_device = 1.
 * Errors: FE_ERR_INVALID_ARG (nrhs < 1, NULL), FE_ERR_OOM, FE_ERR_CUDA. */
fe_status fe_rhs(fe_ctx* ctx, const fe_system* s, int32_t nrhs, const fe_planewave* waves, void* b_out,
                 int32_t on_device);

/* y = A x for the block matrix of `s` in `precision` (FE_PREC_FP64: complex128
 * vectors and matrix; FE_PREC_MIXED: complex64 vectors and the complex64
 * matrix copy; FE_PREC_DF: vectors of complex FP32 pairs, 16 bytes per entry
 * (re_hi, im_hi, re_lo, im_lo), and the FP32-pair matrix copy).  x, y:
 * DEVICE buffers [n_dof][nrhs], nrhs >= 1; no aliasing.
 * This is the sparse product at the heart of the Krylov loop (Section 3.1.5.1). */
fe_status fe_spmv(fe_ctx* ctx, const fe_system* s, int32_t precision, int32_t nrhs, const void* x, void* y);

/* Half (symmetric) storage, storage #1 of Section 4.2: the symmetrised
 * matrix kept by its lower part only.  fe_system_pack_half copies, per block
 * row, the blocks (I, J <= I) of the system's complex128 values (and of its
 * complex64 copy when it has one) into compacted planes, and indexes, for
 * every block (I, J > I), the kept block (J, I) whose transpose it is.  The
 * storage stays with the system (a new call replaces it), keeps a block's
 * nine entries together, and costs about 14/27 of the values plus 4 bytes
 * per block.  kept_blocks (optional) receives the number of kept blocks.  Errors: FE_ERR_INVALID_ARG (NULL,
 * variant L, which is not symmetric, or no rows), FE_ERR_OOM, FE_ERR_CUDA. */
fe_status fe_system_pack_half(fe_ctx* ctx, fe_system* s, int64_t* kept_blocks);

/* y = A x from the half storage (the product of Section 4.2.5.1 on storage
 * #1): an upper block is read as the transpose of the kept block of the
 * neighbour's row.  precision FE_PREC_FP64 (complex128 vectors) or
 * FE_PREC_MIXED (complex64 vectors; the system needs its complex64 copy).
 * x, y: DEVICE buffers [n_dof][nrhs], nrhs a power of two <= 32; no
 * aliasing.  Errors: FE_ERR_INVALID_ARG (NULL, nrhs, precision, no half
 * storage), FE_ERR_CUDA. */
fe_status fe_spmv_half(fe_ctx* ctx, const fe_system* s, int32_t precision, int32_t nrhs, const void* x, void* y);

/* ------------------------------------------------------------------------
 * Solve (Sections 3.1.5 and 4.2.5: conjugate gradients on the symmetric
 * system with diagonal preconditioning; here the complex-symmetric form,
 * COCG, with 3x3 block-Jacobi preconditioning).  FE_PREC_MIXED runs the
 * sparse products of the Krylov loop on the complex64 copy of the matrix
 * (FP32 arithmetic and accumulation) while the recurrences, inner products
 * and the preconditioner stay FP64; each time the recursive residual has
 * dropped by `reliable`, the FP64 true residual b - A x replaces it and the
 * directions restart (FP64 iterative refinement around complex64 Krylov
 * passes).  FE_PREC_DF runs the whole Krylov loop in FP32 pairs (about 48
 * significant bits on the FP32 pipes, which GB300 issues at 64 times the FP64
 * rate): products, vectors, inner products and the recurrence scalars; like
 * FE_PREC_FP64 it keeps the directions across true-residual refreshes.  The true residual decides convergence: ||b - A x|| / ||b|| <= tol
 * for every right-hand side.  Up to
 * rhs_tile right-hand sides are solved together in one persistent device
 * launch.  With rhs_tile = 0 and at least 8 right-hand sides, the first solve
 * of a system shape (unknowns, right-hand sides, precision, variant, device)
 * runs the autotuner: short trial launches (32 iterations of the first
 * columns) for every tile width in {8, 16, 32} up to the column count and
 * grids of all or three quarters of the SMs, timed with CUDA events; the
 * fastest per column and iteration is kept for that shape in a process-wide
 * cache and reported in fe_solve_stats.  Fewer right-hand sides use the
 * widest power of two up to their count.
 * ---------------------------------------------------------------------- */
/* The form of the COCG step length alpha = gamma / (p^T A p).  Every
 * iteration fuses its inner products into one grid reduction after the
 * product w = A u (u = M r); p^T A p then comes either from the
 * Chronopoulos-Gear recurrence e = delta - beta gamma / alpha_old (fastest
 * per iteration), or as u^T w + 2 beta u^T s + beta^2 p^T s with the
 * recursively updated s = A p (A is symmetric, so p^T A u = u^T s): u^T s and
 * p^T s are taken in the vector update and summed at the grid barrier that
 * ends it.  The recurrence subtracts nearly equal quantities on systems whose
 * residual plateaus for thousands of iterations, and there rounding errors
 * in the inner products (FP32 pairs in particular) lengthen the plateau: on
 * the 40^3 voxel aircraft the expanded form needs 12 339 FP32-pair iterations
 * against 19 385 (1.03 s against 1.49 s), and the 80^3 aircraft converges
 * only with it.  Solves with the
 * block incomplete Cholesky preconditioner use the recurrence. */
typedef enum fe_recurrence {
    FE_RECURRENCE_CG = 0,       /* Chronopoulos-Gear (default) */
    FE_RECURRENCE_EXPANDED = 1  /* p^T A p = u^T w + 2 beta u^T s + beta^2 p^T s */
} fe_recurrence;

typedef enum fe_preconditioner {
    FE_PRECOND_BLOCK_JACOBI = 0, /* inverse 3x3 node blocks (the diagonal preconditioning of Section
                                    3.1.5.1 on the node blocks); every precision */
    FE_PRECOND_BICP = 1          /* block incomplete Cholesky, one band per CTA (fe_system_factor_bicp
                                    first); FE_PREC_FP64 only, one system per launch */
} fe_preconditioner;

typedef struct fe_solve_opts {
    int32_t precision;   /* fe_precision; default FE_PREC_DF */
    double tol;          /* true FP64 relative residual target; default 1e-8 */
    double reliable;     /* mixed mode: each time the recursive residual has dropped by this factor since the
                            last FP64 pass, the FP64 true residual b - A x replaces it and the complex64
                            Krylov directions restart (iterative refinement); default 1e-4 */
    int32_t max_iter;    /* cap on Krylov iterations per right-hand side; default 100000 */
    int32_t max_outer;   /* cap on true-residual replacements per right-hand side; default 200 */
    int32_t rhs_tile;    /* right-hand sides per device pass, 0 = automatic */
    int32_t max_pass_iter; /* mixed mode: a complex64 pass that has not dropped by `reliable` after this
                              many iterations is replaced all the same (its recursion has stalled);
                              0 = no cap; default 2000 */
    int32_t wait_timeout_us; /* bound on every device-side wait of the solve (grid barriers, copy
                              completions); on expiry the solve ends with FE_ERR_TIMEOUT and the
                              context stays usable; 0 = default 4 000 000 (4 s) */
    int32_t preconditioner; /* fe_preconditioner; default FE_PRECOND_BLOCK_JACOBI */
    int32_t recurrence;     /* fe_recurrence; default FE_RECURRENCE_CG */
} fe_solve_opts;

void fe_solve_opts_default(fe_solve_opts* o);

typedef struct fe_solve_report {
    int32_t status;        /* fe_status of this right-hand side */
    int32_t iterations;    /* Krylov iterations (sum over refinement passes) */
    int32_t outer;         /* FP64 true-residual evaluations */
    int32_t reserved;
    double rel_residual;   /* final true FP64 ||b - A x|| / ||b|| */
} fe_solve_report;

/* Builds B from the plane waves (Eq. 4) and solves A X = B.
 * x_out: complex128 [n_dof][nrhs], host or device (x_on_device).  rep:
 * optional host array of nrhs reports.  Returns FE_OK when every column met
 * tol, else the first failing column's status (the reports and x are still
 * written).  Errors: FE_ERR_INVALID_ARG, FE_ERR_OOM, FE_ERR_CUDA,
 * FE_ERR_NOT_CONVERGED, FE_ERR_BREAKDOWN, FE_ERR_TIMEOUT. */
fe_status fe_solve_batch(fe_ctx* ctx, const fe_system* s, int32_t nrhs, const fe_planewave* waves,
                         const fe_solve_opts* o, void* x_out, int32_t x_on_device, fe_solve_report* rep);

/* As fe_solve_batch with a caller right-hand side b (complex128 [n_dof][nrhs],
 * host or device as b_on_device) and optional initial guess in x_out
 * (use_x0 = 1: x_out holds x0 on entry; this is how a solve is resumed). */
fe_status fe_solve_rhs(fe_ctx* ctx, const fe_system* s, int32_t nrhs, const void* b, int32_t b_on_device,
                       const fe_solve_opts* o, void* x_out, int32_t x_on_device, int32_t use_x0,
                       fe_solve_report* rep);

/* Solve without any allocation.  Some callers cannot let a library allocate
 * device memory while they run: an application that reserves all device
 * memory for itself up front (an allocation would fail, or evict its own
 * data), a host thread with a latency bound that must not wait on the
 * device allocator (cudaMalloc and cudaFree can synchronise the device), or
 * an embedding that accounts for every byte of device memory its process
 * uses.  The paper has no counterpart.
 *
 * Same method and options as fe_solve_rhs, for a caller right-hand side in
 * DEVICE memory: b_dev and x_dev are complex128 [n_dof][nrhs] buffers in the
 * device memory of ctx's device (anything else, a host pointer included, is
 * rejected with FE_ERR_INVALID_ARG before any GPU work); x_dev holds the
 * initial guess when use_x0 = 1; nrhs is one of 1, 2, 4, 8, 16, 32.  rep:
 * optional host array of nrhs reports.
 *
 * Scratch: the call keeps all of its workspace in one file-scope device array
 * of 32 MiB (every GPU that loads the library holds it until the process
 * exits); it calls no cudaMalloc / cudaFree and no allocating routine.  The
 * need is 80 bytes per unknown and right-hand side in the FP64 and FP32-pair
 * modes and 88 in the mixed mode, plus a few KiB, so n_dof * nrhs may reach
 * about 415 000 (FP64, FP32 pairs) or 380 000 (mixed); a larger problem is
 * rejected with FE_ERR_INVALID_ARG and a message naming the bytes it would
 * need.  The first call on a device looks the array's device address up
 * (once per device, with that device current), so make that first call
 * before any stream capture; if the device's context is destroyed later (a
 * device reset), the next call looks it up again.  The call synchronises the
 * context's stream to read the reports back, so it must not be made while
 * that stream (or any stream, in global capture mode) is being captured.
 * Every call uses the same array: two calls whose GPU work overlaps (two
 * contexts or streams at once) race on it and corrupt each other's results.
 * Errors: as fe_solve_rhs. */
fe_status fe_solve_rhs_noalloc(fe_ctx* ctx, const fe_system* s, int32_t nrhs, const void* b_dev, void* x_dev,
                               int32_t use_x0, const fe_solve_opts* o, fe_solve_report* rep);

/* ------------------------------------------------------------------------
 * Serving: a queue of independent scattering problems (each its own voxel
 * box, frequency and plane waves) solved with continuous batching.  The
 * server owns a worker thread and CUDA streams of its own on the device of
 * the context passed to fe_serve_create (whose options, variant, abc_sigma
 * and penalty_s, apply to every request; that context stays free for the
 * caller).  The worker admits queued requests in arrival order while the
 * sum of their estimated device memory stays within the budget, and builds
 * each admitted request's mesh, system (Eqs. 1-4) and right-hand sides.
 * Solves then run in segments of about 25 ms: each segment is one
 * persistent cooperative launch per right-hand-side tile width (1, 2, 4, 8,
 * 16 or 32 after padding with zero columns), the widths side by side on
 * their own streams; every request has its own range of CTAs, synchronises
 * only among them, and keeps its Krylov state on the device from segment to
 * segment.  Between segments finished requests are handed out and their
 * memory freed, and requests that arrived meanwhile are admitted and start
 * beside the ones in flight.  A request's CTA count depends on its own size
 * only (fe_serve_plan), so its result is bitwise the same whether it is
 * served alone or among others.
 * ---------------------------------------------------------------------- */
typedef struct fe_serve_opts {
    int32_t precision;     /* FE_PREC_DF (default), FE_PREC_FP64 or FE_PREC_MIXED, for every request */
    double tol;            /* true relative residual target; default 1e-8 */
    double reliable;       /* FE_PREC_MIXED refinement trigger; default 1e-4 */
    int32_t max_iter;      /* default 100000 */
    int32_t max_outer;     /* default 200 */
    int64_t hbm_budget;    /* device bytes for admitted requests; 0: 80 % of the free memory at creation */
    int32_t max_ctas;      /* CTAs of one launch, 1..one per SM; 0: one per SM */
    int32_t work_per_cta;  /* packing target, block rows x tile width per CTA; 0: 2048 */
    int32_t max_job_ctas;  /* CTAs one request may take (a cap leaves room for requests that arrive while a
                              large one runs); 0: three quarters of max_ctas; max_ctas: no cap */
    int32_t seg_iters;     /* Krylov iterations per segment; 0 (default): each request runs as many as fill
                              about 25 ms at its own measured time per iteration (64 in its first segment) */
    int32_t recurrence;    /* fe_recurrence of every request's solve; default FE_RECURRENCE_EXPANDED (a stream of
                              voxel cubes at 1-6 GHz, 8-50 nodes per side: 4.13 solves/s and all of the first 128
                              requests converged, against 2.24 and 127 with FE_RECURRENCE_CG) */
} fe_serve_opts;
void fe_serve_opts_default(fe_serve_opts* o);

typedef struct fe_request {
    fe_mesh_desc mesh;          /* host pointers only (material_on_device = 0); copied by fe_serve_submit */
    double freq_hz;             /* > 0 */
    int32_t nrhs;               /* 1..32 */
    const fe_planewave* waves;  /* host, nrhs entries; copied */
} fe_request;

typedef struct fe_result {
    int32_t status;             /* FE_OK, or why the request failed (FE_ERR_MESH, FE_ERR_OOM, FE_ERR_NOT_CONVERGED ...) */
    int32_t nrhs;
    int64_t n_dof;              /* 3 x active nodes (0 when the mesh failed) */
    const fe_complex* x;        /* [n_dof][nrhs] total H at the active nodes, ranked as everywhere else;
                                   NULL when no solve ran.  Owned by the server until fe_serve_release. */
    const int32_t* node_id;     /* [n_dof / 3] grid node id of every rank; owned like x */
    const fe_solve_report* reports; /* [nrhs] per right-hand side; owned like x (NULL when no solve ran) */
    double t_submit, t_admit, t_done; /* seconds since fe_serve_create */
    int32_t batch_jobs;         /* most requests (all widths) that ran in one segment with it */
    int32_t batch_ctas;         /* CTAs it had (the same in every segment) */
    const char* message;        /* "" or the error text; owned like x */
} fe_result;

typedef struct fe_serve_stats {
    int64_t submitted, completed, failed;
    int64_t launches;           /* persistent solve launches (one per tile width per segment) */
    int64_t jobs_launched;      /* requests summed over segments */
    int64_t budget_bytes;       /* admission budget */
    int64_t peak_admitted_bytes;/* largest sum of admitted estimates */
    double solve_device_s;      /* time the worker spent in segments (launch to completion) */
} fe_serve_stats;

/* Errors: FE_ERR_INVALID_ARG (NULL, options out of range), FE_ERR_OOM, FE_ERR_CUDA. */
fe_status fe_serve_create(fe_ctx* ctx, const fe_serve_opts* o, fe_server** out);
/* Non-blocking.  Validates and copies the request, returns its ticket (> 0).
 * Errors: FE_ERR_INVALID_ARG (NULL pointers, sizes, nrhs, a device material
 * pointer, a stopped server).  Mesh rules are checked later: such a request
 * finishes with status FE_ERR_MESH. */
fe_status fe_serve_submit(fe_server* srv, const fe_request* r, uint64_t* ticket);
/* FE_PENDING while the request is queued or running; FE_OK with *out filled
 * once it has finished, whether it succeeded or not (out->status says which);
 * FE_ERR_INVALID_ARG for an unknown or released ticket. */
fe_status fe_serve_poll(fe_server* srv, uint64_t ticket, fe_result* out);
/* As fe_serve_poll, but blocks until the request finishes or timeout_s
 * seconds pass (then FE_PENDING). */
fe_status fe_serve_wait(fe_server* srv, uint64_t ticket, double timeout_s, fe_result* out);
/* Frees a finished request's result; the pointers in its fe_result die.
 * Errors: FE_ERR_INVALID_ARG (unknown ticket), FE_PENDING (not finished). */
fe_status fe_serve_release(fe_server* srv, uint64_t ticket);
fe_status fe_serve_info(fe_server* srv, fe_serve_stats* out);
/* Stops the worker after its current segment, drops unfinished requests and
 * frees everything, including unreleased results. */
void fe_serve_destroy(fe_server* srv);
/* The server's scheduling rule for one segment, a host-only function (no
 * device work): given n active requests in arrival order with their block
 * rows and tile widths, fills n_cta[i] (0: not in this segment) and returns
 * how many requests run.  A request's CTA count is fixed by its own size,
 * ceil(rows x width / work_per_cta) clamped to 1..min(rows, max_job_ctas)
 * (values < 1 or > max_ctas mean max_ctas), never by the other requests, so
 * its solve is partitioned, reduced and rounded the same way alone or in any
 * mix.  Requests are taken in order while their count fits in what the
 * earlier ones left of max_ctas; a later, smaller request may run while an
 * earlier one waits (every segment is planned afresh, so the earlier one is
 * considered first again at the next segment). */
int32_t fe_serve_plan(int32_t n, const int64_t* rows, const int32_t* width, int32_t max_ctas, int32_t max_job_ctas,
                      int32_t work_per_cta, int32_t* n_cta);

/* Device-side statistics of the most recent fe_solve_batch / fe_solve_rhs
 * call on this context, measured with CUDA events on the context stream
 * around the persistent solve launches. */
typedef struct fe_solve_stats {
    double kernel_ms;        /* device time of the persistent solve launch(es), summed over tiles */
    int64_t launches;        /* persistent launches (one per right-hand-side tile) */
    int64_t inner_iters;     /* Krylov iterations, summed over right-hand sides */
    int64_t passes;          /* refinement passes (true-residual evaluations), summed over tiles */
    int64_t tile_width;      /* right-hand sides per launch */
    int64_t grid_ctas;       /* CTAs of the cooperative launch */
    int64_t tuned;           /* how tile_width and grid_ctas were chosen: 0 the fixed rule (or the caller's
                                rhs_tile), 1 timed by the autotuner in this call, 2 the autotuner's cached choice */
    double tune_ms;          /* device time of the autotuner's trial launches in this call */
} fe_solve_stats;
fe_status fe_last_solve_stats(const fe_ctx* ctx, fe_solve_stats* out);

/* Thread-local description of the last error of the calling thread. */
const char* fe_last_error(void);
/* Number of kernel launches the library has issued on any context so far. */
int64_t fe_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* FE_H */
