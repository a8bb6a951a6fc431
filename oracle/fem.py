"""FP64 CPU oracle for the nodal H-field finite-element scattering method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs import this package; the library
never does, and it shares no code with the CUDA path.

What it computes (Vollaire, Nicolas & Nicolas, "Parallel computing for the
finite element method", Section 2):

* the weak Galerkin H-field vector wave equation (Eq. 1) with the grad-div
  penalty (Eq. 2), tested with W = N_a e_alpha (trilinear hexahedral hat times
  a Cartesian unit vector) and integrated by parts, giving per element

      a_e(W, H) = int (1/eps_r)(curl W).(curl H) + s (div W)(div H)
                  - k0^2 mu_r W.H  dv;

* the second-order Engquist-Majda absorbing condition on the rectangular
  outer faces (Eq. 3), written in weak form with the transverse Laplacian
  integrated by parts (edge line integrals dropped):

      G(W, H) = j k0 int W_t.H_t ds
                + sigma (j / 2k0) int sum_g grad_t (W_t)_g . grad_t (H_t)_g ds;

* the penalty surface term of Eq. 4 on Sext + Spec,
      L(W, H) = - s int (W.n)(div H) ds;

* the total-field right-hand side of Eq. 4,
      b(W) = G(W, H_i) - int_Sext W.(n x curl H_i) ds,
  evaluated in the same integrated-by-parts form as the left-hand side;

* variants: 'S' = a + G (complex symmetric), 'L' = a + L + G (literal Eq. 4),
  'P' = (A_L + A_L^T)/2 (the symmetrisation by the transpose of Section 3.1.4).

Readings of the paper used here: mass term -k0^2 mu_r (Eq. 1; Eq. 4 prints
+, which turns the Helmholtz operator into a non-oscillatory one); sigma = +1,
Eq. 3 as printed (g = j k0 H_t - (j/2k0) lap_t H_t, whose weak form adds
+ (j/2k0) int grad_t W : grad_t H): the imaginary part of G is then positive
for every tangential mode, i.e. the boundary absorbs; the opposite sign
(sigma = -1, the sign a Taylor expansion of the normal wavenumber suggests)
makes k0 M - K/(2k0) negative for tangential wavenumbers above sqrt(2) k0,
an active boundary for most mesh modes; s = 1 (Eq. 4 shows no coefficient);
PEC elements are not meshed and PEC faces carry only L (Section 3.1.3: the H
formulation needs no conductor condition).

Element integrals use 2x2x2 Gauss-Legendre points (exact for products of
trilinear functions); face integrals 2x2 points.  Assembly is a plain
coordinate-list sum into a SciPy CSR matrix; solves are SuperLU (or dense
LAPACK for tiny systems).
"""
from __future__ import annotations

import functools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

C0 = 299_792_458.0
PEC = 255

# local node a = ix + 2*iy + 4*iz
LOCAL_NODES = np.array([(a & 1, (a >> 1) & 1, (a >> 2) & 1) for a in range(8)], dtype=np.int64)
UNIT = np.eye(3)


def wavenumber(freq_hz: float) -> float:
    """k0 = 2 pi f / c0 (free-space wavenumber of Eq. 1)."""
    return 2.0 * np.pi * freq_hz / C0


def gauss_legendre_01(n: int):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def _hat(t, side):
    return 1.0 - t if side == 0 else t


def _dhat(side):
    return -1.0 if side == 0 else 1.0


def shape_functions(xi, h):
    """Trilinear hats N[8] and their physical gradients grad[8, 3] at the
    reference point xi in [0, 1]^3 of a brick with edge lengths h."""
    N = np.empty(8)
    grad = np.empty((8, 3))
    for a, (ix, iy, iz) in enumerate(LOCAL_NODES):
        f = (_hat(xi[0], ix), _hat(xi[1], iy), _hat(xi[2], iz))
        d = (_dhat(ix) / h[0], _dhat(iy) / h[1], _dhat(iz) / h[2])
        N[a] = f[0] * f[1] * f[2]
        grad[a] = (d[0] * f[1] * f[2], f[0] * d[1] * f[2], f[0] * f[1] * d[2])
    return N, grad


def vector_basis(N, grad):
    """The 24 test/trial functions W = N_a e_alpha (index 3a + alpha): their
    values [24, 3], curls [24, 3] and divergences [24]."""
    val = np.zeros((24, 3))
    curl = np.zeros((24, 3))
    div = np.zeros(24)
    for a in range(8):
        for al in range(3):
            i = 3 * a + al
            val[i] = N[a] * UNIT[al]
            curl[i] = np.cross(grad[a], UNIT[al])  # curl(N e) = grad N x e
            div[i] = grad[a][al]
    return val, curl, div


@functools.lru_cache(maxsize=None)
def _element_parts(h):
    """Real 24x24 volume integrals of a brick: curl.curl, div.div, val.val."""
    xg, wg = gauss_legendre_01(2)
    vol = h[0] * h[1] * h[2]
    cc = np.zeros((24, 24))
    dd = np.zeros((24, 24))
    mm = np.zeros((24, 24))
    for qx in range(2):
        for qy in range(2):
            for qz in range(2):
                w = wg[qx] * wg[qy] * wg[qz] * vol
                N, grad = shape_functions((xg[qx], xg[qy], xg[qz]), h)
                val, curl, div = vector_basis(N, grad)
                cc += w * curl @ curl.T
                dd += w * np.outer(div, div)
                mm += w * val @ val.T
    return cc, dd, mm


def element_matrix(h, eps_r, mu_r, k0, s=1.0):
    """24x24 complex element matrix of Eq. 1 + Eq. 2 (volume parts):
    A[3a+alpha, 3b+beta] = a_e(N_a e_alpha, N_b e_beta)."""
    cc, dd, mm = _element_parts(tuple(float(v) for v in h))
    return (1.0 / eps_r) * cc + s * dd - (k0 * k0) * mu_r * mm


def _face_frame(face):
    axis = face // 2
    side = face % 2
    n = (2.0 * side - 1.0) * UNIT[axis]
    tang = [g for g in range(3) if g != axis]
    return axis, side, n, tang


def _face_points(h, face):
    """2x2 Gauss points on a face of the reference brick (reference coords)
    and their physical weights."""
    axis, side, _, tang = _face_frame(face)
    xg, wg = gauss_legendre_01(2)
    area = h[tang[0]] * h[tang[1]]
    pts = []
    for p in range(2):
        for q in range(2):
            xi = np.zeros(3)
            xi[axis] = side
            xi[tang[0]] = xg[p]
            xi[tang[1]] = xg[q]
            pts.append((xi, wg[p] * wg[q] * area))
    return pts


@functools.lru_cache(maxsize=None)
def _face_parts(h, face):
    """Real 24x24 face integrals: W_t.H_t, sum_g grad_t(W_t)_g.grad_t(H_t)_g
    and (W.n)(div H)."""
    _, _, n, _ = _face_frame(face)
    mt = np.zeros((24, 24))
    kt = np.zeros((24, 24))
    pn = np.zeros((24, 24))
    proj = np.eye(3) - np.outer(n, n)  # tangential projector
    for xi, w in _face_points(h, face):
        N, grad = shape_functions(xi, h)
        val, _, div = vector_basis(N, grad)
        val_t = val @ proj  # W_t for every basis function
        # (W_t)_g = N_a (e_alpha)_t[g]; grad_t of it = (e_alpha)_t[g] * grad_t N_a
        gt = grad @ proj  # [8, 3] tangential gradients of the hats
        tg = np.zeros((24, 3, 3))  # [basis, component g, direction]
        for a in range(8):
            for al in range(3):
                et = proj @ UNIT[al]
                tg[3 * a + al] = np.outer(et, gt[a])
        mt += w * val_t @ val_t.T
        kt += w * np.einsum("igd,jgd->ij", tg, tg)
        pn += w * np.outer(val @ n, div)
    return mt, kt, pn


def face_abc_matrix(h, face, k0, sigma=1.0):
    """24x24 (element-local) matrix of the weak Engquist-Majda form G (Eq. 3)."""
    mt, kt, _ = _face_parts(tuple(float(v) for v in h), face)
    return 1j * k0 * mt + sigma * (1j / (2.0 * k0)) * kt


def face_penalty_matrix(h, face, s=1.0):
    """24x24 matrix of the penalty surface term L = -s int (W.n)(div H) ds (Eq. 4)."""
    _, _, pn = _face_parts(tuple(float(v) for v in h), face)
    return -s * pn


def face_rhs(h, face, elem_corner, k0, k_hat, p_hat, amp, sigma=1.0):
    """Right-hand side of Eq. 4 on outer faces of one orientation, [F, 24, R]:
    b[f, 3a+alpha, r] = G(N_a e_alpha, H_i) - int N_a e_alpha . (n x curl H_i) ds
    for H_i = p_hat[r] amp[r] exp(-j k0 k_hat[r] . x); elem_corner[f] = world
    position of local node 0 of the element owning face f."""
    _, _, n, _ = _face_frame(face)
    proj = np.eye(3) - np.outer(n, n)
    corner = np.atleast_2d(np.asarray(elem_corner, dtype=float))  # [F, 3]
    k_hat = np.atleast_2d(np.asarray(k_hat, dtype=float))
    p_hat = np.atleast_2d(np.asarray(p_hat, dtype=float))
    amp = np.atleast_1d(np.asarray(amp, dtype=complex))
    kt = k_hat @ proj  # [R, 3] tangential part of k_hat
    out = np.zeros((corner.shape[0], 24, k_hat.shape[0]), dtype=complex)
    for xi, w in _face_points(h, face):
        N, grad = shape_functions(xi, h)
        val, _, _ = vector_basis(N, grad)
        val_t = val @ proj  # W_t of each basis function [24, 3]
        gt = grad @ proj  # tangential gradients of the hats [8, 3]
        tgw = np.zeros((24, 3, 3))  # grad_t of (W_t)_g: [basis, g, direction]
        for a in range(8):
            for al in range(3):
                tgw[3 * a + al] = np.outer(proj @ UNIT[al], gt[a])
        x = corner + xi * np.asarray(h)  # [F, 3] physical Gauss point
        phase = np.exp(-1j * k0 * (x @ k_hat.T)) * amp[None, :]  # [F, R]
        hi = phase[:, :, None] * p_hat[None, :, :]  # [F, R, 3]
        hi_t = hi @ proj
        # grad_t of each component g of H_i,t is -j k0 k_t (H_i,t)_g
        grad_hi_t = hi_t[:, :, :, None] * (-1j * k0 * kt)[None, :, None, :]  # [F, R, g, d]
        curl_hi = -1j * k0 * np.cross(k_hat[None, :, :], hi)  # [F, R, 3]
        n_curl = np.cross(n, curl_hi)  # [F, R, 3]
        out += w * (1j * k0 * np.einsum("ig,frg->fir", val_t, hi_t)
                    + sigma * (1j / (2.0 * k0)) * np.einsum("igd,frgd->fir", tgw, grad_hi_t)
                    - np.einsum("ig,frg->fir", val, n_curl))
    return out


# --------------------------------------------------------------------------
# Integer maps: active entities, lexicographic ranks, 3x3-block sparsity
# pattern, element-to-slot map and face lists (Section 3.1.2 storage by
# node rows; Section 4.2.1 matrix structure).
# --------------------------------------------------------------------------

class Maps:
    pass


def mesh_maps(problem) -> Maps:
    nx, ny, nz = problem.nx, problem.ny, problem.nz
    mat = np.asarray(problem.material, dtype=np.uint8).reshape(nz, ny, nx)
    act_el = mat != PEC
    node_act = np.zeros((nz + 1, ny + 1, nx + 1), dtype=bool)
    for dz in range(2):
        for dy in range(2):
            for dx in range(2):
                node_act[dz:dz + nz, dy:dy + ny, dx:dx + nx] |= act_el
    node_act = node_act.ravel()
    n_nodes_total = node_act.size
    node_rank = np.full(n_nodes_total, -1, dtype=np.int64)
    n_act = int(node_act.sum())
    node_rank[node_act] = np.arange(n_act)
    # element -> 8 node ids
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    conn = np.empty((i.size, 8), dtype=np.int64)
    for a, (ix, iy, iz) in enumerate(LOCAL_NODES):
        conn[:, a] = (i + ix) + (nx + 1) * ((j + iy) + (ny + 1) * (k + iz))
    act_ids = np.flatnonzero(act_el.ravel())
    ranks = node_rank[conn[act_ids]]  # [E_act, 8]
    ra = np.repeat(ranks, 8, axis=1)
    rb = np.tile(ranks, (1, 8))
    keys = np.unique(ra.ravel() * n_act + rb.ravel())
    rows = keys // n_act
    row_ptr = np.zeros(n_act + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    col_idx = keys % n_act
    elem_slot = np.full((i.size, 8, 8), -1, dtype=np.int64)
    slots = np.searchsorted(keys, ra * n_act + rb).reshape(-1, 8, 8)
    elem_slot[act_ids] = slots
    # faces: (element id, face id 0..5 = -x,+x,-y,+y,-z,+z) encoded 6*e + f
    ext = []
    pec = []
    dims = (nx, ny, nz)
    coords = (i, j, k)
    mflat = mat.ravel()
    bnd = boundary_kinds(problem)
    for f in range(6):
        axis, side = f // 2, f % 2
        c = coords[axis]
        on_box = (c == 0) if side == 0 else (c == dims[axis] - 1)
        ext_f = act_el.ravel() & on_box & (bnd[f] == 0)  # only absorbing faces are Sext
        ext.append(6 * np.flatnonzero(ext_f) + f)
        step = (1, nx, nx * ny)[axis] * (1 if side == 1 else -1)
        inside = act_el.ravel() & ~on_box
        e_in = np.flatnonzero(inside)
        nb = e_in + step
        pec.append(6 * e_in[mflat[nb] == PEC] + f)
    m = Maps()
    m.nx, m.ny, m.nz = nx, ny, nz
    m.node_active = node_act
    m.node_rank = node_rank
    m.n_act = n_act
    m.row_ptr = row_ptr
    m.col_idx = col_idx
    m.nnzb = int(keys.size)
    m.elem_slot = elem_slot
    m.conn = conn
    m.elem_active = act_el.ravel()
    m.faces_ext = np.sort(np.concatenate(ext))
    m.faces_pec = np.sort(np.concatenate(pec))
    m.n_dof = 3 * n_act
    m.fixed = fixed_dofs(problem, m)
    return m


def boundary_kinds(problem):
    """Kind of each box face (-x, +x, -y, +y, -z, +z): 0 absorbing (Eq. 3),
    1 symmetry plane (n . H = 0, Eq. 6a), 2 antisymmetry plane (n x H = 0,
    Eq. 6b)."""
    b = tuple(int(v) for v in getattr(problem, "boundary", (0,) * 6))
    if len(b) != 6 or any(v not in (0, 1, 2) for v in b):
        raise ValueError("boundary kinds are 0, 1 or 2 per face")
    return b


def fixed_dofs(problem, maps):
    """Unknowns held at zero by symmetry planes: on a symmetry plane the
    normal component of H (Eq. 6a), on an antisymmetry plane its two
    tangential components (Eq. 6b)."""
    bnd = boundary_kinds(problem)
    nx, ny, nz = problem.nx, problem.ny, problem.nz
    ids = np.flatnonzero(maps.node_active)
    ijk = (ids % (nx + 1), (ids // (nx + 1)) % (ny + 1), ids // ((nx + 1) * (ny + 1)))
    dims = (nx, ny, nz)
    fixed = np.zeros((ids.size, 3), dtype=bool)
    for f in range(6):
        if bnd[f] == 0:
            continue
        axis, side = f // 2, f % 2
        on = ijk[axis] == (dims[axis] if side else 0)
        for al in range(3):
            if (bnd[f] == 1) == (al == axis):  # 6a: the normal component; 6b: the tangential ones
                fixed[on, al] = True
    return fixed.reshape(-1)


def validate(problem):
    """Mesh rules: every outer-layer element is in vacuum (eps_r = mu_r = 1),
    so the absorbing condition of Eq. 3 applies in free space; material bytes
    index the table or are 255 (PEC)."""
    mat = np.asarray(problem.material).reshape(problem.nz, problem.ny, problem.nx)
    nm = len(problem.eps_r)
    bad = (mat != PEC) & (mat >= nm)
    if bad.any():
        raise ValueError("material byte outside the table")
    if np.all(mat == PEC):
        raise ValueError("no active element")
    bnd = boundary_kinds(problem)
    shell = np.zeros_like(mat, dtype=bool)  # elements on an absorbing face
    for f in range(6):
        if bnd[f] != 0:
            continue
        axis, side = f // 2, f % 2  # mat is indexed [k, j, i]
        idx = [slice(None)] * 3
        idx[2 - axis] = -1 if side else 0
        shell[tuple(idx)] = True
    sm = mat[shell]
    if np.any(sm == PEC):
        raise ValueError("PEC touches the outer box")
    for m in np.unique(sm):
        if problem.eps_r[m] != 1 or problem.mu_r[m] != 1:
            raise ValueError("outer faces must be in vacuum")


def _elem_dofs(maps, elems):
    ranks = maps.node_rank[maps.conn[elems]]  # [n, 8]
    return (3 * ranks[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 24)


def _coo_add(rows, cols, vals, dofs, mat_block):
    n = dofs.shape[0]
    if n == 0:
        return
    rows.append(np.repeat(dofs, 24, axis=1).ravel())
    cols.append(np.tile(dofs, (1, 24)).ravel())
    vals.append(np.broadcast_to(mat_block.ravel(), (n, 576)).ravel())


def pec_surface_dofs(problem, maps):
    """E formulation: unknowns held at zero on PEC surfaces (n x E = 0).  Around
    an active node, axis a is a surface normal when two elements of the box
    that differ only along a are one PEC and one active; every component but
    a is then tangential and held (at PEC edges and corners all three)."""
    nx, ny, nz = problem.nx, problem.ny, problem.nz
    mat = np.asarray(problem.material).reshape(nz, ny, nx)
    ids = np.flatnonzero(maps.node_active)
    i = ids % (nx + 1)
    j = (ids // (nx + 1)) % (ny + 1)
    k = ids // ((nx + 1) * (ny + 1))
    pec = np.zeros((ids.size, 8), dtype=bool)
    act = np.zeros((ids.size, 8), dtype=bool)
    for b in range(8):
        ex, ey, ez = b & 1, (b >> 1) & 1, (b >> 2) & 1
        a, bb, c = i - 1 + ex, j - 1 + ey, k - 1 + ez
        inside = (a >= 0) & (a < nx) & (bb >= 0) & (bb < ny) & (c >= 0) & (c < nz)
        m = np.full(ids.size, 0, dtype=np.int64)
        m[inside] = mat[c[inside], bb[inside], a[inside]]
        pec[:, b] = inside & (m == PEC)
        act[:, b] = inside & (m != PEC)
    held = np.zeros((ids.size, 3), dtype=bool)
    for axis in range(3):
        bit = 1 << axis
        normal = np.zeros(ids.size, dtype=bool)
        for b in range(8):
            if b & bit:
                continue
            normal |= (pec[:, b] & act[:, b | bit]) | (act[:, b] & pec[:, b | bit])
        for al in range(3):
            if al != axis:
                held[normal, al] = True
    return held.reshape(-1)


def held_dofs(problem, maps, formulation="H"):
    """All unknowns held at zero: symmetry planes, and PEC surfaces in the E
    formulation."""
    if formulation not in ("H", "E"):
        raise ValueError(formulation)
    return maps.fixed | pec_surface_dofs(problem, maps) if formulation == "E" else maps.fixed


def assemble(problem, variant="S", sigma=1.0, s=1.0, maps=None, chunk=20000, formulation="H"):
    """Global n_dof x n_dof complex128 CSR matrix of Eq. 4's left-hand side.

    Element matrices are summed into the global matrix entry by entry
    (coordinate list, duplicates summed); variant 'P' then forms
    (A_L + A_L^T)/2 (Section 3.1.4).  formulation 'E' solves for the total
    E field with the same steps (Section 2): 1/mu_r in the curl-curl term,
    eps_r in the mass term, and n x E = 0 held on PEC surfaces."""
    if variant not in ("S", "L", "P"):
        raise ValueError(variant)
    validate(problem)
    maps = maps if maps is not None else mesh_maps(problem)
    k0 = wavenumber(problem.freq_hz)
    h = tuple(float(v) for v in problem.h)
    n = maps.n_dof
    mflat = np.asarray(problem.material).ravel()
    total = sp.csr_matrix((n, n), dtype=complex)

    def flush(rows, cols, vals):
        nonlocal total
        if rows:
            r = np.concatenate(rows)
            c = np.concatenate(cols)
            v = np.concatenate(vals)
            total = total + sp.csr_matrix((v, (r, c)), shape=(n, n))
            rows.clear(), cols.clear(), vals.clear()

    rows, cols, vals = [], [], []
    act = np.flatnonzero(maps.elem_active)
    for m in np.unique(mflat[act]):
        if formulation == "E":
            ae = element_matrix(h, problem.mu_r[m], problem.eps_r[m], k0, s)
        else:
            ae = element_matrix(h, problem.eps_r[m], problem.mu_r[m], k0, s)
        el = act[mflat[act] == m]
        for c0 in range(0, el.size, chunk):
            _coo_add(rows, cols, vals, _elem_dofs(maps, el[c0:c0 + chunk]), ae)
            flush(rows, cols, vals)
    use_l = variant in ("L", "P")
    for f in range(6):
        ext_e = maps.faces_ext[maps.faces_ext % 6 == f] // 6
        t = face_abc_matrix(h, f, k0, sigma)
        if use_l:
            t = t + face_penalty_matrix(h, f, s)
        _coo_add(rows, cols, vals, _elem_dofs(maps, ext_e), t)
        if use_l:
            pec_e = maps.faces_pec[maps.faces_pec % 6 == f] // 6
            _coo_add(rows, cols, vals, _elem_dofs(maps, pec_e), face_penalty_matrix(h, f, s))
        flush(rows, cols, vals)
    total.sum_duplicates()
    if variant == "P":
        total = (0.5 * (total + total.T)).tocsr()
        total.sum_duplicates()
    held = held_dofs(problem, maps, formulation)
    if held.any():
        # unknowns held at zero (symmetry planes, PEC surfaces for E): identity rows and columns
        keep = sp.diags((~held).astype(float))
        total = (keep @ total @ keep + sp.diags(held.astype(float))).tocsr()
        total.sum_duplicates()
    return total


def element_corner(problem, e):
    """World position of local node 0 of element(s) e."""
    e = np.asarray(e)
    nx, ny = problem.nx, problem.ny
    i = e % nx
    j = (e // nx) % ny
    k = e // (nx * ny)
    o = np.asarray(problem.origin, dtype=float)
    h = np.asarray(problem.h, dtype=float)
    return o + np.stack([i, j, k], axis=-1).astype(float) * h


def rhs(problem, waves, sigma=1.0, maps=None, formulation="H"):
    """B[n_dof, R]: right-hand side of Eq. 4 for each plane wave, summed over
    the outer (Sext) faces (the waves' p_hat polarises the formulation's
    field, H or E)."""
    maps = maps if maps is not None else mesh_maps(problem)
    k0 = wavenumber(problem.freq_hz)
    h = tuple(float(v) for v in problem.h)
    B = np.zeros((maps.n_dof, waves.count), dtype=complex)
    for f in range(6):
        elems = maps.faces_ext[maps.faces_ext % 6 == f] // 6
        if elems.size == 0:
            continue
        dofs = _elem_dofs(maps, elems)  # [F, 24]
        corners = element_corner(problem, elems)
        contrib = face_rhs(h, f, corners, k0, waves.k_hat, waves.p_hat, waves.amplitude, sigma)
        np.add.at(B, dofs.ravel(), contrib.reshape(-1, waves.count))
    B[held_dofs(problem, maps, formulation)] = 0.0
    return B


def solve_direct(A, B):
    """x = A^{-1} B: dense LAPACK below 3000 unknowns, SuperLU above."""
    B2 = B.reshape(B.shape[0], -1)
    if A.shape[0] <= 3000:
        X = np.linalg.solve(A.toarray(), B2)
    else:
        # the block pattern is structurally symmetric: order on A^T + A
        lu = spla.splu(A.tocsc(), permc_spec="MMD_AT_PLUS_A", options=dict(SymmetricMode=True))
        X = lu.solve(B2)
    return X.reshape(B.shape)


def true_relative_residual(A, X, B):
    """Per-column ||b - A x||_2 / ||b||_2 in FP64."""
    X2 = X.reshape(X.shape[0], -1)
    B2 = B.reshape(B.shape[0], -1)
    R = B2 - A @ X2
    return np.linalg.norm(R, axis=0) / np.linalg.norm(B2, axis=0)


def to_bsr_values(A, maps):
    """Values of the 3x3 blocks of A on the block pattern (row_ptr, col_idx):
    out[slot, alpha, beta] = A[3*row + alpha, 3*col + beta]."""
    rows = np.repeat(np.arange(maps.n_act), np.diff(maps.row_ptr))
    cols = maps.col_idx
    Ac = A.tocsr()
    out = np.empty((maps.nnzb, 3, 3), dtype=complex)
    for al in range(3):
        for be in range(3):
            out[:, al, be] = np.asarray(Ac[3 * rows + al, 3 * cols + be]).ravel()
    return out


def node_positions(problem, maps):
    """World coordinates [n_act, 3] of the active nodes in rank order."""
    nx, ny = problem.nx, problem.ny
    ids = np.flatnonzero(maps.node_active)
    i = ids % (nx + 1)
    j = (ids // (nx + 1)) % (ny + 1)
    k = ids // ((nx + 1) * (ny + 1))
    o = np.asarray(problem.origin, dtype=float)
    h = np.asarray(problem.h, dtype=float)
    return o + np.stack([i, j, k], axis=1) * h


def plane_wave_at_nodes(problem, maps, waves):
    """H_i sampled at the active nodes, laid out [n_dof, R]."""
    pos = node_positions(problem, maps)
    k0 = wavenumber(problem.freq_hz)
    R = waves.count
    out = np.empty((maps.n_dof, R), dtype=complex)
    for r in range(R):
        ph = np.exp(-1j * k0 * pos @ waves.k_hat[r]) * waves.amplitude[r]
        out[:, r] = (ph[:, None] * waves.p_hat[r][None, :]).ravel()
    return out
