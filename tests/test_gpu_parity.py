"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Integer maps bit-exact; complex128 block values within 1e-12 of the oracle
(relative to the block row's largest entry: the two sides sum the same
element contributions in different orders and derive them differently, Gauss
quadrature vs closed-form Kronecker products); the complex64 copy within one
ulp of the oracle value rounded to complex64; right-hand sides within 1e-11
(relative to the largest entry); products within the FP32/FP64 dot-product
error bound; solves with FP64 true residual <= 1e-8 (recomputed on the CPU
with the oracle matrix) and relative field error <= 1e-6 against the oracle's
direct solve."""
import numpy as np
import pytest

from oracle import fem, krylov
from paper_0704_2344_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SMALL = {
    "box2": lambda: W.empty_box(2),
    "config1": lambda: W.config1()[0],
    "rand1": lambda: W.random_small_grid(1, n_max=6),
    "rand2": lambda: W.random_small_grid(2, n_max=7, n_pec_boxes=3),
    "rand3": lambda: W.random_small_grid(3, n_max=5),
    "slab": lambda: W.empty_box((3, 5, 17)),
}


def _torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def config2():
    prob, waves = W.config2()
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps)
    return prob, waves, maps, A


def _row_scale(ref, maps):
    """Largest |entry| of each block row, broadcast to the row's blocks."""
    blk = np.abs(ref).reshape(ref.shape[0], -1).max(axis=1)
    rows = np.repeat(np.arange(maps.n_act), np.diff(maps.row_ptr))
    rmax = np.zeros(maps.n_act)
    np.maximum.at(rmax, rows, blk)
    return rmax[rows][:, None, None]


def _check_maps(fe, ctx, prob):
    m = fe.fe_mesh_create_from(ctx, prob)
    try:
        g = fe.fe_mesh_export_maps(ctx, m)
        info = fe.fe_mesh_info(m)
    finally:
        fe.fe_mesh_destroy(m)
    o = fem.mesh_maps(prob)
    assert np.array_equal(g["node_rank"], o.node_rank)
    assert np.array_equal(g["row_ptr"], o.row_ptr)
    assert np.array_equal(g["col_idx"], o.col_idx)
    assert np.array_equal(g["elem_slot"], o.elem_slot)
    assert np.array_equal(g["faces_ext"], o.faces_ext)
    assert np.array_equal(g["faces_pec"], o.faces_pec)
    assert info["n_active_elements"] == int(o.elem_active.sum())
    assert info["n_dof"] == o.n_dof and info["nnzb"] == o.nnzb


@pytest.mark.parametrize("name", list(SMALL))
def test_maps_bit_exact_small(fe, ctx, name):
    _check_maps(fe, ctx, SMALL[name]())


@pytest.mark.parametrize("seed", range(10, 20))
def test_maps_bit_exact_random(fe, ctx, seed):
    _check_maps(fe, ctx, W.random_small_grid(seed, n_max=9, n_pec_boxes=3))


def test_maps_bit_exact_config2(fe, ctx):
    _check_maps(fe, ctx, W.config2()[0])


def test_maps_bit_exact_aircraft(fe, ctx):
    _check_maps(fe, ctx, W.aircraft_mesh(40, 4))


def _check_values(fe, ctx, prob, variant="S", A=None, maps=None):
    maps = maps or fem.mesh_maps(prob)
    A = A if A is not None else fem.assemble(prob, variant=variant, maps=maps)
    m = fe.fe_mesh_create_from(ctx, prob)
    try:
        s = fe.fe_assemble(ctx, m, prob.freq_hz, fe.FE_PREC_MIXED)
        try:
            g = fe.fe_system_export(ctx, s, m, c128=True, c64=True, dinv=True)
        finally:
            fe.fe_system_destroy(s)
    finally:
        fe.fe_mesh_destroy(m)
    ref = fem.to_bsr_values(A, maps)
    scale = _row_scale(ref, maps)
    err = np.abs(g["c128"] - ref) / scale
    assert err.max() <= 1e-12, err.max()
    # the complex64 copy is exactly the round-to-nearest of the complex128 values
    assert np.array_equal(g["c64"], g["c128"].astype(np.complex64))
    # and within one ulp of the oracle value rounded to complex64, wherever the
    # value is not rounding noise of a cancelling sum (|ref| > 1e-12 row scale)
    r32 = ref.astype(np.complex64)
    for part in (np.real, np.imag):
        d = np.abs(part(g["c64"]).astype(np.float64) - part(r32).astype(np.float64))
        ulp = np.spacing(np.abs(part(r32))).astype(np.float64)
        significant = np.abs(part(ref)) > 1e-12 * scale
        assert np.all(d[significant] <= ulp[significant]), d[significant].max()
        assert np.all(np.abs(part(g["c64"]))[~significant] <= 2e-12 * np.broadcast_to(scale, d.shape)[~significant])
    dref = krylov.block_jacobi_inverse(A)
    derr = np.abs(g["dinv"] - dref).reshape(len(dref), -1).max(axis=1) / np.abs(dref).reshape(len(dref), -1).max(axis=1)
    assert derr.max() <= 1e-10, derr.max()


def _df_split(v):
    """Exact FP32-pair split of float64 values: hi = RN32(v), lo = RN32(v - hi)."""
    hi = v.astype(np.float32)
    return hi, (v - hi.astype(np.float64)).astype(np.float32)


@pytest.mark.parametrize("name", ["rand1", "config1"])
def test_assembly_df_pairs(fe, ctx, name):
    """The FP32-pair copy (FE_PREC_DF) is exactly the split of the complex128
    values, and hi + lo recovers them to about 2^-48 relative."""
    prob = SMALL[name]()
    m = fe.fe_mesh_create_from(ctx, prob)
    try:
        s = fe.fe_assemble(ctx, m, prob.freq_hz, fe.FE_PREC_DF)
        try:
            g = fe.fe_system_export(ctx, s, m, c128=True)["c128"]
            df = fe.fe_system_export_df(ctx, s, m)
        finally:
            fe.fe_system_destroy(s)
    finally:
        fe.fe_mesh_destroy(m)
    rh, rl = _df_split(g.real)
    ih, il = _df_split(g.imag)
    for k, ref in enumerate((rh, ih, rl, il)):
        assert np.array_equal(df[..., k], ref), k
    back = (df[..., 0].astype(np.float64) + df[..., 2]) + 1j * (df[..., 1].astype(np.float64) + df[..., 3])
    assert np.abs(back - g).max() <= 2.0 ** -47 * np.abs(g).max()


@pytest.mark.parametrize("name", list(SMALL))
def test_assembly_values_small(fe, ctx, name):
    _check_values(fe, ctx, SMALL[name]())


@pytest.mark.parametrize("variant,code", [("L", 1), ("P", 2)])
def test_assembly_variants(fe, variant, code):
    torch = _torch()
    c = fe.fe_ctx_create(0, variant=code)
    try:
        for seed in (1, 2):
            _check_values(fe, c, W.random_small_grid(seed, n_max=6), variant=variant)
    finally:
        fe.fe_ctx_synchronize(c)
        fe.fe_ctx_destroy(c)
    torch.cuda.synchronize()


def test_assembly_values_config2(fe, ctx, config2):
    prob, _, maps, A = config2
    _check_values(fe, ctx, prob, A=A, maps=maps)


def test_rhs_matches_oracle(fe, ctx):
    for prob, waves in [(W.config1()[0], W.sphere_waves(4, 7)), (W.random_small_grid(4, n_max=6), W.random_waves(5, np.random.default_rng(3)))]:
        maps = fem.mesh_maps(prob)
        ref = fem.rhs(prob, waves, maps=maps)
        m = fe.fe_mesh_create_from(ctx, prob)
        s = fe.fe_assemble(ctx, m, prob.freq_hz, fe.FE_PREC_FP64)
        try:
            g = fe.fe_rhs(ctx, s, waves, maps.n_dof)
        finally:
            fe.fe_system_destroy(s)
            fe.fe_mesh_destroy(m)
        assert np.abs(g - ref).max() <= 1e-11 * np.abs(ref).max()


def _spmv_check(fe, ctx, prob, nrhs, seed=0):
    torch = _torch()
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((maps.n_dof, nrhs)) + 1j * rng.standard_normal((maps.n_dof, nrhs))
    m = fe.fe_mesh_create_from(ctx, prob)
    s = fe.fe_assemble(ctx, m, prob.freq_hz, fe.FE_PREC_MIXED)
    try:
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        x32 = xd.to(torch.complex64)
        y32 = torch.empty_like(x32)
        torch.cuda.synchronize()
        fe.fe_spmv(ctx, s, fe.FE_PREC_FP64, nrhs, xd, yd)
        fe.fe_spmv(ctx, s, fe.FE_PREC_MIXED, nrhs, x32, y32)
        fe.fe_ctx_synchronize(ctx)
        y64 = yd.cpu().numpy()
        y32h = y32.cpu().numpy().astype(np.complex128)
    finally:
        fe.fe_system_destroy(s)
        fe.fe_mesh_destroy(m)
    ref = A @ x
    bound = abs(A) @ np.abs(x)
    assert np.all(np.abs(y64 - ref) <= 1e-13 * bound + 1e-300)
    # complex64 matrix and vector: rounding of the inputs plus FP32 accumulation
    A32 = fem.to_bsr_values(A, maps)
    assert np.all(np.abs(y32h - ref) <= 4e-6 * bound)


@pytest.mark.parametrize("nrhs", [1, 3, 8, 16, 32])
def test_spmv_small(fe, ctx, nrhs):
    _spmv_check(fe, ctx, W.random_small_grid(5, n_max=8, n_pec_boxes=2), nrhs)


@pytest.mark.parametrize("nrhs", [1, 16])
def test_spmv_config2(fe, ctx, nrhs):
    """Full size: 29 666 block rows, so the products' row groups run over many
    tiles and end in a ragged one."""
    _spmv_check(fe, ctx, W.config2()[0], nrhs, seed=3)


@pytest.mark.parametrize("nrhs", [1, 3, 8, 16])
def test_spmv_fp32_pairs(fe, ctx, nrhs):
    """FE_PREC_DF product: FP32-pair matrix and vector, error-free product
    and sum steps.  Its error is a few 2^-48 of sum |a_ij x_j| per entry; the
    bound 1e-12 is far below what complex64 arithmetic reaches (4e-6)."""
    torch = _torch()
    prob = W.random_small_grid(5, n_max=8, n_pec_boxes=2)
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps)
    rng = np.random.default_rng(7)
    x = rng.standard_normal((maps.n_dof, nrhs)) + 1j * rng.standard_normal((maps.n_dof, nrhs))
    rh, rl = _df_split(x.real)
    ih, il = _df_split(x.imag)
    xp = np.ascontiguousarray(np.stack([rh, ih, rl, il], axis=-1))
    m = fe.fe_mesh_create_from(ctx, prob)
    s = fe.fe_assemble(ctx, m, prob.freq_hz, fe.FE_PREC_DF)
    try:
        xd = torch.from_numpy(xp).cuda()
        yd = torch.empty_like(xd)
        torch.cuda.synchronize()
        fe.fe_spmv(ctx, s, fe.FE_PREC_DF, nrhs, xd, yd)
        fe.fe_ctx_synchronize(ctx)
        y = yd.cpu().numpy().astype(np.float64)
    finally:
        fe.fe_system_destroy(s)
        fe.fe_mesh_destroy(m)
    ydf = (y[..., 0] + y[..., 2]) + 1j * (y[..., 1] + y[..., 3])
    ref = A @ x
    bound = abs(A) @ np.abs(x)
    assert np.all(np.abs(ydf - ref) <= 1e-12 * bound)


def _solve(fe, ctx, prob, waves, precision, **kw):
    m = fe.fe_mesh_create_from(ctx, prob)
    s = fe.fe_assemble(ctx, m, prob.freq_hz, precision)
    try:
        n_dof = fe.fe_mesh_info(m)["n_dof"]
        st, x, rep = fe.fe_solve_batch(ctx, s, waves, n_dof, fe.solve_opts(precision=precision, **kw))
    finally:
        fe.fe_system_destroy(s)
        fe.fe_mesh_destroy(m)
    return x, rep


@pytest.mark.parametrize("precision", ["FP64", "MIXED", "DF"])
@pytest.mark.parametrize("name", ["box2", "config1", "rand1", "rand2"])
def test_solve_matches_direct(fe, ctx, name, precision):
    prob = SMALL[name]()
    waves = W.normal_incidence() if name != "rand2" else W.oblique_wave(0.6, 1.1)
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps)
    B = fem.rhs(prob, waves, maps=maps)
    xref = fem.solve_direct(A, B)
    x, rep = _solve(fe, ctx, prob, waves, getattr(fe, f"FE_PREC_{precision}"))
    res = fem.true_relative_residual(A, x, B)
    assert rep[0]["status"] == 0
    assert res.max() <= 1e-8, (res, rep)
    assert abs(rep[0]["rel_residual"] - res[0]) <= 1e-9
    err = np.linalg.norm(x - xref) / np.linalg.norm(xref)
    assert err <= 1e-6, err


def test_batched_columns_match_single_solves(fe, ctx):
    prob = W.random_small_grid(6, n_max=7, n_pec_boxes=1)
    waves = W.random_waves(8, np.random.default_rng(1))
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps)
    B = fem.rhs(prob, waves, maps=maps)
    xref = fem.solve_direct(A, B)
    xb, repb = _solve(fe, ctx, prob, waves, fe.FE_PREC_MIXED)
    assert all(r["status"] == 0 for r in repb)
    res = fem.true_relative_residual(A, xb, B)
    assert res.max() <= 1e-8
    for j in (0, 3, 7):
        xs, reps = _solve(fe, ctx, prob, waves.column(j), fe.FE_PREC_MIXED)
        assert np.linalg.norm(xs[:, 0] - xb[:, j]) <= 1e-6 * np.linalg.norm(xref[:, j])
        assert np.linalg.norm(xb[:, j] - xref[:, j]) <= 1e-6 * np.linalg.norm(xref[:, j])


def test_batched_columns_match_single_solves_fp32_pairs(fe, ctx):
    """Eight columns in one FE_PREC_DF launch keep their Krylov vectors as FP32
    pairs; each column still meets the single-column FP64-recurrence solve
    and the oracle's direct solution."""
    prob = W.random_small_grid(6, n_max=7, n_pec_boxes=1)
    waves = W.random_waves(8, np.random.default_rng(1))
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps)
    B = fem.rhs(prob, waves, maps=maps)
    xref = fem.solve_direct(A, B)
    xb, repb = _solve(fe, ctx, prob, waves, fe.FE_PREC_DF)
    assert all(r["status"] == 0 for r in repb)
    assert fem.true_relative_residual(A, xb, B).max() <= 1e-8
    for j in (0, 5):
        xs, _ = _solve(fe, ctx, prob, waves.column(j), fe.FE_PREC_DF)
        assert np.linalg.norm(xs[:, 0] - xb[:, j]) <= 1e-6 * np.linalg.norm(xref[:, j])
    for j in range(8):
        assert np.linalg.norm(xb[:, j] - xref[:, j]) <= 1e-6 * np.linalg.norm(xref[:, j])


def test_solve_config2_32_waves_one_launch(fe, ctx, config2):
    """The 3-wavelength cube at full size with 32 plane waves (the first 32 of
    the 64-wave workload) in one 32-column FP32-pair launch: every column's
    FP64 true residual, recomputed on the CPU with the oracle's matrix, is at
    most 1e-8."""
    prob, _, maps, A = config2
    w64 = W.config3()[1]
    waves = w64.__class__(w64.k_hat[:32], w64.p_hat[:32], w64.amplitude[:32])
    x, rep = _solve(fe, ctx, prob, waves, fe.FE_PREC_DF)
    stats = fe.fe_last_solve_stats(ctx)
    assert stats["launches"] == 1 and stats["tile_width"] == 32
    assert all(r["status"] == 0 for r in rep), rep
    B = fem.rhs(prob, waves, maps=maps)
    res = fem.true_relative_residual(A, x, B)
    assert res.max() <= 1e-8, res.max()
    assert np.allclose([r["rel_residual"] for r in rep], res, rtol=0, atol=1e-9)


def test_mesh_errors(fe, ctx):
    p = W.empty_box(4)
    p.material[0, 1, 1] = 255
    with pytest.raises(fe.FeError) as e:
        fe.fe_mesh_create_from(ctx, p)
    assert e.value.status == fe.FE_ERR_MESH
    p = W.empty_box(4)
    p.material[2, 2, 2] = 7  # outside a one-entry table
    with pytest.raises(fe.FeError) as e:
        fe.fe_mesh_create_from(ctx, p)
    assert e.value.status == fe.FE_ERR_INVALID_ARG
    p = W.empty_box(4)
    p.eps_r = np.array([1.0 + 0j, 2.0 + 0j])
    p.mu_r = np.array([1.0 + 0j, 1.0 + 0j])
    p.material[0, 0, 0] = 1
    with pytest.raises(fe.FeError) as e:
        fe.fe_mesh_create_from(ctx, p)
    assert e.value.status == fe.FE_ERR_MESH


@pytest.mark.parametrize("precision", ["FP64", "MIXED", "DF"])
@pytest.mark.parametrize("name", ["box2", "rand1", "rand2"])
def test_expanded_recurrence_matches_direct(fe, ctx, name, precision):
    """FE_RECURRENCE_EXPANDED (p^T A p from its three inner products with the
    recursive s) solves to the same bar as the default recurrence."""
    prob = SMALL[name]()
    waves = W.normal_incidence() if name != "rand2" else W.oblique_wave(0.6, 1.1)
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps)
    B = fem.rhs(prob, waves, maps=maps)
    xref = fem.solve_direct(A, B)
    x, rep = _solve(fe, ctx, prob, waves, getattr(fe, f"FE_PREC_{precision}"), recurrence=fe.FE_RECURRENCE_EXPANDED)
    res = fem.true_relative_residual(A, x, B)
    assert rep[0]["status"] == 0
    assert res.max() <= 1e-8, (res, rep)
    assert np.linalg.norm(x - xref) <= 1e-6 * np.linalg.norm(xref)


def test_unknown_recurrence_is_rejected(fe, ctx):
    prob = SMALL["box2"]()
    with pytest.raises(fe.FeError):
        _solve(fe, ctx, prob, W.normal_incidence(), fe.FE_PREC_DF, recurrence=7)


@pytest.mark.parametrize("recurrence", ["CG", "EXPANDED"])
@pytest.mark.parametrize("precision", ["FP64", "MIXED", "DF"])
def test_solve_config2_full_size(fe, ctx, config2, precision, recurrence):
    """The 3-wavelength cube at full size (88 998 unknowns) in the launch
    configuration the benchmark times: FP64 true residual <= 1e-8 with the
    oracle's matrix, and relative field error <= 1e-6 against the oracle's
    direct (SuperLU) solution stored by tests/golden/make_reference.py."""
    from pathlib import Path
    prob, waves, maps, A = config2
    ref = np.load(Path(__file__).with_name("golden") / "config2_x.npz")
    xref = ref["x"].astype(np.complex128)
    B = fem.rhs(prob, waves, maps=maps)
    x, rep = _solve(fe, ctx, prob, waves, getattr(fe, f"FE_PREC_{precision}"),
                    recurrence=getattr(fe, f"FE_RECURRENCE_{recurrence}"))
    res = fem.true_relative_residual(A, x, B)
    assert rep[0]["status"] == 0, rep
    assert res.max() <= 1e-8, (res, rep)
    err = np.linalg.norm(x - xref) / np.linalg.norm(xref)
    assert err <= 1e-6, err


@pytest.mark.parametrize("precision", ["df", "mixed"])
@pytest.mark.parametrize("name", ["config1", "rand2", "config2"])
def test_block_dictionary_counts_the_distinct_blocks(fe, ctx, name, precision):
    """The block dictionary lists each distinct block once: its size equals a
    bitwise count of the distinct blocks in the exported complex128 values
    (the dictionary's values are the exported ones, rounded to the inner
    precision, so equal complex128 blocks are equal there too)."""
    prob = W.config2()[0] if name == "config2" else SMALL[name]()
    prec = {"df": fe.FE_PREC_DF, "mixed": fe.FE_PREC_MIXED}[precision]
    m = fe.fe_mesh_create_from(ctx, prob)
    try:
        s = fe.fe_assemble(ctx, m, prob.freq_hz, prec)
        try:
            info = fe.fe_system_info(s)
            g = fe.fe_system_export(ctx, s, m, c128=True)["c128"]
        finally:
            fe.fe_system_destroy(s)
    finally:
        fe.fe_mesh_destroy(m)
    flat = np.ascontiguousarray(g.reshape(len(g), -1)).view(np.uint64)
    distinct = np.unique(flat, axis=0).shape[0]
    assert info["dict_blocks"] == (distinct if distinct <= 4096 else 0)
    if name == "config2":
        assert 0 < info["dict_blocks"] <= 4096
