"""GPU parity of the half (symmetric) storage, storage #1 of Section 4.2, and
its product (Section 4.2.5.1) through the C ABI: y = A x from the kept lower
blocks against the oracle's matrix (complex128 within 1e-13 |A||x|,
complex64 within 4e-6 |A||x|, the bounds of the full-storage product), for
several column counts, on random grids with PEC boxes, the symmetrised
variant P and the full-size 3-wavelength cube; the number of kept blocks
against the lower block pattern; and the argument errors."""
import numpy as np
import pytest

from oracle import fem
from paper_0704_2344_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _half_check(fe, ctx, prob, nrhs, seed=0, variant="S"):
    import torch
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, variant=variant, maps=maps)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((maps.n_dof, nrhs)) + 1j * rng.standard_normal((maps.n_dof, nrhs))
    m = fe.fe_mesh_create_from(ctx, prob)
    s = fe.fe_assemble(ctx, m, prob.freq_hz, fe.FE_PREC_MIXED)
    try:
        kept = fe.fe_system_pack_half(ctx, s)
        rows = np.repeat(np.arange(maps.n_act), np.diff(maps.row_ptr))
        assert kept == int(np.count_nonzero(np.asarray(maps.col_idx) <= rows))
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        x32 = xd.to(torch.complex64)
        y32 = torch.empty_like(x32)
        torch.cuda.synchronize()
        fe.fe_spmv_half(ctx, s, fe.FE_PREC_FP64, nrhs, xd, yd)
        fe.fe_spmv_half(ctx, s, fe.FE_PREC_MIXED, nrhs, x32, y32)
        fe.fe_ctx_synchronize(ctx)
        y64 = yd.cpu().numpy()
        y32h = y32.cpu().numpy().astype(np.complex128)
    finally:
        fe.fe_system_destroy(s)
        fe.fe_mesh_destroy(m)
    ref = A @ x
    bound = abs(A) @ np.abs(x)
    assert np.all(np.abs(y64 - ref) <= 1e-13 * bound + 1e-300)
    assert np.all(np.abs(y32h - ref) <= 4e-6 * bound)


@pytest.mark.parametrize("nrhs", [1, 2, 8])
@pytest.mark.parametrize("seed", [5, 9])
def test_half_spmv_small(fe, ctx, seed, nrhs):
    _half_check(fe, ctx, W.random_small_grid(seed, n_max=8, n_pec_boxes=2), nrhs, seed=seed)


def test_half_spmv_variant_p(fe):
    c = fe.fe_ctx_create(0, variant=fe.FE_VARIANT_P)
    try:
        _half_check(fe, c, W.random_small_grid(3, n_max=7, n_pec_boxes=2), 1, variant="P")
    finally:
        fe.fe_ctx_destroy(c)


def test_half_spmv_config2(fe, ctx):
    _half_check(fe, ctx, W.config2()[0], 1, seed=3)


def test_half_argument_errors(fe, ctx):
    import torch
    prob = W.random_small_grid(4, n_max=6)
    m = fe.fe_mesh_create_from(ctx, prob)
    s = fe.fe_assemble(ctx, m, prob.freq_hz, fe.FE_PREC_FP64)
    n = fe.fe_mesh_info(m)["n_dof"]
    x = torch.zeros((n, 1), dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    try:
        with pytest.raises(fe.FeError) as e:            # not packed yet
            fe.fe_spmv_half(ctx, s, fe.FE_PREC_FP64, 1, x, y)
        assert e.value.status == fe.FE_ERR_INVALID_ARG
        before = fe.fe_system_info(s)["device_bytes"]
        kept = fe.fe_system_pack_half(ctx, s)
        assert fe.fe_system_info(s)["device_bytes"] - before >= kept * 9 * 16   # counted with the system
        for prec, nrhs in ((fe.FE_PREC_MIXED, 1), (fe.FE_PREC_DF, 1), (fe.FE_PREC_FP64, 3)):
            with pytest.raises(fe.FeError) as e:         # no complex64 copy; DF; nrhs not a power of two
                fe.fe_spmv_half(ctx, s, prec, nrhs, x, y)
            assert e.value.status == fe.FE_ERR_INVALID_ARG
        fe.fe_spmv_half(ctx, s, fe.FE_PREC_FP64, 1, x, y)
        fe.fe_ctx_synchronize(ctx)
    finally:
        fe.fe_system_destroy(s)
        fe.fe_mesh_destroy(m)
    c = fe.fe_ctx_create(0, variant=fe.FE_VARIANT_L)
    try:
        m = fe.fe_mesh_create_from(c, prob)
        s = fe.fe_assemble(c, m, prob.freq_hz, fe.FE_PREC_FP64)
        try:
            with pytest.raises(fe.FeError) as e:         # the literal Eq. 4 matrix is not symmetric
                fe.fe_system_pack_half(c, s)
            assert e.value.status == fe.FE_ERR_INVALID_ARG
        finally:
            fe.fe_system_destroy(s)
            fe.fe_mesh_destroy(m)
    finally:
        fe.fe_ctx_destroy(c)

