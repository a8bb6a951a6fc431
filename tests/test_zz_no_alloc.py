"""GPU test of fe_solve_rhs_noalloc, the solve entry point that allocates
nothing.

Some callers cannot let a library allocate device memory in the middle of
their work: code that is already inside a CUDA stream capture (an allocation
there breaks the capture), a host thread that must not block on the device
allocator, or an application that owns every allocation of its process.  For
them the library keeps the solve's workspace in one fixed device array and
this entry point uses only that array and the caller's buffers.

The test calls it through the C ABI twice in a row (the array keeps the
previous call's contents) and compares each result with the allocating entry
point fe_solve_rhs, within the field tolerance of the other solve tests, and
checks the FP64 true residual with the CPU oracle's matrix.  This file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

from oracle import fem
from paper_0704_2344_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["MIXED", "FP64", "DF"])
def test_noalloc_solve_matches_allocating_solve(fe, ctx, precision):
    import torch

    prec = getattr(fe, f"FE_PREC_{precision}")
    prob = W.random_small_grid(8, n_max=7, n_pec_boxes=1)
    waves = W.random_waves(4, np.random.default_rng(2))
    A = fem.assemble(prob)
    mesh = fe.fe_mesh_create_from(ctx, prob)
    system = fe.fe_assemble(ctx, mesh, prob.freq_hz, prec)
    try:
        n_dof = fe.fe_mesh_info(mesh)["n_dof"]
        B = fe.fe_rhs(ctx, system, waves, n_dof)
        opts = fe.solve_opts(precision=prec)
        _, x_ref, rep_ref = fe.fe_solve_rhs(ctx, system, B, 4, opts)
        assert all(r["status"] == fe.FE_OK for r in rep_ref)
        b_dev = torch.from_numpy(B).cuda()
        for call in range(2):
            # stale contents in the output buffer: without use_x0 they must not matter
            x_dev = torch.full_like(b_dev, complex(call + 1.0, -1.0))
            torch.cuda.synchronize()
            st, rep = fe.fe_solve_rhs_noalloc(ctx, system, 4, b_dev, x_dev, opts)
            x = x_dev.cpu().numpy()
            assert st == fe.FE_OK and all(r["status"] == fe.FE_OK for r in rep)
            assert np.linalg.norm(x - x_ref) <= 1e-6 * np.linalg.norm(x_ref)
            assert fem.true_relative_residual(A, x, B).max() <= 1e-8
    finally:
        fe.fe_system_destroy(system)
        fe.fe_mesh_destroy(mesh)


def test_noalloc_rejects_sizes_beyond_its_scratch(fe, ctx):
    import torch

    prob, _ = W.config2()  # 88 998 unknowns: 8 right-hand sides need more than the 32 MiB array
    mesh = fe.fe_mesh_create_from(ctx, prob)
    system = fe.fe_assemble(ctx, mesh, prob.freq_hz, fe.FE_PREC_MIXED)
    try:
        n_dof = fe.fe_mesh_info(mesh)["n_dof"]
        b = torch.zeros((n_dof, 8), dtype=torch.complex128, device="cuda")
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        with pytest.raises(fe.FeError) as err:
            fe.fe_solve_rhs_noalloc(ctx, system, 8, b, x, fe.solve_opts(precision=fe.FE_PREC_MIXED))
        assert err.value.status == fe.FE_ERR_INVALID_ARG
        assert "scratch" in str(err.value)
        with pytest.raises(fe.FeError) as err:
            fe.fe_solve_rhs_noalloc(ctx, system, 3, b, x, fe.solve_opts(precision=fe.FE_PREC_MIXED))  # not a width
        assert err.value.status == fe.FE_ERR_INVALID_ARG
    finally:
        fe.fe_system_destroy(system)
        fe.fe_mesh_destroy(mesh)
