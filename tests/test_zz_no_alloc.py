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


def test_noalloc_rejects_host_and_misshapen_buffers(fe, ctx):
    """The kernel reads b and writes x in place, so the C entry point itself
    rejects host memory (before any GPU work), and the binding rejects
    tensors of another type, layout or shape."""
    import ctypes as C

    import torch

    prob = W.random_small_grid(9, n_max=5, n_pec_boxes=1)
    mesh = fe.fe_mesh_create_from(ctx, prob)
    system = fe.fe_assemble(ctx, mesh, prob.freq_hz, fe.FE_PREC_DF)
    try:
        n_dof = fe.fe_mesh_info(mesh)["n_dof"]
        b_host = np.zeros((n_dof, 1), np.complex128)
        x_host = np.zeros((n_dof, 1), np.complex128)
        opts = fe.solve_opts(precision=fe.FE_PREC_DF)
        rep = (fe.fe_solve_report * 1)()
        st = fe.load().fe_solve_rhs_noalloc(ctx, system, 1, b_host.ctypes.data_as(C.c_void_p),
                                            x_host.ctypes.data_as(C.c_void_p), 0, C.byref(opts), rep)
        assert st == fe.FE_ERR_INVALID_ARG
        assert "device memory" in fe.fe_last_error()
        b = torch.zeros((n_dof, 1), dtype=torch.complex128, device="cuda")
        bad = [torch.zeros((n_dof, 1), dtype=torch.complex64, device="cuda"),       # wrong type
               torch.zeros((n_dof, 2), dtype=torch.complex128, device="cuda")[:, :1],  # not contiguous
               torch.zeros((n_dof + 3, 1), dtype=torch.complex128, device="cuda"),  # wrong shape
               x_host]                                                               # host array
        for x in bad:
            with pytest.raises(fe.FeError) as err:
                fe.fe_solve_rhs_noalloc(ctx, system, 1, b, x, opts)
            assert err.value.status == fe.FE_ERR_INVALID_ARG
    finally:
        fe.fe_system_destroy(system)
        fe.fe_mesh_destroy(mesh)


@pytest.mark.parametrize("precision", ["DF", "MIXED"])
def test_noalloc_resumes_from_an_initial_guess(fe, ctx, precision):
    """use_x0 = 1: x_dev holds the starting point.  Started from a solution cut
    short at a loose tolerance, the call reaches the same field as a solve
    from zero (1e-6), with a true residual of 1e-8."""
    import torch

    prec = getattr(fe, f"FE_PREC_{precision}")
    prob = W.random_small_grid(8, n_max=7, n_pec_boxes=1)
    waves = W.random_waves(2, np.random.default_rng(4))
    A = fem.assemble(prob)
    mesh = fe.fe_mesh_create_from(ctx, prob)
    system = fe.fe_assemble(ctx, mesh, prob.freq_hz, prec)
    try:
        n_dof = fe.fe_mesh_info(mesh)["n_dof"]
        B = fe.fe_rhs(ctx, system, waves, n_dof)
        _, x_ref, _ = fe.fe_solve_rhs(ctx, system, B, 2, fe.solve_opts(precision=prec))
        _, x0, _ = fe.fe_solve_rhs(ctx, system, B, 2, fe.solve_opts(precision=prec, tol=1e-3))
        assert fem.true_relative_residual(A, x0, B).max() > 1e-6   # a real head start, not the answer
        b_dev = torch.from_numpy(B).cuda()
        x_dev = torch.from_numpy(np.ascontiguousarray(x0)).cuda()
        torch.cuda.synchronize()
        st, rep = fe.fe_solve_rhs_noalloc(ctx, system, 2, b_dev, x_dev, fe.solve_opts(precision=prec), use_x0=True)
        x = x_dev.cpu().numpy()
        assert st == fe.FE_OK and all(r["status"] == fe.FE_OK for r in rep)
        assert fem.true_relative_residual(A, x, B).max() <= 1e-8
        assert np.linalg.norm(x - x_ref) <= 1e-6 * np.linalg.norm(x_ref)
    finally:
        fe.fe_system_destroy(system)
        fe.fe_mesh_destroy(mesh)


def test_noalloc_fp32_pair_limit_of_one_column(fe, ctx):
    """One column in the FP32-pair mode needs 80 bytes per unknown: a 51^3
    box (421 824 unknowns, 33.7 MB) is rejected, a 50^3 box (397 953
    unknowns, 31.8 MB) fits the 32 MiB array."""
    import torch

    for n, fits in ((51, False), (50, True)):
        prob = W.empty_box(n)
        mesh = fe.fe_mesh_create_from(ctx, prob)
        system = fe.fe_assemble(ctx, mesh, prob.freq_hz, fe.FE_PREC_DF)
        try:
            n_dof = fe.fe_mesh_info(mesh)["n_dof"]
            assert n_dof == 3 * (n + 1) ** 3
            B = fe.fe_rhs(ctx, system, W.normal_incidence(), n_dof)
            b = torch.from_numpy(B).cuda()
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            opts = fe.solve_opts(precision=fe.FE_PREC_DF)
            if fits:
                st, rep = fe.fe_solve_rhs_noalloc(ctx, system, 1, b, x, opts)
                assert st == fe.FE_OK and rep[0]["rel_residual"] <= 1e-8
            else:
                with pytest.raises(fe.FeError) as err:
                    fe.fe_solve_rhs_noalloc(ctx, system, 1, b, x, opts)
                assert err.value.status == fe.FE_ERR_INVALID_ARG and "scratch" in str(err.value)
        finally:
            fe.fe_system_destroy(system)
            fe.fe_mesh_destroy(mesh)
