"""Failure detection on the GPU without a fault.

Every device-side wait of the persistent solve (the grid barriers, the
completion of the halo copy) is bounded.  Here the bound is set far below
the latency of a grid barrier across the device's CTAs (1 microsecond), so a
wait runs out: the kernel records the expiry in its status word, every CTA
leaves at its next barrier, a halo copy in flight is waited for before its
CTA leaves, and the host reports FE_ERR_TIMEOUT.  The same context must then
solve normally.  Nothing faults, traps or hangs.
"""
import numpy as np
import pytest

from oracle import fem
from paper_0704_2344_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,nrhs", [("DF", 1), ("FP64", 4), ("MIXED", 1)])
def test_expired_wait_is_reported_and_context_survives(fe, ctx, precision, nrhs):
    prob, _ = W.config1()
    waves = W.random_waves(nrhs, np.random.default_rng(9))
    prec = getattr(fe, f"FE_PREC_{precision}")
    mesh = fe.fe_mesh_create_from(ctx, prob)
    system = fe.fe_assemble(ctx, mesh, prob.freq_hz, prec)
    try:
        n_dof = fe.fe_mesh_info(mesh)["n_dof"]
        with pytest.raises(fe.FeError) as err:
            fe.fe_solve_batch(ctx, system, waves, n_dof, fe.solve_opts(precision=prec, wait_timeout_us=1))
        assert err.value.status == fe.FE_ERR_TIMEOUT
        assert "expired" in str(err.value)
        # the context and the system are intact: a normal solve succeeds
        fe.fe_ctx_synchronize(ctx)
        st, x, rep = fe.fe_solve_batch(ctx, system, waves, n_dof, fe.solve_opts(precision=prec))
        assert st == fe.FE_OK and all(r["status"] == fe.FE_OK for r in rep)
        maps = fem.mesh_maps(prob)
        A = fem.assemble(prob, maps=maps)
        B = fem.rhs(prob, waves, maps=maps)
        assert fem.true_relative_residual(A, x, B).max() <= 1e-8
    finally:
        fe.fe_system_destroy(system)
        fe.fe_mesh_destroy(mesh)
