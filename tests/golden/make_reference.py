"""Writes the stored oracle reference solutions used by the GPU parity tests
at full size (where a direct solve takes minutes on a CPU).

Calls only the oracle (oracle/) on inputs from the seeded generators; run from
the repository root:  python tests/golden/make_reference.py [config2 config3 aircraft40]
Outputs (x as complex64 is enough for a 1e-6 relative field comparison: its
rounding is ~6e-8 relative):
  tests/golden/config2_x.npz     the 3-wavelength cube, one wave, SuperLU;
  tests/golden/config3_x.npz     the same mesh with the 64 sphere waves, SuperLU:
                                 the columns in CONFIG3_COLUMNS (two of each
                                 32-column launch) in full, and all 64 on a
                                 seeded sample of CONFIG3_SAMPLE unknowns;
  tests/golden/aircraft40_x.npz  the 40^3 aircraft with the first of the
                                 large-scatterer waves, the oracle's COCG down
                                 to a true residual of 1e-12 (a direct
                                 factorisation of its 206 k unknowns takes
                                 about an hour on one core)."""
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

from oracle import fem, krylov  # noqa: E402
from paper_0704_2344_gb300 import workloads as W  # noqa: E402

HERE = Path(__file__).resolve().parent
CONFIG3_COLUMNS = (0, 17, 32, 63)
CONFIG3_SAMPLE = 4096


def config2():
    prob, waves = W.config2()
    t = time.time()
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps)
    B = fem.rhs(prob, waves, maps=maps)
    X = fem.solve_direct(A, B)
    res = fem.true_relative_residual(A, X, B)
    print("config 2: n_dof", maps.n_dof, "solve s", round(time.time() - t, 1), "residual", res)
    t = time.time()
    xc, its, _ = krylov.cocg(A, B[:, 0], tol=1e-8)
    t_cocg = time.time() - t
    print("oracle COCG: iterations", its, "s", round(t_cocg, 1))
    np.savez_compressed(HERE / "config2_x.npz", x=X.astype(np.complex64),
                        residual=res, n_dof=maps.n_dof, cocg_iterations=its, cocg_seconds=t_cocg)


def config3():
    prob, waves = W.config3()
    t = time.time()
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps)
    B = fem.rhs(prob, waves, maps=maps)
    X = fem.solve_direct(A, B)
    res = fem.true_relative_residual(A, X, B)
    print("config 3: n_dof", maps.n_dof, "solve s", round(time.time() - t, 1), "max residual", res.max())
    cols = np.array(CONFIG3_COLUMNS)
    # every column on a seeded sample of unknowns, for a per-column field check of all 64
    rows = np.sort(np.random.default_rng(20070704 + 33).choice(maps.n_dof, size=CONFIG3_SAMPLE, replace=False))
    np.savez_compressed(HERE / "config3_x.npz", x=X[:, cols].astype(np.complex64), columns=cols,
                        residual=res[cols], n_dof=maps.n_dof, sample_rows=rows,
                        x_sample=X[rows, :].astype(np.complex64), residual_all=res)


def aircraft40():
    prob = W.aircraft_mesh(40, 4)
    waves = W.config4()[1].column(0)
    t = time.time()
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps)
    B = fem.rhs(prob, waves, maps=maps)
    x, its, _ = krylov.cocg(A, B[:, 0], tol=1e-12, maxiter=200000)
    res = fem.true_relative_residual(A, x[:, None], B)[0]
    print("aircraft 40^3: n_dof", maps.n_dof, "COCG iterations", its, "s", round(time.time() - t, 1),
          "true residual", res)
    np.savez_compressed(HERE / "aircraft40_x.npz", x=x.astype(np.complex64), residual=res, n_dof=maps.n_dof,
                        cocg_iterations=its)


if __name__ == "__main__":
    jobs = {"config2": config2, "config3": config3, "aircraft40": aircraft40}
    for name in (sys.argv[1:] or list(jobs)):
        jobs[name]()
