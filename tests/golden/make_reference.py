"""Writes the stored oracle reference solutions used by the GPU parity tests
at full size (where a direct solve takes minutes on a CPU).

Calls only the oracle (oracle/) on inputs from the seeded generators; run from
the repository root:  python tests/golden/make_reference.py
Output: tests/golden/config2_x.npz  (x as complex64 is enough for a 1e-6
relative field comparison: its rounding is ~6e-8 relative)."""
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

from oracle import fem, krylov  # noqa: E402
from paper_0704_2344_gb300 import workloads as W  # noqa: E402


def main():
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
    np.savez_compressed(Path(__file__).with_name("config2_x.npz"), x=X.astype(np.complex64),
                        residual=res, n_dof=maps.n_dof, cocg_iterations=its, cocg_seconds=t_cocg)


if __name__ == "__main__":
    main()
