"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/fe.h (no compute call: this runs without a GPU)."""
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def declared():
    txt = (ROOT / "include" / "fe.h").read_text()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fe_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ["fe_ctx_create", "fe_mesh_create", "fe_mesh_export_maps", "fe_assemble", "fe_system_export",
              "fe_rhs", "fe_spmv", "fe_solve_batch", "fe_solve_rhs", "fe_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(fe):
    import ctypes
    lib = fe.load()
    for n in declared():
        assert isinstance(getattr(lib, n), ctypes._CFuncPtr), n


def test_nm_exports(fe):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", str(fe.LIB_PATH)], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (fe_[a-z0-9_]+)\b", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing


def test_option_defaults_without_gpu(fe):
    import ctypes
    o = fe.fe_solve_opts()
    o.preconditioner = 77                       # the C default writes the struct's last field too
    fe.load().fe_solve_opts_default(ctypes.byref(o))
    assert o.precision == fe.FE_PREC_DF and o.tol == 1e-8 and o.max_iter == 100000 and o.max_pass_iter == 2000
    assert o.preconditioner == fe.FE_PRECOND_BLOCK_JACOBI
    s = fe.fe_serve_opts()
    fe.load().fe_serve_opts_default(ctypes.byref(s))
    assert s.precision == fe.FE_PREC_DF and s.tol == 1e-8 and s.work_per_cta == 2048
    opt = fe.fe_options()
    fe.load().fe_options_default(ctypes.byref(opt))
    assert opt.variant == fe.FE_VARIANT_S and opt.abc_sigma == 1.0 and opt.penalty_s == 1.0
