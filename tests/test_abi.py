"""CPU checks of the boundary: libsap builds, loads without a GPU and exports
every entry point that the headers under include/ declare (no compute calls
here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def declared_symbols():
    src = "".join(open(os.path.join(INCLUDE, f)).read() for f in sorted(os.listdir(INCLUDE)) if f.endswith(".h"))
    return sorted(set(re.findall(r"SAP_API\s+[\w\s\*]*?\b(sap_\w+)\s*\(", src)))


def test_header_declares_the_entry_points():
    names = declared_symbols()
    for must in ("sap_factor", "sap_solve", "sap_solve_adjoint", "sap_grad_band", "sap_spmv",
                 "sap_apply_preconditioner", "sap_destroy", "sap_status_string", "sap_db_reorder",
                 "sap_cm_reorder", "sap_sparse_to_band"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    lib_path = __graft_entry__._load_build_module().build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    lib.sap_status_string.restype = ctypes.c_char_p
    assert lib.sap_status_string(0) == b"ok"
    assert lib.sap_max_K(1) >= 64


def test_package_refuses_to_run_without_library(tmp_path, monkeypatch):
    """The binding raises at import when libsap.so is absent (no CPU fallback)."""
    import importlib.util
    import shutil
    pkg = tmp_path / "paper_1509_07919_gb300"
    shutil.copytree(os.path.join(ROOT, "paper_1509_07919_gb300"), pkg,
                    ignore=shutil.ignore_patterns("*.so", "_build", "__pycache__"))
    spec = importlib.util.spec_from_file_location("sap_nolib", pkg / "__init__.py",
                                                  submodule_search_locations=[str(pkg)])
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError):
        spec.loader.exec_module(mod)


def test_host_only_calls_on_cpu():
    """Entry points that need no GPU: the K limits (the sweep ring's shared
    memory, two chunks ahead: 512 for FP32 factors with or without the
    tensor-core update, 256 for FP64), the status strings of every status and
    the default options."""
    import paper_1509_07919_gb300 as S
    assert S.sap_max_K(S.SAP_FP64) == 256
    assert S.sap_max_K(S.SAP_FP32) == 512 and S.sap_max_K(S.SAP_FP32_BF16TU) == 512
    names = {st: S.sap_status_string(st) for st in range(0, 10)}
    assert names[S.SAP_OK] == "ok"
    assert len(set(names.values())) >= 8          # distinct messages for the defined statuses
    o = S.sap_default_options()
    assert (o.P, o.variant, o.precision, o.max_iters, o.tol, o.segments, o.krylov) == \
        (1, S.SAP_D, S.SAP_FP64, 500, 1e-10, 0, 0)
