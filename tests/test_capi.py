"""The C-ABI library builds, loads and exports every symbol include/fv.h
declares (no GPU calls)."""
import os
import re
import subprocess

import pytest

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "fv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fv_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libfv():
    from paper_1704_01144_gb300 import build, fv
    build.build()
    return fv.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("fv_mesh_load", "fv_assign_levels", "fv_residual_level", "fv_advance"):
        assert required in names


def test_library_exports_every_declared_symbol(libfv):
    from paper_1704_01144_gb300 import fv
    out = subprocess.run(["nm", "-D", "--defined-only", fv.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.split() and ln.split()[-2] == "T"}
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        getattr(libfv, n)
    # the binding covers the whole boundary, and nothing else
    assert sorted(fv.EXPORTS) == _declared()


def test_version_and_defaults(libfv):
    from paper_1704_01144_gb300 import fv
    assert "sm_103a" in fv.fv_version()
    cfg = fv.fv_config_default()
    assert cfg.gamma == 1.4 and cfg.cfl == 0.5 and cfg.newton_tol == 1e-10
    assert cfg.newton_max_iter == 50 and cfg.max_levels == 1


def test_library_is_built_for_sm_103a_only(libfv):
    from paper_1704_01144_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_null_handle_is_rejected_without_gpu(libfv):
    from paper_1704_01144_gb300 import fv
    import ctypes as C
    assert libfv.fv_status(None) == fv.FV_ERR_INVALID_ARG
    assert libfv.fv_advance(None, 1, None, None) == fv.FV_ERR_INVALID_ARG
    assert "fv_advance" in fv.fv_last_error()
    out = C.c_void_p(1)
    assert libfv.fv_mesh_load(None, 0, None, 0, None, None, C.byref(out)) == fv.FV_ERR_INVALID_ARG
    assert out.value is None


@pytest.mark.parametrize("std,compiler,flags", [("c99", "gcc", ["-x", "c"]), ("c++17", "g++", ["-x", "c++"])])
def test_header_is_plain_c_and_cxx(tmp_path, std, compiler, flags):
    """include/fv.h is a C ABI: it compiles on its own as pedantic C99 (no
    C++ constructs outside its extern "C" guard) and as C++, warning-free."""
    import shutil
    import subprocess
    if shutil.which(compiler) is None:
        pytest.skip(f"{compiler} not found")
    src = tmp_path / "use_header.c"
    src.write_text('#include "fv.h"\nint main(void) { fv_config c; (void)c; return FV_OK; }\n')
    r = subprocess.run([compiler, *flags, f"-std={std}", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), "-c", str(src), "-o", str(tmp_path / "o.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_product_path_fails_loudly_without_a_gpu_or_library(libfv, monkeypatch):
    """There is no CPU fallback: without a CUDA device the first call that
    needs one raises FvError with FV_ERR_CUDA, and without the built library
    the binding raises ImportError."""
    import torch
    from paper_1704_01144_gb300 import fv, inputs as I
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    mesh, _ = I.blast_case(n=3)
    with pytest.raises(fv.FvError, match="FV_ERR_CUDA"):
        fv.Mesh(mesh, max_levels=2)
    monkeypatch.setattr(fv, "_lib", None)
    monkeypatch.setattr(fv, "library_path", lambda: os.path.join(ROOT, "no_such_libfv.so"))
    with pytest.raises(ImportError, match="no CPU fallback"):
        fv.lib()


def test_empty_inputs_are_refused_or_no_ops_without_gpu(libfv):
    """Empty inputs are decided before any device call: an empty mesh and an
    empty batch are refused with FV_ERR_INVALID_ARG, an empty flux batch is
    a no-op (FV_OK, nothing read or written)."""
    import ctypes as C
    from paper_1704_01144_gb300 import fv
    cfg = fv.fv_config_default()
    xyz = (C.c_double * 3)()
    tets = (C.c_int64 * 4)()
    bc = (C.c_int8 * 4)()
    out = C.c_void_p(1)
    rc = libfv.fv_mesh_load(xyz, 1, tets, 0, bc, C.byref(cfg), C.byref(out))
    assert rc == fv.FV_ERR_INVALID_ARG and out.value is None and "bad sizes" in fv.fv_last_error()
    rc = libfv.fv_mesh_load(xyz, 0, tets, 1, bc, C.byref(cfg), C.byref(out))
    assert rc == fv.FV_ERR_INVALID_ARG
    meshes = (C.c_void_p * 1)()
    assert libfv.fv_batch_create(meshes, 0, C.byref(out)) == fv.FV_ERR_INVALID_ARG
    dummy = C.c_void_p(256)  # never dereferenced: nothing to do for count 0
    assert libfv.fv_godunov_flux_batch(dummy, dummy, dummy, 0, C.byref(cfg), 0, dummy, dummy,
                                       None) == fv.FV_OK
