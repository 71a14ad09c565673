"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function declared in include/bspai.h (no compute calls here)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "bspai.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\**\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    from paper_2307_03914_gb300 import build

    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = _declared_functions()
    for need in ["bspai_build", "bspai_bucket", "bspai_apply", "gmres_ir_solve", "bspai_free",
                 "bspai_last_error"]:
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_no_gpu_calls_needed_to_query(lib):
    lib.bspai_version.restype = ctypes.c_int
    assert lib.bspai_version() >= 100
    lib.bspai_last_error.restype = ctypes.c_char_p
    assert lib.bspai_last_error() == b"no error"
    # invalid arguments are rejected on the host, before any CUDA call
    lib.bspai_free.argtypes = [ctypes.c_void_p]
    bogus = ctypes.create_string_buffer(16)
    assert lib.bspai_free(ctypes.cast(bogus, ctypes.c_void_p)) == 1  # BSPAI_ERR_INVALID
    assert b"not a live bspai handle" in lib.bspai_last_error()


def test_binding_imports_and_mirrors_names(lib):
    from paper_2307_03914_gb300 import bspai

    for n in ["bspai_build", "bspai_bucket", "apply", "gmres_ir_solve", "gmres", "residual", "spmv_up",
              "matrix_create", "M_export", "bucket_export", "apply_uf"]:
        assert hasattr(bspai, n), n


def test_ctypes_structs_match_header_sizes():
    """Struct layouts in the binding agree with the header (field count and order)."""
    from paper_2307_03914_gb300 import bspai

    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "bspai.h")).read(), flags=re.S)
    for cname, py in [("bspai_opts_t", bspai.Opts), ("bspai_solve_info_t", bspai.SolveInfo),
                      ("bspai_bucket_info_t", bspai.BucketInfo), ("bspai_build_info_t", bspai.BuildInfo),
                      ("bspai_csr_t", bspai.CsrT), ("bspai_gmres_plan_t", bspai.GmresPlan),
                      ("bspai_batch_info_t", bspai.BatchInfo), ("bspai_batch_schedule_t", bspai.BatchSchedule)]:
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + cname + ";", src).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = re.findall(r"([A-Za-z_][A-Za-z0-9_]*)\s*(?:\[[^\]]*\])?\s*;", body)
        assert fields == [f for f, _ in py._fields_], cname
