"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function include/sq.h declares (no compute calls without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sq_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2007_06524_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("sq_build_coeffs", "sq_precond_setup", "sq_pcg_solve", "sq_homogenized_matrix",
                     "sq_workspace_create", "sq_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], stdout=subprocess.PIPE, text=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_reports_errors(libpath):
    import paper_2007_06524_gb300 as sq

    lib = sq.load_library()
    for name in _declared():
        assert hasattr(lib, name)
    assert sq.sq_strerror(sq.SQ_EINVAL) == "invalid argument"
    assert sq.sq_strerror(sq.SQ_ENOCONV).startswith("not converged")


def test_binding_names_match_header():
    import paper_2007_06524_gb300 as sq

    for name in _declared():
        if name.endswith("_destroy"):
            continue
        assert hasattr(sq, name), name
