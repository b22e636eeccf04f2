"""The C-ABI library builds, loads and exports every entry point include/qxd.h declares.

No GPU needed: only calls that return before touching CUDA are made."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def qxd():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2502_02490_gb300 import qxd as q

    return q


def declared_functions():
    src = open(os.path.join(ROOT, "include", "qxd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qxd_[A-Za-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["qxd_create_lattice", "qxd_destroy_lattice", "qxd_load_gauge", "qxd_build_clover",
                     "qxd_apply_D", "qxd_apply_Dhat_eo", "qxd_solve"]:
        assert required in names


def test_library_exports_every_declared_symbol(qxd):
    lib = ctypes.CDLL(qxd.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_invalid_extents_rejected_without_gpu(qxd):
    for L in [(3, 4, 4, 4), (4, 4, 4, 0), (4, 4, 5, 4)]:
        with pytest.raises(qxd.QxdError) as e:
            qxd.create_lattice(L)
        assert e.value.status == qxd.EINVAL
    assert "even" in qxd.last_error(None)


def test_default_params(qxd):
    p = qxd.default_params()
    assert p.version == qxd.PARAMS_VERSION and p.tol == 1e-10 and p.solver == qxd.SOLVER_MP_CG_EO
    assert p.gcr_restart == 16 and p.gcr_reorth == 1 and p.check_every == 1 and p.fallback == -1
    assert qxd.lib.qxd_destroy_lattice(None) == qxd.OK
    assert qxd.launch_count(None) == 0
