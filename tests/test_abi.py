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
    # the boundary's call list: the operator and solve calls, the batched solve, the one-call
    # training of the preconditioner, its checkpoint, the clover export and the error message
    for required in ["qxd_create_lattice", "qxd_destroy_lattice", "qxd_load_gauge", "qxd_build_clover",
                     "qxd_get_clover", "qxd_apply_D", "qxd_apply_Dhat_eo", "qxd_solve", "qxd_solve_batch",
                     "qxd_train_precond", "qxd_net_save", "qxd_net_load", "qxd_last_error"]:
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
    assert p.use_x0 == 0 and p.restart_f32 == 1
    assert list(p.sap_block) == [4, 4, 4, 4] and p.sap_ncy == 2 and p.sap_nmr == 4
    assert list(qxd.default_params(sap_block=(2, 2, 2, 4)).sap_block) == [2, 2, 2, 4]
    assert qxd.lib.qxd_destroy_lattice(None) == qxd.OK
    import ctypes as C

    assert qxd.lib.qxd_check_guards(None, C.byref(C.c_int64())) == qxd.EINVAL
    assert qxd.launch_count(None) == 0


def test_params_struct_matches_library_layout(qxd):
    """qxd_default_params writes exactly sizeof(SolveParams) bytes, ending with the version-4 fields."""
    import ctypes as C

    n = C.sizeof(qxd.SolveParams)
    buf = (C.c_ubyte * (n + 64))(*([0xA5] * (n + 64)))
    qxd.lib.qxd_default_params(C.cast(buf, C.POINTER(qxd.SolveParams)))
    p = qxd.SolveParams.from_buffer(buf)
    assert p.version == qxd.PARAMS_VERSION and p.restart_f32 == 1 and p.use_x0 == 0 and p.fallback == -1
    assert bytes(buf[n:]) == bytes([0xA5] * 64)
    # a version-3 struct ends where use_x0 begins, a version-4 struct where sap_block begins
    assert qxd.SolveParams.use_x0.offset == qxd.SolveParams.fallback.offset + C.sizeof(C.c_int)
    assert qxd.SolveParams.use_x0.offset % 8 == 0
    assert qxd.SolveParams.sap_block.offset == qxd.SolveParams.restart_f32.offset + C.sizeof(C.c_int)


def test_train_params_layout_and_binding_checks(qxd):
    """Version-2 training params append the one-call fields after eps; the binding rejects a channel
    list the library cannot hold before any call."""
    import ctypes as C

    T = qxd.TrainParams
    assert qxd.TRAIN_VERSION == 2 and T.nlayers.offset == T.eps.offset + C.sizeof(C.c_double)
    assert T.channels.size == 9 * C.sizeof(C.c_int)
    with pytest.raises(ValueError):
        qxd.train_precond(None, [1] * 10, nsamp=1, sample_seed=0)
    assert qxd.lib.qxd_train_precond(None, None, None) == qxd.EINVAL


def test_without_a_gpu_calls_fail_with_a_status_not_an_abort(qxd):
    """Every entry point returns a status: on a machine without a usable GPU, creating a lattice
    reports QXD_ECUDA with the CUDA message instead of aborting the process."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(qxd.QxdError) as e:
        qxd.create_lattice((4, 4, 4, 4))
    assert e.value.status == qxd.ECUDA and "cuda" in qxd.last_error(None).lower()


def test_multigrid_entry_points_and_params_layout(qxd):
    """The multigrid calls refuse a NULL lattice with QXD_EINVAL before touching CUDA, and the
    binding's parameter struct has the header's layout (version, agg[4], then six ints)."""
    import ctypes as C

    P = qxd.MgParams
    assert C.sizeof(P) == 11 * C.sizeof(C.c_int) and P.agg.offset == C.sizeof(C.c_int)
    assert P.ncy_pre.offset == 10 * C.sizeof(C.c_int) and qxd.MG_VERSION == 1
    p = qxd.mg_params(agg=(2, 2, 2, 2), ns2=8)
    assert list(p.agg) == [2, 2, 2, 2] and p.version == qxd.MG_VERSION and p.m == 8
    lib = qxd.lib
    assert lib.qxd_mg_setup(None, C.byref(p), None, 0) == qxd.EINVAL
    assert lib.qxd_mg_generate(None, 1, 1, 1, None, None, 0) == qxd.EINVAL
    assert lib.qxd_mg_get_coarse(None, None, None) == qxd.EINVAL
    assert lib.qxd_mg_info(None, None, None, None) == qxd.EINVAL
    assert lib.qxd_mg_apply_level1(None, None, None, 0) == qxd.EINVAL
    assert lib.qxd_mg_precond(None, None, None, None, 1, 1, 0) == qxd.EINVAL
    assert qxd.SOLVER_MP_MG_GCR == 7


def test_noalloc_forget_needs_no_device(qxd):
    """qxd_vec_dot_noalloc_forget only drops host-side cached addresses: it returns QXD_OK on a
    machine without a GPU, and calling it twice is harmless."""
    assert qxd.lib.qxd_vec_dot_noalloc_forget() == qxd.OK
    qxd.vec_dot_noalloc_forget()
