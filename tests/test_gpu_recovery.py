"""Solver restart and recovery: an initial guess (resume from a stored solution), the FP32-inner
restart of a 16-bit mixed-precision solve, the plain fallback solver, and the version-3 params
layout.  Every solution is judged by the oracle's FP64 true residual."""
import ctypes as C

import numpy as np
import pytest

from oracle import qxd_oracle as O
from paper_2502_02490_gb300 import synth
from tests.gpu_util import Case, as_c128

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def qxd():
    import __graft_entry__

    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_02490_gb300 import qxd as q

    return q


@pytest.mark.parametrize("solver,prec", [(0, 1), (1, 1), (2, 2), (3, 1)])
def test_initial_guess_resumes_a_solve(qxd, solver, prec):
    c = Case(qxd, torch, (4, 4, 4, 4))
    try:
        eta = synth.gaussian_spinor(c.dims, 2200)
        b = c.dev_tensor(eta)
        kw = dict(solver=solver, inner_prec=prec, gcr_restart=16)
        x = torch.empty_like(b)
        st, full = qxd.solve(c.lat, x, b, tol=1e-10, **kw)
        x1 = torch.empty_like(b)
        st, part = qxd.solve(c.lat, x1, b, tol=1e-5, **kw)
        r1 = O.true_rel_residual(c.op, as_c128(x1, eta.shape), eta)
        assert 1e-10 < r1 <= 1e-5
        st, rest = qxd.solve(c.lat, x1, b, tol=1e-10, use_x0=1, **kw)
        assert st == qxd.OK
        assert O.true_rel_residual(c.op, as_c128(x1, eta.shape), eta) <= 1e-10
        assert rest["iters_inner"] < full["iters_inner"], (rest, full)
        # a converged guess is returned as it is
        before = x1.clone()
        st, again = qxd.solve(c.lat, x1, b, tol=1e-10, use_x0=1, **kw)
        assert st == qxd.OK and again["iters_inner"] == 0 and again["iters_outer"] == 0
        assert torch.equal(before, x1)
    finally:
        c.close()


def test_initial_guess_from_host_memory_and_zero_source(qxd):
    c = Case(qxd, torch, (4, 2, 2, 4), cstar=True)
    try:
        eta = synth.gaussian_spinor(c.dims, 2201)
        b = np.ascontiguousarray(eta)
        x = np.zeros_like(b)
        st, _ = qxd.solve(c.lat, x, b, tol=1e-4, solver=qxd.SOLVER_MP_BICGSTAB_EO)
        r1 = O.true_rel_residual(c.op, x, eta)
        st, info = qxd.solve(c.lat, x, b, tol=1e-10, solver=qxd.SOLVER_MP_BICGSTAB_EO, use_x0=1)
        assert st == qxd.OK and O.true_rel_residual(c.op, x, eta) <= 1e-10 < r1
        # b = 0 has the solution 0, whatever the guess
        z = np.zeros_like(b)
        st, info = qxd.solve(c.lat, x, z, tol=1e-10, use_x0=1)
        assert st == qxd.OK and np.abs(x).max() == 0
    finally:
        c.close()


def test_f32_restart_rescues_a_16bit_solve(qxd):
    """One outer round of a 16-bit inner solve leaves about inner_tol; the restart finishes it."""
    c = Case(qxd, torch, (4, 4, 4, 4))
    try:
        eta = synth.gaussian_spinor(c.dims, 2202)
        b = c.dev_tensor(eta)
        kw = dict(solver=qxd.SOLVER_MP_BICGSTAB_EO, inner_prec=qxd.F16N, tol=1e-10, max_outer=1)
        x = torch.empty_like(b)
        st, info = qxd.solve(c.lat, x, b, check=False, restart_f32=0, **kw)
        assert st == qxd.ENOCONV and info["fallback_used"] == 0
        first = info["iters_inner"]
        st, info = qxd.solve(c.lat, x, b, check=False, **kw)  # restart_f32 is on by default
        assert st == qxd.OK and info["fallback_used"] == 2 and info["status"] == qxd.OK, info
        assert info["iters_inner"] > first and info["iters_outer"] >= 2
        assert O.true_rel_residual(c.op, as_c128(x, eta.shape), eta) <= 1e-10
        # an FP32 inner solve is not restarted
        st, info = qxd.solve(c.lat, x, b, check=False, **dict(kw, inner_prec=qxd.F32))
        assert st == qxd.ENOCONV and info["fallback_used"] == 0
    finally:
        c.close()


def test_restart_then_fallback_chain(qxd):
    """A tolerance the restarted solve cannot reach in one round goes on to the FP64 fallback."""
    c = Case(qxd, torch, (4, 4, 4, 4))
    try:
        eta = synth.gaussian_spinor(c.dims, 2203)
        b = c.dev_tensor(eta)
        x = torch.empty_like(b)
        st, info = qxd.solve(c.lat, x, b, check=False, solver=qxd.SOLVER_MP_CG_EO, inner_prec=qxd.BF16N, tol=1e-13,
                             max_outer=1, fallback=qxd.SOLVER_CG_EO)
        assert st == qxd.OK and info["fallback_used"] == 3 and info["status"] == qxd.OK, info
        assert O.true_rel_residual(c.op, as_c128(x, eta.shape), eta) <= 1e-13
        # the fallback also serves a plain mixed-precision solve
        st, info = qxd.solve(c.lat, x, b, check=False, solver=qxd.SOLVER_MP_CG_EO, inner_prec=qxd.F32, tol=1e-10,
                             max_outer=1, fallback=qxd.SOLVER_MP_BICGSTAB_EO)
        assert st == qxd.OK and info["fallback_used"] == 1, info
        assert O.true_rel_residual(c.op, as_c128(x, eta.shape), eta) <= 1e-10
    finally:
        c.close()


class ParamsV3(C.Structure):
    """The version-3 layout: qxd_solve_params up to and including `fallback`."""
    _fields_ = [("version", C.c_int), ("solver", C.c_int), ("tol", C.c_double), ("maxiter", C.c_int),
                ("inner_prec", C.c_int), ("inner_tol", C.c_double), ("reliable_delta", C.c_double),
                ("max_outer", C.c_int), ("on_device", C.c_int), ("check_every", C.c_int),
                ("gcr_restart", C.c_int), ("net", C.c_void_p), ("gcr_reorth", C.c_int), ("fallback", C.c_int)]


def test_version3_params_are_accepted(qxd):
    c = Case(qxd, torch, (4, 4, 2, 2))
    try:
        eta = synth.gaussian_spinor(c.dims, 2204)
        b = c.dev_tensor(eta)
        x = torch.empty_like(b)
        cur = qxd.default_params(solver=qxd.SOLVER_MP_BICGSTAB_EO)
        p3 = ParamsV3()
        C.memmove(C.addressof(p3), C.addressof(cur), C.sizeof(ParamsV3))
        p3.version = 3
        info = qxd.SolveInfo()
        st = qxd.lib.qxd_solve(c.lat, C.c_void_p(x.data_ptr()), C.c_void_p(b.data_ptr()),
                               C.cast(C.pointer(p3), C.POINTER(qxd.SolveParams)), C.byref(info))
        assert st == qxd.OK, qxd.last_error(c.lat)
        assert O.true_rel_residual(c.op, as_c128(x, eta.shape), eta) <= 1e-10
        p3.version = 2
        st = qxd.lib.qxd_solve(c.lat, C.c_void_p(x.data_ptr()), C.c_void_p(b.data_ptr()),
                               C.cast(C.pointer(p3), C.POINTER(qxd.SolveParams)), C.byref(info))
        assert st == qxd.EINVAL and "version" in qxd.last_error(c.lat)
        # multi-RHS and batched solves take no initial guess
        st, _ = qxd.solve_mrhs(c.lat, x.view(1, -1), b.view(1, -1), 1, check=False, solver=qxd.SOLVER_MP_BICGSTAB_EO,
                               use_x0=1)
        assert st == qxd.EINVAL
    finally:
        c.close()


@pytest.mark.parametrize("solver,prec", [(s, p) for s in (2, 1) for p in (2, 1)])
def test_breakdown_exit_fills_the_solve_info(qxd, solver, prec):
    """An inner solver that gives up early still reports what it did.

    With U = 1, A = 0, m0 = 0, no clover term and periodic time, the constant spinor is a zero
    mode of D (the free operator at p = 0 is m0).  For a constant source the Schur source is
    constant too and Dhat maps it to exactly zero, so BiCGStab divides by <r_hat, Dhat p> = 0 at
    every step and CG on the normal equations by <p, Dhat^+ Dhat p> = 0: every inner solve breaks
    down.  The solve must return ENOCONV with the iterations it spent, the true residual of the x
    it returns (judged by the oracle), and a 16-bit solve's FP32 restart must only get the
    iterations left of maxiter.
    """
    c = Case(qxd, torch, (4, 4, 4, 4), anti=False, eps=0.0, m0=0.0, csw=0.0, csw_qed=0.0)
    try:
        eta = np.ones((c.V, 4, 3), dtype=np.complex128)
        b = c.dev_tensor(eta)
        maxiter = 15
        for restart in (0, 1):
            x = torch.empty_like(b)
            st, info = qxd.solve(c.lat, x, b, check=False, solver=solver, inner_prec=prec, tol=1e-10,
                                 maxiter=maxiter, check_every=1, fallback=-1, restart_f32=restart)
            assert st == qxd.ENOCONV and info["status"] == qxd.ENOCONV, info
            assert info["iters_inner"] > 0, info
            assert info["iters_inner"] <= maxiter, info
            xh = as_c128(x, eta.shape)
            assert np.isfinite(xh).all()
            ref = O.true_rel_residual(c.op, xh, eta)
            assert abs(info["true_rel_res"] - ref) <= 1e-12, (info, ref)
            restarted = restart and prec == qxd.F16N
            assert bool(info["fallback_used"] & 2) == bool(restarted), info
            if solver == qxd.SOLVER_MP_BICGSTAB_EO:
                # BiCGStab gives up after 11 breakdowns; the FP32 restart then gets the 4 left
                assert info["iters_inner"] == (maxiter if restarted else 11), info
    finally:
        c.close()
