"""GPU solves judged by the oracle's FP64 true residual (the method's tolerance 1e-10)."""
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


def run_solve(qxd, c, eta, **kw):
    b = c.dev_tensor(c.to_boundary(eta))
    x = torch.empty_like(b)
    st, info = qxd.solve(c.lat, x, b, check=False, **kw)
    return st, info, c.from_boundary(as_c128(x, eta.shape))


@pytest.mark.parametrize("solver,prec", [(0, 1), (1, 1), (1, 2), (1, 3), (2, 1), (2, 2), (2, 3)])
@pytest.mark.parametrize("L,cstar,order", [((4, 4, 4, 4), False, 0), ((6, 4, 4, 6), False, 1),
                                           ((4, 2, 2, 4), True, 0)])
def test_solve_reaches_tolerance(qxd, L, cstar, order, solver, prec):
    c = Case(qxd, torch, L, cstar=cstar, order=order)
    try:
        eta = synth.gaussian_spinor(c.dims, 2000)
        st, info, psi = run_solve(qxd, c, eta, solver=solver, inner_prec=prec, tol=1e-10)
        assert st == qxd.OK, info
        res = O.true_rel_residual(c.op, psi, eta)
        assert res <= 1e-10, (res, info)
        ref, _ = O.solve_eo_cg(c.op, eta, tol=1e-12)
        err = np.linalg.norm(psi - ref) / np.linalg.norm(ref)
        print(f"{L} cstar={cstar} solver={solver} prec={prec}: {info}, true res {res:.2e}, err {err:.2e}")
        assert err < 1e-7
    finally:
        c.close()


def test_nan_source_reports_no_convergence(qxd):
    c = Case(qxd, torch, (2, 2, 2, 2))
    try:
        eta = synth.gaussian_spinor(c.dims, 3)
        eta[3, 1, 2] = np.nan
        st, info, _ = run_solve(qxd, c, eta, solver=1, inner_prec=1)
        assert st == qxd.ENOCONV
    finally:
        c.close()


def test_maxiter_exceeded_reports_no_convergence(qxd):
    c = Case(qxd, torch, (4, 4, 4, 4))
    try:
        eta = synth.gaussian_spinor(c.dims, 4)
        st, info, psi = run_solve(qxd, c, eta, solver=0, maxiter=3, tol=1e-10)
        assert st == qxd.ENOCONV and info["iters_inner"] <= 3
        assert 0 < O.true_rel_residual(c.op, psi, eta) < 1
    finally:
        c.close()


def test_zero_source_gives_zero(qxd):
    c = Case(qxd, torch, (2, 2, 2, 2))
    try:
        st, info, psi = run_solve(qxd, c, np.zeros((c.V, 4, 3), dtype=complex))
        assert st == qxd.OK and np.abs(psi).max() == 0
    finally:
        c.close()
