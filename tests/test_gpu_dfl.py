"""Inexact deflation on the GPU (the "DFL" of DFL_SAP_GCR, Sec. 5.1) against the deflation
oracle: the little Dirac operator entry by entry, the generated subspace, and DFL-SAP-GCR solves
to the paper's 1e-12 judged by the oracle's true residual."""
import numpy as np
import pytest

from oracle import dfl_oracle as F
from oracle import qxd_oracle as O
from oracle import sap_oracle as S
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


def dense_little(A, nbr):
    """The block-sparse little operator as a dense matrix, rows and columns (block, k)."""
    nb, _, ns, _ = A.shape
    D = np.zeros((nb * ns, nb * ns), dtype=np.complex128)
    for b in range(nb):
        for s in range(9):
            bp = nbr[b, s]
            D[b * ns:(b + 1) * ns, bp * ns:(bp + 1) * ns] += A[b, s]
    return D


@pytest.mark.parametrize("L,block,cstar,ns", [
    ((4, 4, 4, 4), (2, 2, 2, 2), False, 3),
    ((6, 4, 4, 8), (3, 2, 2, 4), False, 2),
    ((4, 4, 4, 4), (2, 2, 2, 2), True, 3),   # C*: the device lattice is 4 x 8 x 4 x 4
    ((4, 4, 4, 4), (4, 2, 4, 2), False, 4),  # a grid of one block in two directions
])
def test_little_operator_matches_oracle(qxd, L, block, cstar, ns):
    """A = P^+ D P built on the GPU equals the oracle's Galerkin product entry by entry (1e-10 of
    its largest entry), for the same subspace fields."""
    c = Case(qxd, torch, L, cstar=cstar)
    try:
        vs = np.stack([synth.gaussian_spinor(c.dims, 4000 + k) for k in range(ns)])
        qxd.dfl_setup(c.lat, block, c.dev_tensor(vs))
        A, nbr = qxd.dfl_get_little(c.lat)
        got = dense_little(A, nbr)
        ref = F.Deflation(c.op, S.sap_blocks(c.dims, block, cstar_L1=L[1] if cstar else None), list(vs)).A
        err = np.abs(got - ref).max() / np.abs(ref).max()
        print(f"{L} block {block} cstar={cstar} ns={ns}: little operator max rel err {err:.2e}")
        assert err < 1e-10, err
    finally:
        c.close()


def test_generated_subspace_matches_oracle(qxd):
    """SAP inverse iteration on the GPU (FP32 SAP) against the oracle's FP64 iteration."""
    c = Case(qxd, torch, (4, 4, 4, 4))
    try:
        start = np.stack([synth.gaussian_spinor(c.dims, 4100 + k) for k in range(2)])
        out = np.empty_like(start)
        qxd.dfl_generate(c.lat, (2, 2, 2, 2), np.ascontiguousarray(start), out, n_it=3, ncy=1, nmr=4)
        ref = F.generate_subspace(c.op, S.sap_blocks(c.dims, (2, 2, 2, 2)), list(start), n_it=3, ncy=1, nmr=4)
        for k in range(2):
            err = np.linalg.norm(out[k] - ref[k]) / np.linalg.norm(ref[k])
            assert err < 1e-5, (k, err)
    finally:
        c.close()


@pytest.mark.parametrize("L,cstar,m0", [((8, 4, 4, 4), False, 0.0), ((4, 4, 4, 8), True, -0.1)])
def test_dfl_sap_gcr_solve(qxd, L, cstar, m0):
    """DFL-SAP-GCR (deflation subspace from 8 SAP-improved random fields) to the paper's 1e-12,
    judged by the oracle; the coarse solves run."""
    c = Case(qxd, torch, L, cstar=cstar, m0=m0)
    try:
        sb, db = (2, 2, 2, 2), (2, 2, 2, 2)
        start = c.dev_tensor(np.stack([synth.gaussian_spinor(c.dims, 4200 + k) for k in range(8)]))
        vecs = torch.empty_like(start)
        qxd.dfl_generate(c.lat, sb, start, vecs, n_it=4, ncy=1, nmr=4)
        qxd.dfl_setup(c.lat, db, vecs, coarse_tol=1e-3, coarse_maxiter=64)
        eta = synth.gaussian_spinor(c.dims, 2600)
        b = c.dev_tensor(eta)
        x = torch.empty_like(b)
        st, info = qxd.solve(c.lat, x, b, solver=qxd.SOLVER_MP_DFL_SAP_GCR, tol=1e-12, sap_block=sb, sap_ncy=2,
                             sap_nmr=4, gcr_restart=16, maxiter=2000)
        assert st == qxd.OK, info
        res = O.true_rel_residual(c.op, as_c128(x, eta.shape), eta)
        assert res <= 1e-12, (res, info)
        st2, info2 = qxd.solve(c.lat, x, b, solver=qxd.SOLVER_MP_SAP_GCR, tol=1e-12, sap_block=sb, sap_ncy=2,
                               sap_nmr=4, gcr_restart=16, maxiter=2000)
        stats = qxd.dfl_info(c.lat)
        assert stats["coarse_calls"] >= info["iters_inner"]
        print(f"{L} cstar={cstar}: DFL-SAP-GCR {info['iters_inner']} steps (residual {res:.1e}), SAP-GCR "
              f"{info2['iters_inner']} steps; coarse {stats}")
        # a field change makes the subspace stale
        qxd.build_clover(c.lat, m0, c.csw, c.csw_qed)
        with pytest.raises(qxd.QxdError) as e:
            qxd.solve(c.lat, x, b, solver=qxd.SOLVER_MP_DFL_SAP_GCR, tol=1e-12, sap_block=sb)
        assert e.value.status == qxd.ESTATE
    finally:
        c.close()


def test_dfl_rejects_bad_input(qxd):
    c = Case(qxd, torch, (4, 4, 4, 4))
    try:
        v = c.dev_tensor(np.stack([synth.gaussian_spinor(c.dims, 1)] * 2))  # the same field twice
        with pytest.raises(qxd.QxdError) as e:
            qxd.dfl_setup(c.lat, (2, 2, 2, 2), v)
        assert e.value.status == qxd.EINVAL and "dependent" in qxd.last_error(c.lat)
        w = c.dev_tensor(np.stack([synth.gaussian_spinor(c.dims, 2)]))
        for blk in [(1, 2, 2, 2), (4, 4, 4, 3), (3, 2, 2, 2)]:
            with pytest.raises(qxd.QxdError) as e:
                qxd.dfl_setup(c.lat, blk, w)
            assert e.value.status == qxd.EINVAL, blk
    finally:
        c.close()
    # C* with a single block in z: the z wrap reaches the x-shifted copy, another block
    c = Case(qxd, torch, (4, 4, 2, 4), cstar=True)
    try:
        w = c.dev_tensor(np.stack([synth.gaussian_spinor(c.dims, 2)]))
        with pytest.raises(qxd.QxdError) as e:
            qxd.dfl_setup(c.lat, (2, 2, 2, 2), w)
        assert e.value.status == qxd.EINVAL
    finally:
        c.close()
