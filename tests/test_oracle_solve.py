"""The oracle's even-odd CG on the 4^4 workload (eps=0.3, q=-1/3, m0=-0.1, c_sw=1.9, c_sw^QED=1)."""
from oracle import qxd_oracle as O
from paper_2502_02490_gb300 import synth


def test_c1_eo_cg_reaches_1e10():
    L = (4, 4, 4, 4)
    lat = O.Lattice(L, antiperiodic=True)
    U, A = synth.gauge_field(L, 1000, 0.3)
    op = O.Operator(lat, U, A, q=-1 / 3, m0=-0.1, csw=1.9, csw_qed=1.0)
    eta = synth.gaussian_spinor(L, 2000)
    psi, info = O.solve_eo_cg(op, eta, tol=1e-10)
    assert info["true_rel_residual"] <= 1e-10
    assert 5 < info["iterations"] < 2000
