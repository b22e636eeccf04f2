"""Helpers for the GPU parity tests: build lattices through the C ABI from seeded inputs."""
import numpy as np

from oracle import qxd_oracle as O
from paper_2502_02490_gb300 import synth

C1 = dict(q=-1 / 3, m0=-0.1, csw=1.9, csw_qed=1.0, eps=0.3, seed=1000)


def rel_max_err(got, ref):
    """max_i |got_i - ref_i| / max_i |ref_i| (element by element)."""
    return float(np.abs(got - ref).max() / np.abs(ref).max())


def as_c128(t, shape):
    return t.detach().cpu().numpy().view(np.complex128).reshape(shape)


class Case:
    """One lattice set up both on the GPU (through the C ABI) and in the oracle."""

    def __init__(self, qxd, torch, L, anti=True, cstar=False, order=0, eps=0.3, seed=1000, q=-1 / 3, m0=-0.1,
                 csw=1.9, csw_qed=1.0, on_device=True, build=True, blocks=None, openqxd_gauge=False):
        self.qxd, self.torch = qxd, torch
        self.L, self.anti, self.cstar, self.order = tuple(L), anti, cstar, order
        self.blocks = tuple(blocks) if blocks is not None else None
        self.q, self.m0, self.csw, self.csw_qed = q, m0, csw, csw_qed
        self.lat_o = O.Lattice(L, antiperiodic=anti, cstar=cstar)
        self.dims = self.lat_o.dims
        self.V = self.lat_o.V
        U, A = synth.gauge_field(L, seed, eps)
        self.U_phys, self.A_phys = U, A
        if cstar:
            self.U, self.A = O.cstar_double_gauge(U, A, L)
        else:
            self.U, self.A = U, A
        self.dev = torch.device("cuda:0")
        self.stream = torch.cuda.current_stream(self.dev)
        self.lat = qxd.create_lattice(L, qxd.BC_ANTIPERIODIC if anti else qxd.BC_PERIODIC, int(cstar), order,
                                      self.stream.cuda_stream)
        if self.blocks is not None:
            qxd.set_ipt_blocks(self.lat, self.blocks)
        Ub, Ab = U, A
        if order == qxd.ORDER_IPT:
            Ub, Ab = O.to_ipt_order(U, L, self.blocks), O.to_ipt_order(A, L, self.blocks)
        if openqxd_gauge:  # the lattice's own field (doubled for C*) as eight links per odd site
            u8, a8 = O.openqxd_gauge(self.U, self.A, self.dims, self.blocks, cstar=cstar)
            qxd.load_gauge_openqxd(self.lat, torch.from_numpy(np.ascontiguousarray(u8).view(np.float64)).to(self.dev),
                                   torch.from_numpy(np.ascontiguousarray(a8)).to(self.dev), q)
        elif on_device:
            qxd.load_gauge(self.lat, torch.from_numpy(np.ascontiguousarray(Ub).view(np.float64)).to(self.dev),
                           torch.from_numpy(np.ascontiguousarray(Ab)).to(self.dev), q)
        else:
            qxd.load_gauge(self.lat, np.ascontiguousarray(Ub), np.ascontiguousarray(Ab), q)
        self._op = None
        if build:
            qxd.build_clover(self.lat, m0, csw, csw_qed)

    @property
    def op(self):
        if self._op is None:
            self._op = O.Operator(self.lat_o, self.U, self.A, self.q, self.m0, self.csw, self.csw_qed)
        return self._op

    def to_boundary(self, arr):
        return O.to_ipt_order(arr, self.dims, self.blocks) if self.order == self.qxd.ORDER_IPT else arr

    def from_boundary(self, arr):
        return O.from_ipt_order(arr, self.dims, self.blocks) if self.order == self.qxd.ORDER_IPT else arr

    def dev_tensor(self, arr):
        return self.torch.from_numpy(np.ascontiguousarray(arr).view(np.float64)).to(self.dev)

    def apply_D(self, psi, prec=0):
        x = self.dev_tensor(self.to_boundary(psi))
        y = self.torch.empty_like(x)
        self.qxd.apply_D(self.lat, y, x, prec)
        return self.from_boundary(as_c128(y, psi.shape))

    def even_half(self, psi):
        """Even sites of a lexicographic field in floor(Lambda/2) order."""
        return psi[self.lat_o.par == 0]

    def apply_Dhat(self, psi_e, prec=0, dagger=0):
        x = self.dev_tensor(psi_e)
        y = self.torch.empty_like(x)
        self.qxd.apply_Dhat_eo(self.lat, y, x, prec, dagger)
        return as_c128(y, psi_e.shape)

    def close(self):
        """Destroy the lattice after checking that no kernel wrote past the end of its buffers."""
        try:
            bad = self.qxd.check_guards(self.lat)
        finally:
            self.qxd.destroy_lattice(self.lat)
        assert bad == 0, f"{bad} guard bytes overwritten behind the lattice's device buffers"
