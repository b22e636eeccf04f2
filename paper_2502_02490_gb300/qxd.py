"""Thin ctypes binding of libqxd (include/qxd.h): argument marshalling only.

Every function keeps the C name without the ``qxd_`` prefix.  Field arguments may be numpy
arrays (host memory, float64 or complex128, C-contiguous) or torch tensors (their data pointer
is passed; CUDA tensors are device pointers on the lattice's stream).  Failures raise
:class:`QxdError` carrying the status and the library's message.  There is no fallback: if
libqxd.so is absent this module fails to import.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqxd.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"libqxd.so not built at {LIB_PATH}; run __graft_entry__.build()")
lib = C.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ECUDA, ESINGULAR, ENOCONV, ESTATE, ETIMEOUT = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ESINGULAR", "ENOCONV", "ESTATE", "ETIMEOUT"]
BC_PERIODIC, BC_ANTIPERIODIC = 0, 1
ORDER_LEXI, ORDER_IPT = 0, 1
F64, F32, F16N, BF16N = 0, 1, 2, 3
(SOLVER_CG_EO, SOLVER_MP_CG_EO, SOLVER_MP_BICGSTAB_EO, SOLVER_MP_FGCR_NET, SOLVER_MP_SAP_GCR, SOLVER_MP_CGNR,
 SOLVER_MP_DFL_SAP_GCR, SOLVER_MP_MG_GCR) = range(8)
MG_VERSION = 1
PARAMS_VERSION = 5
TRAIN_VERSION = 2
PREC = {"f64": F64, "f32": F32, "f16n": F16N, "bf16n": BF16N}


class SolveParams(C.Structure):
    _fields_ = [("version", C.c_int), ("solver", C.c_int), ("tol", C.c_double), ("maxiter", C.c_int),
                ("inner_prec", C.c_int), ("inner_tol", C.c_double), ("reliable_delta", C.c_double),
                ("max_outer", C.c_int), ("on_device", C.c_int), ("check_every", C.c_int),
                ("gcr_restart", C.c_int), ("net", C.c_void_p), ("gcr_reorth", C.c_int), ("fallback", C.c_int),
                ("use_x0", C.c_int), ("restart_f32", C.c_int),
                ("sap_block", C.c_int * 4), ("sap_ncy", C.c_int), ("sap_nmr", C.c_int)]


class TrainParams(C.Structure):
    _fields_ = [("version", C.c_int), ("epochs", C.c_int), ("batch", C.c_int), ("lr", C.c_double),
                ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
                ("nlayers", C.c_int), ("channels", C.c_int * 9), ("nsamp", C.c_int), ("net_seed", C.c_uint64),
                ("sample_seed", C.c_uint64), ("loss_hist", C.c_void_p)]


class MgParams(C.Structure):
    _fields_ = [("version", C.c_int), ("agg", C.c_int * 4), ("ns2", C.c_int), ("nu", C.c_int), ("n1", C.c_int),
                ("n2", C.c_int), ("m", C.c_int), ("ncy_pre", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iters_inner", C.c_int), ("iters_outer", C.c_int), ("reliable_updates", C.c_int),
                ("true_rel_res", C.c_double), ("seconds", C.c_double), ("status", C.c_int),
                ("fallback_used", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp, _i, _d, _i64 = C.c_void_p, C.c_int, C.c_double, C.c_int64
_SIGS = {
    "qxd_create_lattice": [C.POINTER(C.c_int), _i, _i, _i, _vp, C.POINTER(_vp)],
    "qxd_destroy_lattice": [_vp],
    "qxd_load_gauge": [_vp, _vp, _vp, _d, _i],
    "qxd_update_links": [_vp, _i64, _vp, _vp, _vp, _i],
    "qxd_build_clover": [_vp, _d, _d, _d],
    "qxd_get_clover": [_vp, _vp, _i],
    "qxd_apply_D": [_vp, _vp, _vp, _i, _i, _i],
    "qxd_apply_Dhat_eo": [_vp, _vp, _vp, _i, _i, _i],
    "qxd_solve": [_vp, _vp, _vp, C.POINTER(SolveParams), C.POINTER(SolveInfo)],
    "qxd_solve_mrhs": [_vp, _vp, _vp, _i, C.POINTER(SolveParams), _vp],
    "qxd_vec_dot": [_vp, _vp, _vp, _i64, C.POINTER(_d), C.POINTER(_d)],
    "qxd_vec_norm2": [_vp, _vp, _i64, C.POINTER(_d)],
    "qxd_vec_axpy": [_vp, _d, _d, _vp, _vp, _i64],
    "qxd_vec_dot_noalloc": [_vp, _vp, _i64, _vp, _vp],
    "qxd_vec_dot_noalloc_forget": [],
    "qxd_set_profiling": [_vp, _i],
    "qxd_check_guards": [_vp, C.POINTER(_i64)],
    "qxd_sap_apply": [_vp, _vp, _vp, C.POINTER(C.c_int), _i, _i, _i],
    "qxd_solve_batch": [_vp, _i, _vp, _vp, C.POINTER(SolveParams), _vp],
    "qxd_batch_last_config": [C.POINTER(_i), C.POINTER(_i), C.POINTER(_i), C.POINTER(_i)],
    "qxd_batch_set_spin_limit": [C.c_longlong],
    "qxd_batch_tune_cache": [C.c_char_p],
    "qxd_net_create": [_vp, _i, C.POINTER(C.c_int), C.c_uint64, C.POINTER(_vp)],
    "qxd_net_destroy": [_vp],
    "qxd_net_set_weights": [_vp, _vp],
    "qxd_net_get_weights": [_vp, _vp],
    "qxd_net_apply": [_vp, _vp, _vp, _i],
    "qxd_net_apply_adjoint": [_vp, _vp, _vp, _i],
    "qxd_set_ipt_blocks": [_vp, C.POINTER(C.c_int)],
    "qxd_load_gauge_openqxd": [_vp, _vp, _vp, _d, _i],
    "qxd_net_set_precision": [_vp, _i],
    "qxd_net_loss_grad": [_vp, _vp, _vp, _i, _i, C.POINTER(_d), _vp],
    "qxd_net_train": [_vp, _vp, _i, C.POINTER(TrainParams), _vp, _i],
    "qxd_train_precond": [_vp, C.POINTER(TrainParams), C.POINTER(_vp)],
    "qxd_net_save": [_vp, C.c_char_p],
    "qxd_net_load": [_vp, C.c_char_p, C.POINTER(_vp)],
    "qxd_kernel_stats": [_vp, _i, C.POINTER(_i64), C.POINTER(_d), C.POINTER(_d)],
    "qxd_dfl_generate": [_vp, C.POINTER(C.c_int), _i, _i, _i, _i, _vp, _vp, _i],
    "qxd_dfl_setup": [_vp, C.POINTER(C.c_int), _i, _vp, _i, _d, _i],
    "qxd_dfl_get_little": [_vp, _vp, _vp],
    "qxd_dfl_info": [_vp, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i64), C.POINTER(_i64)],
    "qxd_mg_setup": [_vp, C.POINTER(MgParams), _vp, _i],
    "qxd_mg_generate": [_vp, _i, _i, _i, _vp, _vp, _i],
    "qxd_mg_get_coarse": [_vp, _vp, _vp],
    "qxd_mg_info": [_vp, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i64)],
    "qxd_mg_apply_level1": [_vp, _vp, _vp, _i],
    "qxd_mg_precond": [_vp, _vp, _vp, C.POINTER(C.c_int), _i, _i, _i],
}
for _name, _args in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
lib.qxd_default_params.argtypes = [C.POINTER(SolveParams)]
lib.qxd_default_params.restype = None
lib.qxd_last_error.argtypes = [_vp]
lib.qxd_last_error.restype = C.c_char_p
lib.qxd_net_num_weights.argtypes = [_vp]
lib.qxd_net_num_weights.restype = C.c_int64
lib.qxd_launch_count.argtypes = [_vp]
lib.qxd_launch_count.restype = C.c_int64


class QxdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


def last_error(lat=None) -> str:
    return (lib.qxd_last_error(lat) or b"").decode()


def _check(st, lat=None):
    if st != OK:
        raise QxdError(st, last_error(lat))


def _ptr(a):
    """(address, is_device) of a numpy array or torch tensor."""
    if a is None:
        return None, False
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, False
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), bool(a.is_cuda)
    raise TypeError(f"unsupported field type {type(a)}")


def create_lattice(L, tbc=BC_ANTIPERIODIC, cstar=0, order=ORDER_LEXI, stream=None):
    """qxd_create_lattice; returns the opaque handle (an int).  stream: a cudaStream_t address or None."""
    arr = (C.c_int * 4)(*[int(v) for v in L])
    out = _vp()
    _check(lib.qxd_create_lattice(arr, int(tbc), int(cstar), int(order), stream, C.byref(out)))
    return out.value


def destroy_lattice(lat):
    _check(lib.qxd_destroy_lattice(lat))


def load_gauge(lat, su3, a_u1, q):
    p, dev = _ptr(su3)
    pa, _ = _ptr(a_u1)
    _check(lib.qxd_load_gauge(lat, p, pa, float(q), int(dev)), lat)


def update_links(lat, idx, su3, a_u1=None):
    """qxd_update_links: replace the links idx (int64 entries 4 s + mu) with su3 [n][3][3] complex
    (and angles a_u1 [n]); host arrays or CUDA tensors, all of the same kind."""
    pi, dev = _ptr(idx)
    pu, dev2 = _ptr(su3)
    pa, dev3 = _ptr(a_u1)
    if dev != dev2 or (a_u1 is not None and dev3 != dev):
        raise ValueError("idx, su3 and a_u1 must all be host or all be device buffers")
    n = idx.shape[0] if hasattr(idx, "shape") else len(idx)
    _check(lib.qxd_update_links(lat, int(n), pi, pu, pa, int(dev)), lat)


def set_ipt_blocks(lat, B):
    arr = (C.c_int * 4)(*[int(v) for v in B])
    _check(lib.qxd_set_ipt_blocks(lat, arr), lat)


def load_gauge_openqxd(lat, u8, a8, q):
    """qxd_load_gauge_openqxd: u8 [V/2][8][3][3] complex, a8 [V/2][8] (or None), host or device."""
    pu, dev = _ptr(u8)
    pa = _ptr(a8)[0] if a8 is not None else None
    _check(lib.qxd_load_gauge_openqxd(lat, pu, pa, float(q), int(dev)), lat)


def build_clover(lat, m0, csw, csw_qed):
    _check(lib.qxd_build_clover(lat, float(m0), float(csw), float(csw_qed)), lat)


def get_clover(lat, out):
    p, dev = _ptr(out)
    _check(lib.qxd_get_clover(lat, p, int(dev)), lat)


def apply_D(lat, out, inp, prec=F64, nrhs=1):
    po, dev = _ptr(out)
    pi, dev2 = _ptr(inp)
    if dev != dev2:
        raise ValueError("in and out must both be host or both be device buffers")
    _check(lib.qxd_apply_D(lat, po, pi, int(prec), int(nrhs), int(dev)), lat)


def apply_Dhat_eo(lat, out_e, in_e, prec=F64, dagger=0):
    po, dev = _ptr(out_e)
    pi, dev2 = _ptr(in_e)
    if dev != dev2:
        raise ValueError("in and out must both be host or both be device buffers")
    _check(lib.qxd_apply_Dhat_eo(lat, po, pi, int(prec), int(dagger), int(dev)), lat)


def default_params(**kw):
    p = SolveParams()
    lib.qxd_default_params(C.byref(p))
    for k, v in kw.items():
        cur = getattr(p, k)
        setattr(p, k, type(cur)(*v) if isinstance(cur, C.Array) else v)
    return p


def solve(lat, x, b, params=None, check=True, **kw):
    """qxd_solve; returns (status, info dict).  Raises unless check=False or status is OK."""
    p = params if params is not None else default_params(**kw)
    px, dev = _ptr(x)
    pb, dev2 = _ptr(b)
    if dev != dev2:
        raise ValueError("x and b must both be host or both be device buffers")
    p.on_device = int(dev)
    info = SolveInfo()
    st = lib.qxd_solve(lat, px, pb, C.byref(p), C.byref(info))
    if check:
        _check(st, lat)
    return st, info.as_dict()


def solve_mrhs(lat, x, b, nrhs, params=None, check=True, **kw):
    """qxd_solve_mrhs; returns (status, list of nrhs info dicts)."""
    p = params if params is not None else default_params(**kw)
    px, dev = _ptr(x)
    pb, dev2 = _ptr(b)
    if dev != dev2:
        raise ValueError("x and b must both be host or both be device buffers")
    p.on_device = int(dev)
    infos = (SolveInfo * int(nrhs))()
    st = lib.qxd_solve_mrhs(lat, px, pb, int(nrhs), C.byref(p), C.cast(infos, C.c_void_p))
    if check:
        _check(st, lat)
    return st, [i.as_dict() for i in infos]


def vec_dot(lat, a, b, n):
    re, im = C.c_double(), C.c_double()
    _check(lib.qxd_vec_dot(lat, _device_ptr(a, "a"), _device_ptr(b, "b"), int(n), C.byref(re), C.byref(im)), lat)
    return complex(re.value, im.value)


def vec_norm2(lat, a, n):
    out = C.c_double()
    _check(lib.qxd_vec_norm2(lat, _device_ptr(a, "a"), int(n), C.byref(out)), lat)
    return out.value


def vec_axpy(lat, alpha, x, y, n):
    _check(lib.qxd_vec_axpy(lat, float(np.real(alpha)), float(np.imag(alpha)), _device_ptr(x, "x"),
                            _device_ptr(y, "y"), int(n)), lat)


NOALLOC_MAX_N = 16777216


def _device_ptr(t, what):
    """Address of a CUDA tensor (None passes through); anything in host memory is refused."""
    if t is None:
        return None
    p, dev = _ptr(t)
    if not dev:
        raise ValueError(f"{what} must be a CUDA tensor")
    return p


def vec_dot_noalloc(a, b, n, out, stream=None):
    """qxd_vec_dot_noalloc: <a, b> of n complex entries into the 2 doubles of device memory `out`,
    with scratch in a static device array (no allocation).  stream: a cudaStream_t address or None.
    a, b and out must be CUDA tensors; the library also refuses misaligned addresses."""
    _check(lib.qxd_vec_dot_noalloc(_device_ptr(a, "a"), _device_ptr(b, "b"), int(n), _device_ptr(out, "out"),
                                   stream))


def vec_dot_noalloc_forget():
    """qxd_vec_dot_noalloc_forget: drop the cached scratch addresses (after a device reset)."""
    _check(lib.qxd_vec_dot_noalloc_forget())


def set_profiling(lat, on):
    _check(lib.qxd_set_profiling(lat, int(on)), lat)


def kernel_stats(lat, which):
    n, ms, b = C.c_int64(), C.c_double(), C.c_double()
    _check(lib.qxd_kernel_stats(lat, int(which), C.byref(n), C.byref(ms), C.byref(b)), lat)
    return n.value, ms.value, b.value


def launch_count(lat):
    return int(lib.qxd_launch_count(lat))


def check_guards(lat):
    """qxd_check_guards: the number of guard bytes behind the lattice's buffers that changed."""
    bad = C.c_int64()
    _check(lib.qxd_check_guards(lat, C.byref(bad)), lat)
    return int(bad.value)


# ---- learned preconditioner ----
def net_create(lat, channels, seed=0):
    """qxd_net_create with channels = [1, C, ..., 1]; returns the net handle."""
    ch = (C.c_int * len(channels))(*[int(c) for c in channels])
    out = _vp()
    _check(lib.qxd_net_create(lat, len(channels) - 1, ch, int(seed), C.byref(out)), lat)
    return out.value


def net_destroy(net):
    _check(lib.qxd_net_destroy(net))


def net_num_weights(net):
    return int(lib.qxd_net_num_weights(net))


def net_set_weights(net, w):
    w = np.ascontiguousarray(w, dtype=np.complex128)
    _check(lib.qxd_net_set_weights(net, w.ctypes.data))


def net_get_weights(net):
    w = np.empty(net_num_weights(net), dtype=np.complex128)
    _check(lib.qxd_net_get_weights(net, w.ctypes.data))
    return w


NET_F32, NET_BF16_TC = 0, 1


def net_set_precision(net, prec):
    _check(lib.qxd_net_set_precision(net, int(prec)))


def sap_apply(lat, out, inp, block, ncy=2, nmr=4):
    """qxd_sap_apply: out = M_SAP inp (Schwarz alternating procedure, FP32)."""
    po, dev = _ptr(out)
    pi, dev2 = _ptr(inp)
    if dev != dev2:
        raise ValueError("out and inp must both be host or both be device buffers")
    b = (C.c_int * 4)(*[int(v) for v in block])
    _check(lib.qxd_sap_apply(lat, po, pi, b, int(ncy), int(nmr), int(dev)), lat)


# ---- inexact deflation ----
def dfl_generate(lat, sap_block, start, out, n_it, ncy=1, nmr=4):
    """qxd_dfl_generate: ns = len(start) approximate low modes into out (same shape), by n_it
    normalised SAP inverse iterations of each start field."""
    ps, dev = _ptr(start)
    po, dev2 = _ptr(out)
    if dev != dev2:
        raise ValueError("start and out must both be host or both be device buffers")
    b = (C.c_int * 4)(*[int(v) for v in sap_block])
    _check(lib.qxd_dfl_generate(lat, b, int(ncy), int(nmr), int(start.shape[0]), int(n_it), ps, po, int(dev)), lat)


def dfl_setup(lat, block, vectors, coarse_tol=1e-2, coarse_maxiter=64):
    """qxd_dfl_setup with ns = len(vectors) fields [ns][V][4][3] (host array or CUDA tensor)."""
    pv, dev = _ptr(vectors)
    b = (C.c_int * 4)(*[int(v) for v in block])
    _check(lib.qxd_dfl_setup(lat, b, int(vectors.shape[0]), pv, int(dev), float(coarse_tol), int(coarse_maxiter)), lat)


def dfl_info(lat):
    nb, ns, it, calls = C.c_int(), C.c_int(), C.c_int64(), C.c_int64()
    _check(lib.qxd_dfl_info(lat, C.byref(nb), C.byref(ns), C.byref(it), C.byref(calls)), lat)
    return {"nblocks": nb.value, "ns": ns.value, "coarse_iters": it.value, "coarse_calls": calls.value}


def dfl_get_little(lat):
    """(A [nb][9][ns][ns] complex, nbr [nb][9] int) of the current deflation subspace."""
    info = dfl_info(lat)
    nb, ns = info["nblocks"], info["ns"]
    A = np.empty((nb, 9, ns, ns), dtype=np.complex128)
    nbr = np.empty((nb, 9), dtype=np.int32)
    _check(lib.qxd_dfl_get_little(lat, A.ctypes.data, nbr.ctypes.data), lat)
    return A, nbr


def mg_params(agg, ns2, nu=2, n1=4, n2=8, m=8, ncy_pre=0):
    p = MgParams()
    p.version = MG_VERSION
    p.agg = (C.c_int * 4)(*[int(v) for v in agg])
    p.ns2, p.nu, p.n1, p.n2, p.m, p.ncy_pre = int(ns2), int(nu), int(n1), int(n2), int(m), int(ncy_pre)
    return p


def mg_setup(lat, vectors, **kw):
    """qxd_mg_setup with ns2 = len(vectors) level-1 vectors [ns2][n1] complex (host array or CUDA
    tensor of float64 pairs); keyword arguments as mg_params (agg is required)."""
    pv, dev = _ptr(vectors)
    p = mg_params(ns2=int(vectors.shape[0]), **kw)
    _check(lib.qxd_mg_setup(lat, C.byref(p), pv, int(dev)), lat)


def mg_generate(lat, start, out, n_it, k=8):
    """qxd_mg_generate: level-2 vectors by inverse iteration on level 1 (start, out: [ns2][n1])."""
    ps, dev = _ptr(start)
    po, dev2 = _ptr(out)
    if dev != dev2:
        raise ValueError("start and out must both be host or both be device buffers")
    _check(lib.qxd_mg_generate(lat, int(start.shape[0]), int(n_it), int(k), ps, po, int(dev)), lat)


def mg_info(lat):
    nb2, ns2, calls = C.c_int(), C.c_int(), C.c_int64()
    _check(lib.qxd_mg_info(lat, C.byref(nb2), C.byref(ns2), C.byref(calls)), lat)
    return {"nb2": nb2.value, "ns2": ns2.value, "level1_solves": calls.value}


def mg_get_coarse(lat):
    """(A2 [nb2][9][ns2][ns2] complex, nbr2 [nb2][9] int) of the current multigrid."""
    info = mg_info(lat)
    nb, ns = info["nb2"], info["ns2"]
    A = np.empty((nb, 9, ns, ns), dtype=np.complex128)
    nbr = np.empty((nb, 9), dtype=np.int32)
    _check(lib.qxd_mg_get_coarse(lat, A.ctypes.data, nbr.ctypes.data), lat)
    return A, nbr


def mg_apply_level1(lat, out, inp):
    """qxd_mg_apply_level1: out = K1(inp) for one level-1 vector (n1 complex)."""
    po, dev = _ptr(out)
    pi, dev2 = _ptr(inp)
    if dev != dev2:
        raise ValueError("out and in must both be host or both be device buffers")
    _check(lib.qxd_mg_apply_level1(lat, po, pi, int(dev)), lat)


def mg_precond(lat, out, inp, sap_block, ncy=1, nmr=4):
    """qxd_mg_precond: out = M_MG inp for full fields [V][4][3] complex."""
    po, dev = _ptr(out)
    pi, dev2 = _ptr(inp)
    if dev != dev2:
        raise ValueError("out and in must both be host or both be device buffers")
    b = (C.c_int * 4)(*[int(v) for v in sap_block])
    _check(lib.qxd_mg_precond(lat, po, pi, b, int(ncy), int(nmr), int(dev)), lat)


def net_apply(net, out, inp):
    po, dev = _ptr(out)
    pi, _ = _ptr(inp)
    _check(lib.qxd_net_apply(net, po, pi, int(dev)))


def net_apply_adjoint(net, out, inp):
    """qxd_net_apply_adjoint: out = M^+ inp."""
    po, dev = _ptr(out)
    pi, _ = _ptr(inp)
    _check(lib.qxd_net_apply_adjoint(net, po, pi, int(dev)))


def net_loss_grad(net, v, b, nsamp, want_grad=True):
    pv, dev = _ptr(v)
    pb, _ = _ptr(b)
    loss = C.c_double()
    g = np.empty(net_num_weights(net), dtype=np.complex128) if want_grad else None
    _check(lib.qxd_net_loss_grad(net, pv, pb, int(nsamp), int(dev), C.byref(loss),
                                 g.ctypes.data if g is not None else None))
    return loss.value, g


def train_params(**kw):
    p = TrainParams(version=TRAIN_VERSION, epochs=10, batch=4, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def net_train(net, v, nsamp, params=None, **kw):
    p = params if params is not None else train_params(**kw)
    pv, dev = _ptr(v)
    hist = np.zeros(p.epochs)
    _check(lib.qxd_net_train(net, pv, int(nsamp), C.byref(p), hist.ctypes.data, int(dev)))
    return hist


def train_precond(lat, channels, nsamp, sample_seed, net_seed=0, params=None, **kw):
    """qxd_train_precond: a network trained on nsamp device-generated Gaussian samples.
    Returns (net handle, mean loss per epoch)."""
    p = params if params is not None else train_params(**kw)
    if not 2 <= len(channels) <= 9:
        raise ValueError("channels must list 2..9 channel counts (nlayers 1..8)")
    p.nlayers = len(channels) - 1
    for i, c in enumerate(channels):
        p.channels[i] = int(c)
    p.nsamp, p.sample_seed, p.net_seed = int(nsamp), int(sample_seed), int(net_seed)
    hist = np.zeros(p.epochs)
    p.loss_hist = hist.ctypes.data
    out = _vp()
    _check(lib.qxd_train_precond(lat, C.byref(p), C.byref(out)), lat)
    return out.value, hist


def net_save(net, path):
    _check(lib.qxd_net_save(net, str(path).encode()))


def net_load(lat, path):
    out = _vp()
    _check(lib.qxd_net_load(lat, str(path).encode(), C.byref(out)), lat)
    return out.value


# ---- batched persistent solve ----
def solve_batch(lats, xs, bs, params=None, check=True, **kw):
    """qxd_solve_batch over device fields xs[k], bs[k]; returns (status, list of info dicts)."""
    n = len(lats)
    p = params if params is not None else default_params(**kw)
    p.on_device = 1
    L = (C.c_void_p * n)(*lats)
    X = (C.c_void_p * n)(*[_ptr(x)[0] for x in xs])
    B = (C.c_void_p * n)(*[_ptr(b)[0] for b in bs])
    infos = (SolveInfo * n)()
    st = lib.qxd_solve_batch(C.cast(L, C.c_void_p), n, C.cast(X, C.c_void_p), C.cast(B, C.c_void_p), C.byref(p),
                             C.cast(infos, C.c_void_p))
    if check:
        _check(st, lats[0])
    return st, [i.as_dict() for i in infos]


def batch_last_config():
    t, s, m, g = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    _check(lib.qxd_batch_last_config(C.byref(t), C.byref(s), C.byref(m), C.byref(g)))
    return {"threads": t.value, "sites_per_thread": s.value, "blocks_per_sm": m.value, "graph": bool(g.value)}


def batch_set_spin_limit(limit):
    _check(lib.qxd_batch_set_spin_limit(int(limit)))


def batch_tune_cache(path):
    """qxd_batch_tune_cache: the tuning cache file of solve_batch (None = none)."""
    _check(lib.qxd_batch_tune_cache(None if path is None else os.fsencode(path)))
