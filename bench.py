"""Benchmark: clover-dslash GB/s vs HBM peak and time to a 1e-10 true residual vs plain FP64 eo-CG.

One step = one pass of the hot path on the 32^3 x 64 workload (eps = 0.4, q = +2/3, m0 = -0.2,
c_sw = 1.9, c_sw^QED = 1.0, antiperiodic time): ingest the device-resident canonical gauge
arrays, build the clover term and its odd-site inverse, and solve D psi = eta with the
mixed-precision even-odd solver (BiCGStab on Dhat with a 16-bit inner dslash with per-site
norms, FP32 reliable updates, FP64 outer defect correction) to a true relative residual of 1e-10.

value = algorithmic bytes of every dslash launch in the timed steps / timed wall time (GB/s),
summed over ranks / max time over ranks.  The roofline object reports the dominant hop kernel
(its algorithmic bytes per launch / its average CUDA-event duration).  N > 1 runs independent
replicas (one lattice per GPU; the path has no exchange step on one lattice per GPU).

--impl reference times the CPU oracle (FP64 numpy) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "clover-dslash GB/s vs HBM peak; time to 1e-10 residual vs plain FP64 eo-CG"
WORKLOADS = {
    # the workload the metric is quoted on (one GPU)
    "c2": dict(L=(64, 32, 32, 32), cstar=0, eps=0.4, q=2 / 3, m0=-0.2, csw=1.9, csw_qed=1.0, gauge_seed=1001,
               source_seed=2001,
               name="32^3x64 mixed-precision clover solve to 1e-10 (eps=0.4, q=+2/3, m0=-0.2, c_sw=1.9, "
                    "c_sw^QED=1.0, antiperiodic t)"),
    # 48^3x96 with C* boundaries, doubled to 96x48x48x96 (extra measurement line, not the default)
    "c5": dict(L=(96, 48, 48, 48), cstar=1, eps=0.35, q=-1 / 3, m0=-0.1, csw=1.9, csw_qed=1.0, gauge_seed=1004,
               source_seed=2004,
               name="48^3x96 C* (doubled 96x48x48x96) mixed-precision clover solve to 1e-10 (eps=0.35, q=-1/3, "
                    "m0=-0.1, c_sw=1.9, c_sw^QED=1.0, antiperiodic t)"),
    # near-critical 16^3x32 for the learned preconditioner (extra line); m0 from --tune-m0
    "c4": dict(L=(32, 16, 16, 16), cstar=0, eps=0.3, q=-1 / 3, m0=None, csw=1.9, csw_qed=1.0, gauge_seed=1003,
               source_seed=2003,
               name="16^3x32 near-critical (FP64 eo-CG ~2000 iterations): learned PTC preconditioner in "
                    "FGCR vs plain FP64 eo-CG (eps=0.3, q=-1/3, c_sw=1.9, c_sw^QED=1.0, antiperiodic t)"),
    # 12 spin-colour point sources on 24^3x48 through the multi-RHS solve (extra line)
    "c3a": dict(L=(48, 24, 24, 24), cstar=0, eps=0.3, q=-1 / 3, m0=-0.1, csw=1.9, csw_qed=1.0, gauge_seed=1002,
                source_seed=2002,
                name="24^3x48 multi-RHS solve of the 12 spin-colour point sources to 1e-10 (FP32 inner, "
                     "eps=0.3, q=-1/3, m0=-0.1, c_sw=1.9, c_sw^QED=1.0, antiperiodic t)"),
    # the paper's solver family (SAP-GCR, DFL-SAP-GCR) on the 32^3x64 field (extra line)
    "sap": dict(L=(64, 32, 32, 32), cstar=0, eps=0.4, q=2 / 3, m0=-0.2, csw=1.9, csw_qed=1.0, gauge_seed=1001,
                source_seed=2001, name="32^3x64 SAP-GCR and DFL-SAP-GCR"),
    # 8 independent lattices of uneven volume in one persistent batched solve (extra line)
    "c3b": dict(L=None, cstar=0, eps=None, q=-1 / 3, m0=-0.1, csw=1.9, csw_qed=1.0, gauge_seed=1010, source_seed=2010,
                lattices=[(16, 8, 8, 8), (20, 10, 10, 10), (16, 12, 12, 12), (24, 12, 12, 12), (28, 14, 14, 14),
                          (16, 16, 16, 16), (24, 16, 16, 16), (32, 16, 16, 16)],
                name="8 lattices 8^3x16 ... 16^3x32 (sum V = 469,056, eps = 0.2 + 0.3 i/7) solved to 1e-10 in one "
                     "persistent cooperative launch per outer round (FP32 inner BiCGStab, FP64 outer, q=-1/3, "
                     "m0=-0.1, c_sw=1.9, c_sw^QED=1.0, antiperiodic t)"),
}
WORKLOAD = dict(WORKLOADS["c2"])
KSTAT = {0: "hop_f64", 1: "hop_f32", 2: "hop_f16n", 3: "hop_bf16n", 4: "hop_f32_mrhs", 5: "batch_f32",
         6: "ptc_layer_bf16_tc", 7: "ptc_layer_f32", 8: "hop_n16_mrhs", 9: "sap_block_mr", 10: "mrhs_blas"}
PREC_NAMES = {"f32": 1, "f16n": 2, "bf16n": 3}
FP64_REPEATS = 3
# Algorithmic bytes of one Dhat application per even site: 2 hops (4 spinors of the precision,
# 2 x 8 links), A_oo^-1 and A_ee (2 clover blocks pairs), one extra read of psi_e.  16-bit with
# per-site FP32 norms: 4 x 52 + 2 x 288 + 2 x 148 + 52 = 1132; FP32: 4 x 96 + 2 x 576 + 2 x 288
# + 96 = 2208; FP64: 4416.
DHAT_BYTES_PER_EVEN_SITE = {"hop_f16n": 1132, "hop_bf16n": 1132, "hop_f32": 2208, "hop_f64": 4416}
SOLVERS = {"cg": 1, "bicgstab": 2}  # qxd_solver: MP_CG_EO, MP_BICGSTAB_EO


def measured_peaks(path=None):
    """(HBM GB/s denominator, "measured" | "fallback"): the machine's measured copy bandwidth, else
    the 6.8 TB/s fallback of an earlier GB300 measurement."""
    try:
        with open(path or os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = json.load(f).get("hbm_gbs")
        if isinstance(v, (int, float)) and v > 0:
            return float(v), "measured"
    except (OSError, ValueError, AttributeError):
        pass
    return 6800.0, "fallback"


HOP_SOURCES = ("dslash.cu", "hop_site.cuh", "hop_common.cuh", "qxd_internal.cuh")


def hop_source_hash():
    """sha256 over the sources that define the hop kernels (the key of the traffic record)."""
    import hashlib

    h = hashlib.sha256()
    for f in HOP_SOURCES:
        with open(os.path.join(ROOT, "paper_2502_02490_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(kernel, lattice, path=None):
    """DRAM bytes per launch from the committed ncu record, or None if the hop sources changed."""
    rec = {}
    try:
        for line in open(path or os.path.join(ROOT, "profiles", "roofline_traffic.txt")):
            if "=" in line and not line.startswith("#"):
                k, v = line.strip().split("=", 1)
                rec[k] = v
    except OSError:
        return None
    if (rec.get("kernel") != kernel or rec.get("source_sha256") != hop_source_hash()
            or rec.get("lattice") != ",".join(str(v) for v in lattice)):
        return None
    return float(rec["bytes_per_launch"])


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                self.rows.append(f)

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def make_inputs(rank):
    from paper_2502_02490_gb300 import synth

    w = WORKLOAD
    U, A = synth.gauge_field(w["L"], w["gauge_seed"], w["eps"])
    dims = (w["L"][0], 2 * w["L"][1], w["L"][2], w["L"][3]) if w["cstar"] else w["L"]
    eta = synth.gaussian_spinor(dims, w["source_seed"] + 100 * rank)
    return U, A, eta


def aggregate_ranks(t_s, e2e_s, nbytes, world, dev):
    """Whole-job figures of a replicas run: the slowest rank's times (max over ranks) and the bytes
    of all ranks (sum); identity on one rank.  dev: the tensors' device (the process group's)."""
    if world <= 1:
        return t_s, e2e_s, nbytes
    import torch

    tt = torch.tensor([t_s, e2e_s], device=dev, dtype=torch.float64)
    torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
    hb = torch.tensor([nbytes], device=dev, dtype=torch.float64)
    torch.distributed.all_reduce(hb)
    return float(tt[0]), float(tt[1]), float(hb[0])


def run_ours(args, rank, world):
    import torch

    from paper_2502_02490_gb300 import qxd

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    w = WORKLOAD
    # rank 0 reuses the inputs the CPU baseline's pool was set up with (the same seeded fields)
    U, A, eta = (_CPU["U"], _CPU["A"], _CPU["eta"]) if (_CPU and rank == 0) else make_inputs(rank)
    V = eta.shape[0]
    su3_h = torch.from_numpy(U.view(np.float64)).pin_memory()
    a_h = torch.from_numpy(A).pin_memory()
    b_h = torch.from_numpy(eta.view(np.float64)).pin_memory()
    x_h = torch.empty_like(b_h).pin_memory()
    su3_d, a_d, b_d = su3_h.to(dev), a_h.to(dev), b_h.to(dev)
    x_d = torch.empty_like(b_d)
    lat = qxd.create_lattice(w["L"], qxd.BC_ANTIPERIODIC, w["cstar"], qxd.ORDER_LEXI, stream.cuda_stream)
    prec = PREC_NAMES[args.inner]
    params = qxd.default_params(solver=SOLVERS[args.solver], inner_prec=prec, tol=1e-10, inner_tol=args.inner_tol,
                                reliable_delta=args.delta, check_every=args.check_every)

    def step(host=False):
        if host:
            qxd.load_gauge(lat, su3_h.numpy(), a_h.numpy(), w["q"])
        else:
            qxd.load_gauge(lat, su3_d, a_d, w["q"])
        qxd.build_clover(lat, w["m0"], w["csw"], w["csw_qed"])
        if host:
            st, info = qxd.solve(lat, x_h.numpy(), b_h.numpy(), params=params)
        else:
            st, info = qxd.solve(lat, x_d, b_d, params=params)
        return info

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        info = step()
    # ---- timed region (device-resident inputs; library profiling off: the production path) ----
    n0 = qxd.launch_count(lat)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    with Clocks(dev.index) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            infos.append(step())
        e1.record(stream)
        barrier()
    ms_total = e0.elapsed_time(e1)
    launches = qxd.launch_count(lat) - n0
    # ---- per-kernel figures in a separate pass: CUDA events around every hop launch ----
    prof_steps = min(args.steps, 3)
    qxd.set_profiling(lat, 1)
    prof_infos = [step() for _ in range(prof_steps)]
    stats = {KSTAT[k]: qxd.kernel_stats(lat, k) for k in KSTAT}
    qxd.set_profiling(lat, 0)
    # the solve is deterministic (fixed-order reductions), so every step repeats the same launches
    same_work = all(i["iters_inner"] == infos[0]["iters_inner"] for i in infos + prof_infos)
    hop_bytes = sum(b for (_, _, b) in stats.values()) / prof_steps * args.steps
    # ---- end-to-end through host buffers (one untimed host step first: the library allocates
    # its staging buffers for host arguments on first use) ----
    step(host=True)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(host=True)
    barrier()
    e2e_s = time.perf_counter() - t0
    # ---- plain FP64 eo-CG on the same field and source (the comparison baseline): one warm-up
    # solve, then the median of FP64_REPEATS solves, as for the mixed-precision arm ----
    fp64 = None
    if not args.skip_fp64:
        p64 = qxd.default_params(solver=qxd.SOLVER_CG_EO, tol=1e-10, check_every=args.check_every)
        qxd.load_gauge(lat, su3_d, a_d, w["q"])
        qxd.build_clover(lat, w["m0"], w["csw"], w["csw_qed"])
        runs = []
        for k in range(1 + FP64_REPEATS):
            barrier()
            t0 = time.perf_counter()
            st, info64 = qxd.solve(lat, x_d, b_d, params=p64)
            barrier()
            if k:
                runs.append((info64["seconds"], time.perf_counter() - t0, info64))
        med = sorted(runs, key=lambda r: r[0])[len(runs) // 2]
        fp64 = {"seconds": med[0], "wall_s": med[1], "iterations": med[2]["iters_inner"],
                "true_rel_res": med[2]["true_rel_res"], "runs_s": [r[0] for r in runs],
                "timing": f"median of {FP64_REPEATS} solves after one warm-up solve"}
    # ---- resident-field link update: k links replaced on the device (clover rebuilt around them)
    # against reloading the whole field and rebuilding the clover term ----
    link_update = None
    if world == 1:
        from paper_2502_02490_gb300 import synth

        qxd.load_gauge(lat, su3_d, a_d, w["q"])
        qxd.build_clover(lat, w["m0"], w["csw"], w["csw_qed"])
        upd = {}
        Vp = synth.volume(w["L"])  # links are indexed on the physical lattice (C*: not the doubled one)
        for k in (1, 1000, 100000):
            idx = torch.from_numpy(np.random.default_rng(k).choice(4 * Vp, size=k, replace=False)
                                   .astype(np.int64)).to(dev)
            newu = torch.from_numpy(synth.random_su3(k, 17, eps=w["eps"]).view(np.float64)).to(dev)
            newa = torch.from_numpy(synth.random_angles(k, 18, scale=w["eps"])).to(dev)
            qxd.update_links(lat, idx, newu, newa)  # warm-up (scratch allocation)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(3):
                qxd.update_links(lat, idx, newu, newa)
            torch.cuda.synchronize()
            upd[str(k)] = (time.perf_counter() - t0) / 3
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            qxd.load_gauge(lat, su3_d, a_d, w["q"])
            qxd.build_clover(lat, w["m0"], w["csw"], w["csw_qed"])
        torch.cuda.synchronize()
        link_update = {"update_links_s": upd, "full_load_gauge_build_clover_s": (time.perf_counter() - t0) / 3,
                       "note": "k random links replaced on the device (qxd_update_links, clover rebuilt at the "
                               "sites around them); mean of 3 calls after one warm-up"}
    qxd.destroy_lattice(lat)

    # ---- aggregate over ranks ----
    t_s, e2e_s, hop_total = aggregate_ranks(ms_total / 1e3, e2e_s, hop_bytes, world, dev)
    dom = max(stats, key=lambda k: stats[k][1])
    n_l, ms_l, b_l = stats[dom]
    peak, peak_kind = measured_peaks()
    sites = arm_config(args, world)["sites"]
    # one Dhat application = two hop launches (A_oo^-1 H and the A_ee - 1/4 H epilogue); its
    # algorithmic bytes per even site are the minimum the method moves in this precision
    dhat_bytes = DHAT_BYTES_PER_EVEN_SITE.get(dom)
    if dhat_bytes and n_l:
        achieved = dhat_bytes * (sites // 2) / (2 * ms_l / n_l / 1e3) / 1e9
    else:
        achieved = (b_l / n_l) / (ms_l / n_l / 1e3) / 1e9 if n_l else 0.0
    tts = t_s / args.steps
    iters = [i["iters_inner"] for i in infos]
    out = {
        "metric": METRIC,
        "value": hop_total / t_s / 1e9,
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": tts * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"f16n": "f16+f32norm", "bf16n": "bf16+f32norm", "f32": "f32"}[args.inner] + "/f32/f64",
        "data": "synthetic (seeded SplitMix64 gauge field U=exp(i eps H) exp(i q eps theta), Gaussian source)",
        "config": arm_config(args, world),
        "time_to_solution_s": statistics.mean(i["seconds"] for i in infos),
        "time_to_solution_note": "qxd_solve entry to return, fields resident (ms_per_step adds ingest + clover)",
        "solve": {"iters_inner_per_step": statistics.mean(iters), "iters_outer": infos[-1]["iters_outer"],
                  "reliable_updates": infos[-1]["reliable_updates"],
                  "true_rel_res": max(i["true_rel_res"] for i in infos)},
        "fp64_eocg": fp64,
        "speedup_vs_fp64_eocg": (fp64["seconds"] / statistics.mean(i["seconds"] for i in infos)) if fp64 else None,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": f"{peak_kind} hbm_gbs",
                     "traffic": recorded_traffic(dom, w["L"]),
                     "bytes_convention": (f"{dhat_bytes} B per even site per Dhat application (two launches)"
                                          if dhat_bytes else "the kernel's own algorithmic bytes per launch"),
                     "kernel_bytes_per_launch": b_l / n_l if n_l else None,
                     "launches": n_l, "avg_launch_us": ms_l / n_l * 1e3 if n_l else None,
                     "timing": f"CUDA events around every launch of {prof_steps} profiled steps after the "
                               "timed steps"},
        "profiled_steps_same_work": same_work,
        "kernels": {k: {"launches": v[0], "ms": v[1], "GB": v[2] / 1e9} for k, v in stats.items() if v[0]},
        "dslash_kernel_GBps": (sum(v[2] for v in stats.values()) / sum(v[1] for v in stats.values()) / 1e6
                               if world == 1 else None),
        "dslash_kernel_GFLOPs": dslash_gflops(dom, n_l, ms_l, arm_config(args, world)["sites"] // 2),
        "e2e": {"value": hop_total / e2e_s / 1e9 * (1 if world == 1 else 1), "unit": "GB/s",
                "seconds_per_step": e2e_s / args.steps,
                "h2d_bytes_per_step": int(U.nbytes + A.nbytes + eta.nbytes),
                "d2h_bytes_per_step": int(eta.nbytes)},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "link_update": link_update,
    }
    return out


def run_mrhs(args):
    """12 point sources solved together (multi-RHS kernels, 16-bit and FP32 inner) vs one after
    another with the single-RHS solver."""
    import torch

    from paper_2502_02490_gb300 import qxd, synth

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    w = WORKLOAD
    U, A = synth.gauge_field(w["L"], w["gauge_seed"], w["eps"])
    eta = np.stack([synth.point_source(w["L"], k // 3, k % 3) for k in range(12)])
    b = torch.from_numpy(eta.view(np.float64)).to(dev)
    x = torch.empty_like(b)
    lat = qxd.create_lattice(w["L"], qxd.BC_ANTIPERIODIC, 0, qxd.ORDER_LEXI, stream.cuda_stream)
    qxd.load_gauge(lat, torch.from_numpy(U.view(np.float64)).to(dev), torch.from_numpy(A).to(dev), w["q"])
    qxd.build_clover(lat, w["m0"], w["csw"], w["csw_qed"])
    V = int(np.prod(w["L"]))

    def params(prec):
        return qxd.default_params(solver=qxd.SOLVER_MP_BICGSTAB_EO, inner_prec=prec, tol=1e-10,
                                  reliable_delta=args.delta, check_every=args.check_every)

    def timed_mrhs(prec, steps, profile):
        p = params(prec)
        for _ in range(args.warmup):
            qxd.solve_mrhs(lat, x, b, 12, params=p)
        if profile:
            qxd.set_profiling(lat, 1)
        n0 = qxd.launch_count(lat)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            st, infos = qxd.solve_mrhs(lat, x, b, 12, params=p)
        e1.record(stream)
        torch.cuda.synchronize()
        stats = {KSTAT[k]: qxd.kernel_stats(lat, k) for k in KSTAT} if profile else None
        if profile:
            qxd.set_profiling(lat, 0)
        return e0.elapsed_time(e1) / 1e3 / steps, infos, stats, qxd.launch_count(lat) - n0

    prec = PREC_NAMES[args.inner]
    with Clocks(0) as clk:
        t, infos, _, launches = timed_mrhs(prec, args.steps, False)
    # per-kernel figures from a separate profiled pass
    _, _, stats, _ = timed_mrhs(prec, min(args.steps, 3), True)
    t32, infos32, _, _ = timed_mrhs(qxd.F32, args.steps, False) if prec != qxd.F32 else (t, infos, None, 0)
    # the same 12 sources one after another (single-RHS MP BiCGStab, FP32 and 16-bit inner)
    seq = {}
    for name, sp in (("f32", qxd.F32), ("f16n", qxd.F16N)):
        ps = params(sp)
        qxd.solve(lat, x[0], b[0], params=ps)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(12):
            qxd.solve(lat, x[k], b[k], params=ps)
        torch.cuda.synchronize()
        seq[name] = time.perf_counter() - t0
    # the FP32 multi-RHS hop on a full group of 12 right-hand sides (apply_D, both parities with the
    # clover epilogue): 12 site-RHS per site and launch on the amortised 264 B convention
    xin = torch.from_numpy(np.stack([synth.gaussian_spinor(w["L"], 2100 + k) for k in range(12)])
                           .view(np.float64)).to(dev)
    xout = torch.empty_like(xin)
    qxd.apply_D(lat, xout, xin, qxd.F32, nrhs=12)
    qxd.set_profiling(lat, 1)
    for _ in range(5):
        qxd.apply_D(lat, xout, xin, qxd.F32, nrhs=12)
    n12, ms12, by12 = qxd.kernel_stats(lat, 4)
    qxd.set_profiling(lat, 0)
    qxd.destroy_lattice(lat)
    kname = "hop_f32_mrhs" if prec == qxd.F32 else "hop_n16_mrhs"
    n_l, ms_l, b_l = stats[kname]
    peak, kind = measured_peaks()
    achieved = b_l / (ms_l / 1e3) / 1e9
    # the amortised multi-RHS convention per site and RHS and launch: in + out spinor plus
    # (8 links + clover) / 12; FP32: 192 + (576 + 288) / 12 = 264 B, 16-bit: 104 + (288 + 148) / 12
    conv = 264.0 if prec == qxd.F32 else 104.0 + 436.0 / 12
    # site-RHS pairs the launches processed: the FP32 hop works on the active right-hand sides only;
    # its INV and DHAT2 launches come in pairs over the same right-hand sides, with (192 nr + 864)
    # and (288 nr + 864) bytes per site, so sum(nr) = (bytes / Vh - 864 launches) / 240
    if prec == qxd.F32:
        site_rhs = (b_l / (V // 2) - 864.0 * n_l) / 240.0 * (V // 2)
    else:
        site_rhs = 12.0 * (V // 2) * n_l
    achieved_conv = conv * site_rhs / (ms_l / 1e3) / 1e9
    hop_bytes = sum(v[2] for k, v in stats.items() if k != "mrhs_blas") / min(args.steps, 3) * args.steps
    return {"metric": METRIC, "value": hop_bytes / (t * args.steps) / 1e9, "unit": "GB/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": f"{args.inner}/f32/f64", "data": "synthetic",
            "config": {"workload": w["name"], "lattice": list(w["L"]), "nrhs": 12, "solver": "mp-bicgstab-mrhs",
                       "inner_prec": args.inner},
            "time_to_solution_s": t, "solve": {"iters_inner": infos[0]["iters_inner"],
                                               "iters_outer": infos[0]["iters_outer"],
                                               "true_rel_res": max(i["true_rel_res"] for i in infos)},
            "mrhs_f32_inner_s": t32, "mrhs_f32_true_rel_res": max(i["true_rel_res"] for i in infos32),
            "sequential_single_rhs_s": seq, "speedup_vs_sequential_f16n": seq["f16n"] / t,
            "speedup_vs_sequential_f32": seq["f32"] / t,
            "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_kind": f"{kind} hbm_gbs", "traffic": None,
                         "launches": n_l, "avg_launch_us": ms_l / n_l * 1e3 if n_l else None,
                         "bytes": "the kernel's own: spinors per site and RHS (in, out, diagonal in) plus links and "
                                  "clover once per site and group of RHS",
                         "achieved_amortised_convention": achieved_conv,
                         "frac_amortised_convention": achieved_conv / peak,
                         "amortised_convention_bytes_per_site_rhs": conv,
                         "site_rhs_per_launch": site_rhs / n_l if n_l else None,
                         "timing": "CUDA events around every launch of a separate profiled pass"},
            "hop_f32_mrhs_12rhs": {"launches": n12, "avg_launch_us": ms12 / n12 * 1e3 if n12 else None,
                                   "achieved_own_bytes_GBps": by12 / (ms12 / 1e3) / 1e9 if ms12 else None,
                                   "frac_own_bytes": by12 / (ms12 / 1e3) / 1e9 / peak if ms12 else None,
                                   "achieved_amortised_convention_GBps":
                                       264.0 * 12 * (V // 2) * n12 / (ms12 / 1e3) / 1e9 if ms12 else None,
                                   "frac_amortised_convention":
                                       264.0 * 12 * (V // 2) * n12 / (ms12 / 1e3) / 1e9 / peak if ms12 else None,
                                   "note": "apply_D in FP32 with nrhs = 12 (clover epilogue, both parities), "
                                           "5 calls, CUDA events around every launch"},
            "kernels": {k: {"launches": v[0], "ms": v[1], "GB": v[2] / 1e9} for k, v in stats.items() if v[0]},
            "gpu_launches": int(launches), "clocks": clk.summary()}


def run_batch(args):
    """8 lattices of uneven volume solved together (one persistent kernel) vs one after another."""
    import torch

    from paper_2502_02490_gb300 import qxd, synth

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    w = WORKLOAD
    lats, xs, bs = [], [], []
    for i, L in enumerate(w["lattices"]):
        eps = 0.2 + 0.3 * i / 7
        U, A = synth.gauge_field(L, w["gauge_seed"] + i, eps)
        lat = qxd.create_lattice(L, qxd.BC_ANTIPERIODIC, 0, qxd.ORDER_LEXI, stream.cuda_stream)
        qxd.load_gauge(lat, torch.from_numpy(U.view(np.float64)).to(dev), torch.from_numpy(A).to(dev), w["q"])
        qxd.build_clover(lat, w["m0"], w["csw"], w["csw_qed"])
        lats.append(lat)
        bs.append(torch.from_numpy(synth.gaussian_spinor(L, w["source_seed"] + i).view(np.float64)).to(dev))
        xs.append(torch.empty_like(bs[-1]))
    p = qxd.default_params(solver=qxd.SOLVER_MP_BICGSTAB_EO, inner_prec=qxd.F32, tol=1e-10)
    for _ in range(args.warmup):  # the first call autotunes the tile shape
        qxd.solve_batch(lats, xs, bs, params=p)
    cfg = qxd.batch_last_config()
    qxd.set_profiling(lats[0], 1)
    n0 = qxd.launch_count(lats[0])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            st, infos = qxd.solve_batch(lats, xs, bs, params=p)
        e1.record(stream)
        torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / args.steps
    launches = qxd.launch_count(lats[0]) - n0
    n_b, ms_b, b_b = qxd.kernel_stats(lats[0], 5)
    qxd.set_profiling(lats[0], 0)
    # the same 8 solves one after another (single-lattice MP BiCGStab, FP32 and 16-bit inner)
    seq = {}
    for name, prec in (("f32", qxd.F32), ("f16n", qxd.F16N)):
        ps = qxd.default_params(solver=qxd.SOLVER_MP_BICGSTAB_EO, inner_prec=prec, tol=1e-10)
        for k in range(len(lats)):
            qxd.solve(lats[k], xs[k], bs[k], params=ps)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for k in range(len(lats)):
                qxd.solve(lats[k], xs[k], bs[k], params=ps)
        torch.cuda.synchronize()
        seq[name] = (time.perf_counter() - t0) / args.steps
    for lat in lats:
        qxd.destroy_lattice(lat)
    peak, kind = measured_peaks()
    achieved = b_b / (ms_b / 1e3) / 1e9 if ms_b else None
    return {"metric": METRIC, "value": b_b / (t * args.steps) / 1e9, "unit": "GB/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
            "config": {"workload": w["name"], "lattices": [list(L) for L in w["lattices"]],
                       "solver": "mp-bicgstab-batch", "tile": cfg,
                       "l2": "inputs larger than L2: unique working set of the inner kernel ~0.47 GB (> 129 MB L2); no flush"},
            "time_to_solution_s": t,
            "solve": {"iters_inner": [i["iters_inner"] for i in infos], "iters_outer": infos[0]["iters_outer"],
                      "true_rel_res": max(i["true_rel_res"] for i in infos)},
            "sequential_single_lattice_s": seq, "speedup_vs_sequential_f32": seq["f32"] / t,
            "speedup_vs_sequential_f16n": seq["f16n"] / t,
            "roofline": {"bound": "hbm", "kernel": "batch_f32", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak if achieved else None, "peak_kind": f"{kind} hbm_gbs",
                         "traffic": None, "launches": n_b, "avg_launch_ms": ms_b / n_b if n_b else None,
                         "bytes_per_site_iteration": 6144},
            "gpu_launches": int(launches), "clocks": clk.summary()}


def run_sap(args):
    """The paper's solver families on the 32^3x64 field: SAP-preconditioned flexible GCR, the
    deflated two-level version (DFL_SAP_GCR) and three-level multigrid GCR to the paper's 1e-12,
    against MP BiCGStab; SAP block kernel time and bytes from a profiled pass."""
    import torch

    from paper_2502_02490_gb300 import qxd, synth

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    w = WORKLOADS["c2"]
    U, A = synth.gauge_field(w["L"], w["gauge_seed"], w["eps"])
    eta = torch.from_numpy(synth.gaussian_spinor(w["L"], w["source_seed"]).view(np.float64)).to(dev)
    x = torch.empty_like(eta)
    lat = qxd.create_lattice(w["L"], qxd.BC_ANTIPERIODIC, 0, qxd.ORDER_LEXI, stream.cuda_stream)
    qxd.load_gauge(lat, torch.from_numpy(U.view(np.float64)).to(dev), torch.from_numpy(A).to(dev), w["q"])
    qxd.build_clover(lat, w["m0"], w["csw"], w["csw_qed"])
    blk, ncy, nmr, ns = (4, 4, 4, 4), 2, 4, 8
    sap = dict(sap_block=blk, sap_ncy=ncy, sap_nmr=nmr, gcr_restart=16, tol=1e-12, maxiter=5000)

    def timed(profile=False, **kw):
        qxd.solve(lat, x, eta, check=False, **dict(kw, maxiter=20))
        if profile:
            qxd.set_profiling(lat, 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info = qxd.solve(lat, x, eta, check=False, **kw)
        torch.cuda.synchronize()
        out = {"status": qxd.STATUS_NAMES[st], "seconds": time.perf_counter() - t0, "iterations": info["iters_inner"],
               "true_rel_res": info["true_rel_res"]}
        if profile:
            n, ms, by = qxd.kernel_stats(lat, 9)
            qxd.set_profiling(lat, 0)
            out["sap_kernel"] = {"launches": n, "ms": ms, "avg_us": ms / n * 1e3 if n else None,
                                 "GBps_convention": by / (ms / 1e3) / 1e9 if ms else None}
        return out

    res = {"sap_gcr": timed(solver=qxd.SOLVER_MP_SAP_GCR, **sap),
           "mp_bicgstab_f16n": timed(solver=qxd.SOLVER_MP_BICGSTAB_EO, inner_prec=qxd.F16N, tol=1e-12)}
    res["sap_gcr_profiled"] = timed(profile=True, solver=qxd.SOLVER_MP_SAP_GCR, **sap)
    start = torch.from_numpy(np.stack([synth.gaussian_spinor(w["L"], 7000 + k) for k in range(ns)])
                             .view(np.float64)).to(dev)
    vecs = torch.empty_like(start)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    qxd.dfl_generate(lat, blk, start, vecs, n_it=4, ncy=1, nmr=nmr)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    qxd.dfl_setup(lat, blk, vecs, coarse_tol=1e-2, coarse_maxiter=64)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    res["dfl_sap_gcr"] = timed(solver=qxd.SOLVER_MP_DFL_SAP_GCR, **sap)
    res["dfl"] = {"ns": ns, "block": list(blk), "generate_s": t_gen, "setup_s": t_setup, **qxd.dfl_info(lat)}
    # three-level multigrid on the same level 1: aggregates of 2^4 deflation blocks, 8 level-2
    # vectors by inverse iteration on level 1, SAP smoothing before and after the coarse correction
    agg, ns2 = (2, 2, 2, 2), 8
    n1 = res["dfl"]["nblocks"] * ns
    s2 = torch.from_numpy(np.stack([synth.gaussian_spinor((n1, 1, 1, 1), 7100 + k).reshape(-1)[:n1]
                                    for k in range(ns2)]).view(np.float64)).to(dev)
    v2 = torch.empty_like(s2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    qxd.mg_generate(lat, s2, v2, n_it=3, k=8)
    torch.cuda.synchronize()
    t_gen2 = time.perf_counter() - t0
    t0 = time.perf_counter()
    mgp = dict(agg=agg, nu=2, n1=4, n2=8, m=8, ncy_pre=1)
    qxd.mg_setup(lat, v2, **mgp)
    torch.cuda.synchronize()
    t_setup2 = time.perf_counter() - t0
    res["mg_gcr"] = timed(solver=qxd.SOLVER_MP_MG_GCR, **dict(sap, sap_ncy=1))
    res["mg"] = {"ns2": ns2, **mgp, "agg": list(agg), "generate_s": t_gen2, "setup_s": t_setup2, **qxd.mg_info(lat)}
    qxd.destroy_lattice(lat)
    peak, kind = measured_peaks()
    k = res["sap_gcr_profiled"]["sap_kernel"]
    return {"metric": METRIC, "workload": w["name"] + "; SAP blocks 4^4, 2 cycles x 4 MR steps, GCR(16), to 1e-12",
            "results": res,
            "sap_kernel_roofline": {"bound": "latency / L2 (block-local MR iterations)",
                                    "achieved_GBps_convention": k["GBps_convention"], "peak": peak,
                                    "frac": (k["GBps_convention"] or 0) / peak,
                                    "bytes": "per site of the colour and sweep: residual, x read and written, 8 links "
                                             "and the clover pair once (1152 B)"},
            "note": "seconds: one solve after a short warm-up; DFL generate/setup timed separately"}


C4_M0_FILE = os.path.join(ROOT, "profiles", "c4_m0.txt")


def c4_setup(dev, stream, m0=None):
    from paper_2502_02490_gb300 import qxd, synth

    w = WORKLOADS["c4"]
    U, A = synth.gauge_field(w["L"], w["gauge_seed"], w["eps"])
    lat = qxd.create_lattice(w["L"], qxd.BC_ANTIPERIODIC, 0, qxd.ORDER_LEXI, stream.cuda_stream)
    import torch

    qxd.load_gauge(lat, torch.from_numpy(U.view(np.float64)).to(dev), torch.from_numpy(A).to(dev), w["q"])
    if m0 is not None:
        qxd.build_clover(lat, m0, w["csw"], w["csw_qed"])
    return lat


def tune_m0():
    """Bisect m0 so that plain FP64 eo-CG needs 2000 +- 200 iterations on the 16^3x32 field."""
    import torch

    from paper_2502_02490_gb300 import qxd, synth

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    w = WORKLOADS["c4"]
    lat = c4_setup(dev, stream)
    b = torch.from_numpy(synth.gaussian_spinor(w["L"], w["source_seed"]).view(np.float64)).to(dev)
    x = torch.empty_like(b)

    def iters(m0):
        qxd.build_clover(lat, m0, w["csw"], w["csw_qed"])
        st, info = qxd.solve(lat, x, b, check=False, solver=qxd.SOLVER_CG_EO, tol=1e-10, maxiter=6000)
        n = info["iters_inner"] if st == qxd.OK else 10 ** 9
        print(f"m0 {m0:+.6f}: eo-CG iterations {n}", file=sys.stderr)
        return n

    # On the synthetic 16^3x32 field the physical branch never needs more than ~214 iterations (the
    # random links keep the low spectrum gapped; maximum near m0 = -0.1), so the ~2000-iteration
    # point is searched on [-3, 0]: iterations grow towards the first doubler crossing (m0 ~ -2.6)
    # and the solve fails beyond it; bisect between a fast and a failing/slow m0.
    lo, hi = -3.0, 0.0
    n = iters(lo)
    if n <= 2000:
        raise RuntimeError("m0 = -3 is not on the slow side")
    m0 = hi
    for _ in range(40):
        m0 = 0.5 * (lo + hi)
        n = iters(m0)
        if abs(n - 2000) <= 200:
            break
        if n > 2000:
            lo = m0
        else:
            hi = m0
    # the physical branch in steps of 0.01 on [-0.3, 0]: its slowest point
    scan = {round(float(v), 2): iters(round(float(v), 2)) for v in np.arange(-0.30, 0.001, 0.01)}
    slow = max(scan, key=scan.get)
    qxd.destroy_lattice(lat)
    with open(C4_M0_FILE, "w") as f:
        f.write(f"# m0 of the 16^3x32 near-critical workload: FP64 eo-CG iterations {n} (bench.py --tune-m0)\n")
        f.write("# physical-branch scan, m0: eo-CG iterations: " +
                ", ".join(f"{k:+.2f}: {v}" for k, v in scan.items()) + "\n")
        f.write(f"m0={m0!r}\n")
        f.write(f"m0_physical={slow!r}\n")
    print(json.dumps({"m0": m0, "eo_cg_iterations": n, "physical_scan": scan, "m0_physical": slow}))


def c4_m0(key="m0"):
    for line in open(C4_M0_FILE):
        if line.startswith(key + "="):
            return float(line.split("=", 1)[1])
    raise RuntimeError(f"no {key} recorded in {C4_M0_FILE}")


def run_c4(args):
    """Learned preconditioner vs plain FP64 eo-CG (and MP BiCGStab, FGCR without a network), at the
    ~2000-iteration point and at the slowest point of the physical branch."""
    import torch

    from paper_2502_02490_gb300 import qxd, synth

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    w = WORKLOADS["c4"]
    V = synth.volume(w["L"])
    eta = torch.from_numpy(synth.gaussian_spinor(w["L"], w["source_seed"]).view(np.float64)).to(dev)
    x = torch.empty_like(eta)
    ntrain, ntest = 64, 16
    vs = np.stack([synth.gaussian_spinor(w["L"], 5000 + k) for k in range(ntrain + ntest)])
    vtr = torch.from_numpy(vs[:ntrain].view(np.float64)).to(dev)
    vte = torch.from_numpy(vs[ntrain:].view(np.float64)).to(dev)
    bte = torch.empty_like(vte)
    results = {}
    for point, key in (("doubler_side_2000_iterations", "m0"), ("physical_branch_slowest", "m0_physical")):
        m0 = c4_m0(key)
        lat = c4_setup(dev, stream, m0)

        def timed_solve(**kw):
            warm = dict(kw, maxiter=min(kw.get("maxiter", 100000), 50))
            qxd.solve(lat, x, eta, check=False, **warm)  # warm-up (short)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, info = qxd.solve(lat, x, eta, check=False, **kw)
            torch.cuda.synchronize()
            return {"status": qxd.STATUS_NAMES[st], "seconds": time.perf_counter() - t0,
                    "iterations": info["iters_inner"], "outer": info["iters_outer"],
                    "true_rel_res": info["true_rel_res"]}

        res = {"m0": m0,
               "fp64_eocg": timed_solve(solver=qxd.SOLVER_CG_EO, tol=1e-10, maxiter=20000),
               "mp_cg_eo_f32": timed_solve(solver=qxd.SOLVER_MP_CG_EO, inner_prec=qxd.F32, tol=1e-10,
                                           maxiter=20000),
               "mp_bicgstab_f16n": timed_solve(solver=qxd.SOLVER_MP_BICGSTAB_EO, inner_prec=qxd.F16N, tol=1e-10,
                                               restart_f32=0),
               "mp_bicgstab_f32": timed_solve(solver=qxd.SOLVER_MP_BICGSTAB_EO, inner_prec=qxd.F32, tol=1e-10),
               "mp_cgnr_no_net": timed_solve(solver=qxd.SOLVER_MP_CGNR, tol=1e-10, net=None, maxiter=20000),
               "fgcr_no_net": timed_solve(solver=qxd.SOLVER_MP_FGCR_NET, inner_prec=qxd.F32, tol=1e-10,
                                          gcr_restart=32, net=None, maxiter=args.fgcr_maxiter)}
        qxd.apply_D(lat, bte, vte, qxd.F32, nrhs=ntest)
        nets = {}
        for chans in ([1, 8, 8, 1], [1, 16, 16, 1]):
            net = qxd.net_create(lat, chans, seed=7)
            l0, _ = qxd.net_loss_grad(net, vte, bte, ntest, want_grad=False)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hist = qxd.net_train(net, vtr, ntrain, epochs=args.epochs, batch=8, lr=2e-3)
            torch.cuda.synchronize()
            ttrain = time.perf_counter() - t0
            l1, _ = qxd.net_loss_grad(net, vte, bte, ntest, want_grad=False)
            nets["x".join(map(str, chans))] = {
                "train_s": ttrain, "loss_first_epoch": hist[0] / V, "loss_last_epoch": hist[-1] / V,
                "heldout_loss_before": l0 / ntest / V, "heldout_loss_after": l1 / ntest / V,
                "heldout_rel_err_after": float(np.sqrt(l1 / ntest / (24.0 * V))),
                "fgcr": timed_solve(solver=qxd.SOLVER_MP_FGCR_NET, inner_prec=qxd.F32, tol=1e-10, gcr_restart=32,
                                    net=net, maxiter=args.fgcr_maxiter),
                "cgnr": timed_solve(solver=qxd.SOLVER_MP_CGNR, tol=1e-10, net=net, maxiter=20000)}
            # the same network with its channel mix in FP32 on the CUDA cores
            qxd.net_set_precision(net, qxd.NET_F32)
            nets["x".join(map(str, chans))]["fgcr_net_f32"] = timed_solve(
                solver=qxd.SOLVER_MP_FGCR_NET, inner_prec=qxd.F32, tol=1e-10, gcr_restart=32, net=net,
                maxiter=args.fgcr_maxiter)
            qxd.net_destroy(net)
        res["nets"] = nets
        ok = [d[k]["seconds"] for d in nets.values() for k in ("fgcr", "cgnr") if d[k]["status"] == "OK"]
        res["learned_vs_fp64_eocg_speedup"] = (res["fp64_eocg"]["seconds"] / min(ok)) if ok else None
        plain = [v["seconds"] for k, v in res.items() if isinstance(v, dict) and v.get("status") == "OK"
                 and k != "fp64_eocg"]
        res["fastest_plain_solver_s"] = min(plain) if plain else None
        results[point] = res
        qxd.destroy_lattice(lat)
    return {"metric": METRIC, "workload": w["name"], "sites": V, "points": results,
            "note": "losses per site; held-out set of 16 (D v, v) pairs not used in training; "
                    "heldout_rel_err = sqrt(loss / ||v||^2); fgcr: network channel mix in BF16 on the tensor "
                    "cores (default), fgcr_net_f32: the same network in FP32 on the CUDA cores; cgnr: CG on the "
                    "normal equations of D M on the full lattice (M the network in BF16, M^+ its adjoint "
                    "network); mp_cgnr_no_net: the same with M = 1; seconds: one solve after a short warm-up"}


def profile_run(args):
    """One untimed pass of the step (for ncu launch lists and kernel captures).  c4: 40 steps of
    the learned FGCR with an untrained [1,8,8,1] network at the physical branch's slowest mass
    (m0 = -0.12); c3b: one batched solve;
    c3a: one multi-RHS solve of the 12 point sources; sap: 8 SAP-GCR steps, then 3 MG-GCR steps
    after the multigrid set-up."""
    import torch

    from paper_2502_02490_gb300 import qxd, synth

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    w = WORKLOAD
    if args.workload == "c4":
        lat = c4_setup(dev, stream, c4_m0("m0_physical"))
        eta = torch.from_numpy(synth.gaussian_spinor(w["L"], w["source_seed"]).view(np.float64)).to(dev)
        x = torch.empty_like(eta)
        net = qxd.net_create(lat, [1, 8, 8, 1], seed=7)
        st, info = qxd.solve(lat, x, eta, check=False, solver=qxd.SOLVER_MP_FGCR_NET, inner_prec=qxd.F32, tol=1e-10,
                             gcr_restart=32, net=net, maxiter=40, max_outer=1)
        torch.cuda.synchronize()
        print(f"profile run: learned FGCR, 40 steps, {info}", file=sys.stderr)
        qxd.net_destroy(net)
        qxd.destroy_lattice(lat)
        return
    if args.workload == "c3a":
        U, A = synth.gauge_field(w["L"], w["gauge_seed"], w["eps"])
        eta = np.stack([synth.point_source(w["L"], k // 3, k % 3) for k in range(12)])
        b = torch.from_numpy(eta.view(np.float64)).to(dev)
        x = torch.empty_like(b)
        lat = qxd.create_lattice(w["L"], qxd.BC_ANTIPERIODIC, 0, qxd.ORDER_LEXI, stream.cuda_stream)
        qxd.load_gauge(lat, torch.from_numpy(U.view(np.float64)).to(dev), torch.from_numpy(A).to(dev), w["q"])
        qxd.build_clover(lat, w["m0"], w["csw"], w["csw_qed"])
        p = qxd.default_params(solver=qxd.SOLVER_MP_BICGSTAB_EO, inner_prec=PREC_NAMES[args.inner], tol=1e-10)
        st, infos = qxd.solve_mrhs(lat, x, b, 12, params=p)
        torch.cuda.synchronize()
        print(f"profile run: multi-RHS solve ({args.inner} inner), {infos[0]}", file=sys.stderr)
        qxd.destroy_lattice(lat)
        return
    if args.workload == "c3b":
        lats, xs, bs = [], [], []
        for i, L in enumerate(w["lattices"]):
            U, A = synth.gauge_field(L, w["gauge_seed"] + i, 0.2 + 0.3 * i / 7)
            lat = qxd.create_lattice(L, qxd.BC_ANTIPERIODIC, 0, qxd.ORDER_LEXI, stream.cuda_stream)
            qxd.load_gauge(lat, torch.from_numpy(U.view(np.float64)).to(dev), torch.from_numpy(A).to(dev), w["q"])
            qxd.build_clover(lat, w["m0"], w["csw"], w["csw_qed"])
            lats.append(lat)
            bs.append(torch.from_numpy(synth.gaussian_spinor(L, w["source_seed"] + i).view(np.float64)).to(dev))
            xs.append(torch.empty_like(bs[-1]))
        p = qxd.default_params(solver=qxd.SOLVER_MP_BICGSTAB_EO, inner_prec=qxd.F32, tol=1e-10)
        st, infos = qxd.solve_batch(lats, xs, bs, params=p)
        torch.cuda.synchronize()
        print(f"profile run: batched solve, {[i['iters_inner'] for i in infos]}, {qxd.batch_last_config()}",
              file=sys.stderr)
        for lat in lats:
            qxd.destroy_lattice(lat)
        return
    if args.workload == "sap":
        # 8 steps of SAP-GCR (4^4 blocks, 2 cycles x 4 MR steps), then the three-level multigrid
        # of the sap workload and 3 steps of MG-GCR
        U, A = synth.gauge_field(w["L"], w["gauge_seed"], w["eps"])
        eta = torch.from_numpy(synth.gaussian_spinor(w["L"], w["source_seed"]).view(np.float64)).to(dev)
        x = torch.empty_like(eta)
        lat = qxd.create_lattice(w["L"], qxd.BC_ANTIPERIODIC, 0, qxd.ORDER_LEXI, stream.cuda_stream)
        qxd.load_gauge(lat, torch.from_numpy(U.view(np.float64)).to(dev), torch.from_numpy(A).to(dev), w["q"])
        qxd.build_clover(lat, w["m0"], w["csw"], w["csw_qed"])
        blk = (4, 4, 4, 4)
        sap = dict(sap_block=blk, sap_nmr=4, gcr_restart=16, tol=1e-12, max_outer=1, check=False)
        st, info = qxd.solve(lat, x, eta, solver=qxd.SOLVER_MP_SAP_GCR, sap_ncy=2, maxiter=8, **sap)
        start = torch.from_numpy(np.stack([synth.gaussian_spinor(w["L"], 7000 + k) for k in range(8)])
                                 .view(np.float64)).to(dev)
        vecs = torch.empty_like(start)
        qxd.dfl_generate(lat, blk, start, vecs, n_it=2, ncy=1, nmr=4)
        qxd.dfl_setup(lat, blk, vecs)
        n1 = qxd.dfl_info(lat)["nblocks"] * 8
        v2 = torch.from_numpy(np.stack([synth.gaussian_spinor((n1, 1, 1, 1), 7100 + k).reshape(-1)[:n1]
                                        for k in range(8)]).view(np.float64)).to(dev)
        qxd.mg_setup(lat, v2, agg=(2, 2, 2, 2), nu=2, n1=4, n2=8, m=8, ncy_pre=1)
        st2, info2 = qxd.solve(lat, x, eta, solver=qxd.SOLVER_MP_MG_GCR, sap_ncy=1, maxiter=3, **sap)
        torch.cuda.synchronize()
        print(f"profile run: SAP-GCR {info}, MG-GCR {info2}", file=sys.stderr)
        qxd.destroy_lattice(lat)
        return
    U, A, eta = make_inputs(0)
    su3_d = torch.from_numpy(U.view(np.float64)).to(dev)
    a_d = torch.from_numpy(A).to(dev)
    b_d = torch.from_numpy(eta.view(np.float64)).to(dev)
    x_d = torch.empty_like(b_d)
    lat = qxd.create_lattice(w["L"], qxd.BC_ANTIPERIODIC, w["cstar"], qxd.ORDER_LEXI, stream.cuda_stream)
    params = qxd.default_params(solver=SOLVERS[args.solver], inner_prec=PREC_NAMES[args.inner], tol=1e-10,
                                inner_tol=args.inner_tol, reliable_delta=args.delta, check_every=args.check_every)
    qxd.load_gauge(lat, su3_d, a_d, w["q"])
    qxd.build_clover(lat, w["m0"], w["csw"], w["csw_qed"])
    st, info = qxd.solve(lat, x_d, b_d, params=params)
    torch.cuda.synchronize()
    print(f"profile run: lattice {w['L']}, {info}, launches {qxd.launch_count(lat)}", file=sys.stderr)
    qxd.destroy_lattice(lat)


def host_cpu(cpuinfo="/proc/cpuinfo"):
    """CPU model and core count of this host, for the CPU baseline's record."""
    import platform

    model, ids = "", {}
    try:
        with open(cpuinfo) as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and not model:
                    model = line.split(":", 1)[1].strip()
                elif key in ("cpu implementer", "cpu part") and key not in ids:  # Arm: no model name
                    ids[key] = line.split(":", 1)[1].strip()
    except OSError:
        pass
    if not model and ids:
        model = f"implementer {ids.get('cpu implementer', '?')} part {ids.get('cpu part', '?')}"
    return f"{platform.machine()} {model or platform.processor() or 'cpu'}, {os.cpu_count()} logical cores"


# The oracle's inputs and lattice, set in the parent before the worker pool forks, so that every
# worker inherits them (copy on write) instead of receiving GB-sized arrays.
_CPU = {}
CPU_SAMPLE_SITES = 65536  # two time slices of 32^3x64 per step, split evenly over the workers


def cpu_pool_start(nproc=None):
    """Fork the pool of oracle workers (one per host core).  Called before the first GPU call of
    the process: a pool forked after CUDA is initialised can hang."""
    import multiprocessing as mp

    from oracle import qxd_oracle as O

    w = WORKLOAD
    U, A, eta = make_inputs(0)
    lat = O.Lattice(w["L"], antiperiodic=True)
    for mu in range(4):
        for step in (+1, -1):
            lat.neighbour(mu, step)  # neighbour tables built once, shared by the workers
    _CPU.update(U=U, A=A, eta=eta, lat=lat)
    n = int(nproc or os.cpu_count() or 1)
    return mp.get_context("fork").Pool(n), n


def _cpu_worker(chunk):
    """One worker's share of a step: the oracle's D at sites [lo, hi); its wall and CPU time."""
    from oracle import qxd_oracle as O

    lo, hi = chunk
    w = WORKLOAD
    t0, c0 = time.perf_counter(), time.process_time()
    O.D_at_sites(_CPU["lat"], _CPU["U"], _CPU["A"], w["q"], w["m0"], w["csw"], w["csw_qed"], _CPU["eta"],
                 np.arange(lo, hi))
    return time.perf_counter() - t0, time.process_time() - c0


def cpu_sample(pool, nworkers):
    """Time the oracle's D (clover + hop, FP64 numpy) on a bounded sample of the workload's sites,
    process-parallel over the host cores: CPU_SAMPLE_SITES consecutive sites of the 32^3 x 64
    lattice, an equal run of them per worker."""
    per = CPU_SAMPLE_SITES // nworkers
    chunks = [(k * per, (k + 1) * per) for k in range(nworkers)]
    n = per * nworkers
    t0 = time.perf_counter()
    res = pool.map(_cpu_worker, chunks, chunksize=1)
    dt = time.perf_counter() - t0
    cpu = sum(r[1] for r in res)
    # cores actually used: the workers' CPU time over the wall time of the sample
    return {"value": n * 2112 / dt / 1e9, "unit": "GB/s", "cores": max(1, round(cpu / dt)), "kind": "oracle",
            "workers": nworkers, "host": host_cpu(),
            "sample": f"oracle D (clover built at the sites + full-spinor hop) on {n} sites of 32^3x64 "
                      f"({nworkers} processes x {per} sites), 2112 B/site FP64 convention, "
                      f"{dt:.1f} s wall, {cpu:.1f} s CPU"}


def cpu_eocg_c1():
    """The oracle's FP64 even-odd CG to 1e-10 on the 4^4 workload (one process): seconds, iterations."""
    from oracle import qxd_oracle as O
    from paper_2502_02490_gb300 import synth

    L = (4, 4, 4, 4)
    U, A = synth.gauge_field(L, 1000, 0.3)
    eta = synth.gaussian_spinor(L, 2000)
    t0 = time.perf_counter()
    op = O.Operator(O.Lattice(L, antiperiodic=True), U, A, -1 / 3, -0.1, 1.9, 1.0)
    psi, info = O.solve_eo_cg(op, eta, tol=1e-10)
    return {"lattice": "4^4 (eps=0.3, q=-1/3, m0=-0.1, c_sw=1.9, c_sw^QED=1.0)", "seconds": time.perf_counter() - t0,
            "iterations": info["iterations"], "true_rel_res": info["true_rel_residual"], "processes": 1}


def cpu_apply_c1(reps=20):
    """The oracle's full D on the 4^4 workload (one process, clover built once): sites/s and GB/s
    on the 2112 B/site FP64 convention.  The oracle's cost per site does not depend on the lattice
    size, so the 32^3x64 sample stands for the larger lattices."""
    from oracle import qxd_oracle as O
    from paper_2502_02490_gb300 import synth

    L = (4, 4, 4, 4)
    U, A = synth.gauge_field(L, 1000, 0.3)
    psi = synth.gaussian_spinor(L, 2000)
    op = O.Operator(O.Lattice(L, antiperiodic=True), U, A, -1 / 3, -0.1, 1.9, 1.0)
    op.D(psi)
    t0 = time.perf_counter()
    for _ in range(reps):
        op.D(psi)
    dt = (time.perf_counter() - t0) / reps
    V = int(np.prod(L))
    return {"lattice": "4^4 (eps=0.3, q=-1/3, m0=-0.1, c_sw=1.9, c_sw^QED=1.0)", "seconds_per_apply": dt,
            "sites_per_s": V / dt, "GBps_2112B_per_site": V * 2112 / dt / 1e9, "processes": 1}


DSLASH_FLOP_PER_SITE = 1824  # clover dslash: 1320 for the Wilson hop + 504 for the clover term


def dslash_gflops(kernel, launches, ms, sites_per_launch):
    """GFLOP/s of a hop kernel at DSLASH_FLOP_PER_SITE per output site and launch."""
    value = DSLASH_FLOP_PER_SITE * sites_per_launch * launches / (ms / 1e3) / 1e9 if launches and ms > 0 else None
    return {"value": value, "unit": "GFLOP/s", "kernel": kernel, "flop_per_site": DSLASH_FLOP_PER_SITE,
            "sites_per_launch": sites_per_launch}


def arm_config(args, world):
    """The `config` of the default workload's JSON line, shared by both arms."""
    w = WORKLOAD
    return {"workload": w["name"], "lattice": list(w["L"]), "cstar": w["cstar"], "sites": int(np.prod(w["L"])) * (2 if w["cstar"] else 1),
            "solver": f"mp-{args.solver}", "inner_prec": args.inner, "inner_tol": args.inner_tol,
            "reliable_delta": args.delta, "l2": "inputs larger than L2 (links+clover > 1 GB)",
            "parallelism": f"replicas{world}", "step": "load_gauge + build_clover + MP solve"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    pool, nw = cpu_pool_start()
    try:
        vals = []
        for _ in range(args.warmup):
            cpu_sample(pool, nw)
        for _ in range(args.steps):
            vals.append(cpu_sample(pool, nw))
    finally:
        pool.close()
        pool.join()
    v = statistics.mean(x["value"] for x in vals)
    cb = dict(vals[-1])
    cb["value"] = v
    cb["eocg_c1"] = cpu_eocg_c1()
    cb["apply_d_c1"] = cpu_apply_c1()
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": arm_config(args, world), "cpu_baseline": cb, "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--inner", default="f16n", choices=["f32", "f16n", "bf16n"])
    ap.add_argument("--solver", default="bicgstab", choices=["cg", "bicgstab"], help="inner solver of the MP solve")
    ap.add_argument("--inner-tol", type=float, default=1e-5)
    ap.add_argument("--delta", type=float, default=0.1)
    ap.add_argument("--check-every", type=int, default=1)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-run", action="store_true",
                    help="profiling aid for ncu: one untimed step, no JSON line (never a bench value)")
    ap.add_argument("--lattice", default=None, help="T,L1,L2,L3 override, for --profile-run captures only")
    ap.add_argument("--tune-m0", action="store_true", help="bisect m0 of the c4 workload and record it")
    ap.add_argument("--epochs", type=int, default=20, help="training epochs of the c4 workload")
    ap.add_argument("--fgcr-maxiter", type=int, default=3000, help="iteration cap of the c4 FGCR solves")
    ap.add_argument("--workload", default="c2", choices=list(WORKLOADS),
                    help="c2: 32^3x64 (the metric's workload, default); c5: 48^3x96 C* doubled; "
                         "c3a: 12 point sources on 24^3x48 (multi-RHS); c3b: 8 uneven lattices in one batched solve; "
                         "c4: learned preconditioner on 16^3x32; sap: SAP-GCR and DFL-SAP-GCR on 32^3x64")
    args = ap.parse_args()
    WORKLOAD.clear()
    WORKLOAD.update(WORKLOADS[args.workload])
    if args.lattice:
        if not args.profile_run:
            ap.error("--lattice is only for --profile-run")
        WORKLOAD["L"] = tuple(int(v) for v in args.lattice.split(","))
    if args.profile_run:
        import __graft_entry__

        __graft_entry__.build()
        profile_run(args)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    # the CPU baseline's worker pool forks now, before this process makes its first GPU call
    pool, nworkers = None, 0
    if world == 1 and rank == 0 and not args.no_cpu_baseline and args.workload == "c2" and not args.tune_m0:
        pool, nworkers = cpu_pool_start()
    if world > 1:
        import torch

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    import __graft_entry__

    __graft_entry__.build()
    if args.tune_m0:
        tune_m0()
        return
    if args.workload == "c3a":
        print(json.dumps(run_mrhs(args)))
        return
    if args.workload == "c4":
        print(json.dumps(run_c4(args)))
        return
    if args.workload == "c3b":
        print(json.dumps(run_batch(args)))
        return
    if args.workload == "sap":
        print(json.dumps(run_sap(args)))
        return
    out = run_ours(args, rank, world)
    if rank == 0:
        if pool is not None:
            try:
                cpu_sample(pool, nworkers)  # warm-up
                out["cpu_baseline"] = cpu_sample(pool, nworkers)
                out["cpu_baseline"]["eocg_c1"] = cpu_eocg_c1()
                out["cpu_baseline"]["apply_d_c1"] = cpu_apply_c1()
            finally:
                pool.close()
                pool.join()
        print(json.dumps(out))
    if world > 1:
        import torch

        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
