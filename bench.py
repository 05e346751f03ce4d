"""Benchmark of the sparse-lattice D3Q19 TRT stream-collide step on one GB300.

Workload (the paper's fixed-bed-reactor stand-in): a 256^3 bed of radius-12
non-overlapping spheres placed by random sequential addition (seed 1,
stopped after 20000 consecutive rejections), periodic in x, bounce-back
walls elsewhere, body force g = 1e-6 in x, TRT with omega+ = 1 and magic
3/16, FP64, fluid nodes in plain lexicographic order.  One timed step is
one even + one odd step of the AA pattern with RIA (two lattice updates of
every fluid node, the paper's AA-R/AA-RP kernel pair, Sect. 4.1-4.2).

Printed: one JSON line with GFLUP/s (value), the roofline of the dominant
kernel, per-variant numbers (OS-NT / OS-NT-R / AA / AA-R, FP64 / FP32 /
FP16 storage), the oracle timed on the host cores (cpu_baseline) and an
end-to-end figure through host buffers.

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import geometry  # noqa: E402

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# FP64-pipe instructions per node of the AA steps with a uniform body force
# along x, counted by ncu over the nodes of one launch, the same for the even
# and odd step: sm__inst_executed_pipe_fp64.sum = 31 per node with
# omega_plus = 1, of which 27 are arithmetic (smsp__sass_thread_inst_executed
# _op_{dadd,dfma,dmul}_pred_on.sum: 1 DADD, 13 DFMA, 13 DMUL) and 4 the int64 ->
# double conversions of two pairs' outputs.  The moments and the pair update
# run on the integer pipe in fixed point; what stays on the FP64 pipe is the
# per-node terms (density, the reciprocal's Newton steps, velocity, K0, T, O)
# and the rest PDF, which takes one FMA more when omega_plus != 1.
COLL_DP_INSTR_GENERAL = 32
COLL_DP_INSTR_UNIT_OMEGA = 31
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of a
# kernel on the 10,896,954-node bed, from an ncu capture of the current kernel
# version, with the profile that holds it; kernels not listed print null.
TRAFFIC_PROFILED = {
    ("aa_odd_ria_f64", 10896954): (1845508352 + 1595564544, "profiles/aa_pair_f64_packed_bed_256.md"),
    ("aa_even_f64", 10896954): (1656480256 + 1594433024, "profiles/aa_pair_f64_packed_bed_256.md"),
}

WORKLOAD = dict(name="packed_bed_256_rsa_r12", X=256, Y=256, Z=256, radius=12.0, seed=1, rejections=20000,
                periodic=(1, 0, 0), g=(1e-6, 0.0, 0.0), omega_plus=1.0, magic=3.0 / 16.0)


def loop_balance(variant: str, p: int, r: float) -> float:
    """Algorithmic bytes per fluid-node update (Sect. 4, "Loop Balance"; Sect. 4.1).

    D_pdf = 2*19*p, D_idx = 72 (18 x 4 B), D_block = 4 B per run.
    """
    dpdf = 2 * 19 * p
    if variant == "osnt":
        return dpdf + 72
    if variant == "osnt_r":
        return dpdf + 76 * r
    if variant == "aa":
        return dpdf + 36            # even step dpdf, odd step dpdf + 72
    if variant == "aa_r":
        return dpdf + 38 * r        # even step dpdf, odd step dpdf + 76 r
    if variant == "aa_even":
        return dpdf
    if variant == "aa_odd":
        return dpdf + 72
    if variant == "aa_odd_r":
        return dpdf + 76 * r
    if variant == "et":
        return dpdf + 28            # six int32 locations + one uint32 link mask, every step
    if variant == "et_r":
        return dpdf + 28 * r        # the same per run (r = ET runs per node), every step
    raise ValueError(variant)


def job_time_and_value(ms_local, pairs, nodes, world, device=None):
    """Whole-job timing of replicas: the slowest rank's time and the updates of all ranks.

    Every rank times the same work (``pairs`` AA even+odd pairs over ``nodes``
    fluid nodes); the job takes as long as the slowest rank (max over ranks),
    and its throughput counts every rank's updates (weak scaling).
    """
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t)
    return ms, world * 2 * nodes * pairs / (ms / 1e3) / 1e9


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def fp64_pipe_peak(lbm, torch, dev, stream, seconds=1.0):
    """Measured FP64-pipe throughput: the library's DFMA-chain kernel timed with
    CUDA events over about ``seconds``, with the SM clock sampled meanwhile."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    threads = sms * 8 * 256
    out = torch.empty(threads, dtype=torch.float64, device=dev)
    iters = 2048
    for _ in range(2):
        lbm.lbm_fp64_peak_kernel(out, iters, stream)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    lbm.lbm_fp64_peak_kernel(out, iters, stream)
    b.record(stream)
    torch.cuda.synchronize(dev)
    reps = max(3, int(seconds / max(a.elapsed_time(b) / 1e3, 1e-6)))
    with Clocks(dev.index if dev.index is not None else 0) as clk:
        a.record(stream)
        for _ in range(reps):
            lbm.lbm_fp64_peak_kernel(out, iters, stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b)
    c = clk.summary()
    g = 8 * threads * iters * reps / (ms / 1e3) / 1e9
    return {"G_dfma_per_s": g, "sm_mhz": c.get("sm_mhz"), "samples": c.get("samples"), "launches": reps,
            "what": "lbm_fp64_peak_kernel: 8 independent DFMA chains per thread, 8 CTAs of 256 threads per SM, "
                    "CUDA events"}


class NvmlEnergy:
    """Board energy from NVML's cumulative counter (read only), through ctypes."""

    def __init__(self, torch, dev):
        import ctypes
        self.ok = False
        try:
            self.lib = ctypes.CDLL("libnvidia-ml.so.1")
            if self.lib.nvmlInit_v2() != 0:
                return
            want = str(torch.cuda.get_device_properties(dev).uuid)
            n = ctypes.c_uint(0)
            self.lib.nvmlDeviceGetCount_v2(ctypes.byref(n))
            buf = ctypes.create_string_buffer(96)
            for i in range(n.value):
                h = ctypes.c_void_p()
                if self.lib.nvmlDeviceGetHandleByIndex_v2(i, ctypes.byref(h)) != 0:
                    continue
                if self.lib.nvmlDeviceGetUUID(h, buf, 96) != 0:
                    continue
                if buf.value.decode().replace("GPU-", "") == want.replace("GPU-", ""):
                    self.handle = h
                    self.ok = True
                    break
        except Exception:
            self.ok = False

    def millijoules(self):
        import ctypes
        if not self.ok:
            return None
        v = ctypes.c_ulonglong(0)
        if self.lib.nvmlDeviceGetTotalEnergyConsumption(self.handle, ctypes.byref(v)) != 0:
            return None
        return int(v.value)


def energy_leg(lbm, torch, lat, dev, stream, seconds=5.0):
    """Energy to solution of AA-R pairs (the paper's J per lattice update,
    Sect. 5.5) in FP64, FP32 and FP16S: a region of at least ``seconds`` per
    precision, board energy from NVML's counter before and after, power also
    sampled by nvidia-smi every 100 ms."""
    w = WORKLOAD
    nv = NvmlEnergy(torch, dev)
    out = {}
    for prec in ("f64", "f32", "f16s"):
        params = lbm.Params(omega_plus=w["omega_plus"], magic=w["magic"], g=w["g"], shifted=(prec != "f64"))
        sv = lbm.Solver(lat, prec, params, form="aa", ria=True)
        sv.init_equilibrium(1.0)
        sv.step(8, stream)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sv.step(20, stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        pair_s = a.elapsed_time(b) / 1e3 / 10
        pairs = int(seconds / pair_s) + 1
        with Clocks(dev.index if dev.index is not None else 0, period_ms=100) as clk:
            e0 = nv.millijoules()
            a.record(stream)
            sv.step(2 * pairs, stream)
            b.record(stream)
            torch.cuda.synchronize(dev)
            e1 = nv.millijoules()
        sec = a.elapsed_time(b) / 1e3
        gflup = 2 * lat.N * pairs / 1e9
        c = clk.summary()
        rec = {"seconds": sec, "pairs": pairs, "GFLUPs": gflup / sec, "smi_mean_power_w": c.get("power_w_mean"),
               "smi_samples": c.get("samples"), "sm_mhz": c.get("sm_mhz")}
        if e0 is not None and e1 is not None:
            J = (e1 - e0) / 1e3
            rec.update({"J": J, "J_per_GFLUP": J / gflup, "mean_power_w": J / sec,
                        "source": "NVML total energy counter"})
        elif c.get("power_w_mean"):
            J = c["power_w_mean"] * sec
            rec.update({"J": J, "J_per_GFLUP": J / gflup, "mean_power_w": c["power_w_mean"],
                        "source": "nvidia-smi power.draw at 10 Hz"})
        out[prec] = rec
        del sv
        torch.cuda.empty_cache()
    return out


def precision_leg(lbm, torch, lat, dev, stream, steps=1000):
    """FP32 and FP16S storage against FP64 on the same workload (AA-R, from rest,
    ``steps`` steps): PDF max-norm, velocity max and L2, and mass."""
    w = WORKLOAD
    res = {}
    ref = None
    for prec in ("f64", "f32", "f16s"):
        params = lbm.Params(omega_plus=w["omega_plus"], magic=w["magic"], g=w["g"], shifted=(prec != "f64"))
        sv = lbm.Solver(lat, prec, params, form="aa", ria=True)
        sv.init_equilibrium(1.0)
        sv.step(steps, stream)
        F = sv.canonical(stream)
        rho, u, sums = sv.macroscopic(stream=stream)
        if ref is None:
            ref = (F, u, float(sums[0]))
        else:
            Fr, ur, mr = ref
            res[prec] = {"pdf_max_rel": float((F - Fr).abs().max() / Fr.abs().max()),
                         "u_max_rel": float((u - ur).abs().max() / ur.abs().max()),
                         "u_l2_rel": float((u - ur).norm() / ur.norm()),
                         "mass_rel": abs(float(sums[0]) - mr) / mr}
        del sv, F, rho, u
        torch.cuda.empty_cache()
    res["steps"] = steps
    res["max_u_f64"] = float(ref[1].abs().max())
    res["what"] = ("AA-R from rest at rho = 1 on the same bed; errors relative to the FP64 run's max-norm "
                   "(PDFs, velocity) or L2 norm (velocity); FP32 and FP16S store f - w rho0")
    return res


def adjoint_leg(lbm, torch, solid, dev, T=100, K=10):
    """Cost of the checkpointed discrete adjoint on a z < 64 slab of the bed: the
    forward (T steps with checkpoints) and the backward pass (recomputation plus
    T adjoint steps), FP64 and FP32 storage, and the FP32 gradient's error."""
    w = WORKLOAD
    crop = np.ascontiguousarray(solid[:64])
    lat = lbm.Lattice(crop, periodic=w["periodic"], enum="lex", B=1).upload(device=dev)
    s = torch.as_tensor(geometry.node_field(geometry.smooth_noise(crop.shape[2], crop.shape[1], crop.shape[0], 3.0,
                                                                  2), lat.tables(adj=False, runs=False)["node_xyz"]),
                        device=dev).float()
    out = {"fluid_nodes": lat.N, "T": T, "K": K}
    grads = {}
    for prec in ("f64", "f32"):
        params = lbm.Params(omega_plus=1.0, magic=3 / 16, g=(1e-5, 0.0, 0.0), shifted=True)
        G0 = lat.new_grid(prec, device=dev)
        lbm.lbm_init_equilibrium(lat, prec, params, G0, lbm.LBM_LAYOUT_OSNT, 1.0)
        nb = lbm.lbm_ckpt_workspace_bytes(lat, prec, T, K)
        ws = torch.empty((nb + 7) // 8, dtype=torch.float64, device=dev)
        lbm.lbm_flux_forward(lat, prec, params, G0, s, T, K, ws, ria=True)   # warm-up
        lbm.lbm_flux_backward(lat, prec, params, s, T, K, ws, ria=True)
        torch.cuda.synchronize(dev)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        J = lbm.lbm_flux_forward(lat, prec, params, G0, s, T, K, ws, ria=True)
        e[1].record()
        grad = lbm.lbm_flux_backward(lat, prec, params, s, T, K, ws, ria=True)
        e[2].record()
        torch.cuda.synchronize(dev)
        fwd, bwd = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
        out[prec] = {"J": float(J), "forward_ms": fwd, "backward_ms": bwd, "backward_over_forward": bwd / fwd}
        grads[prec] = grad.clone()
        del ws, G0
        torch.cuda.empty_cache()
    out["f32_grad_max_rel_vs_f64"] = float((grads["f32"] - grads["f64"]).abs().max() / grads["f64"].abs().max())
    out["what"] = ("objective J = mean x-momentum after T steps of OS-NT-R with a Brinkman field (smoothed noise, "
                   "sigma 3, seed 2); backward = recomputation from checkpoints every K steps plus T adjoint steps")
    return out


def make_geometry(box=None):
    w = WORKLOAD
    n = box or w["X"]
    solid, _ = geometry.rsa_spheres(n, n, n, w["radius"], w["seed"], periodic=w["periodic"],
                                    max_consecutive_rejections=w["rejections"])
    return solid


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, period_ms: int = 200):
        self.index = index
        self.period_ms = period_ms
        self.proc = None
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix="lbm_clocks_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9], float(parts[3])))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[3] for r in rows), "power_w_mean": statistics.mean(r[3] for r in rows),
                "samples": len(rows), "reasons": reasons}


def cpu_oracle_sample(solid, steps_pairs=1, zslab=16, form="aa"):
    """Time the FP64 oracle (AA even + odd, or two OS-NT steps, per pair) on a
    z-slab of the same bed; GFLUP/s."""
    import torch
    from oracle import lbm as olbm, tables as otables

    w = WORKLOAD
    crop = np.ascontiguousarray(solid[:zslab])
    T = otables.Tables(crop, periodic=w["periodic"], enum="lex", B=1)
    p = olbm.Params(omega_plus=w["omega_plus"], magic=w["magic"], g=w["g"])
    A = olbm.from_canonical(olbm.uniform_state(T.N, p), 1 if form == "aa" else 0, T.adj, p)
    adj = torch.as_tensor(T.adj.astype(np.int64))
    t0 = time.perf_counter()
    for _ in range(steps_pairs):
        if form == "aa":
            A = olbm.aa_even(A, p)
            A = olbm.aa_odd(A, adj, p)
        else:
            A = olbm.osnt_step(olbm.osnt_step(A, adj, p), adj, p)
    dt = time.perf_counter() - t0
    what = "AA even+odd pair(s)" if form == "aa" else "pair(s) of OS-NT steps"
    return {"value": 2 * T.N * steps_pairs / dt / 1e9, "unit": "GFLUP/s", "cores": torch.get_num_threads(),
            "kind": "oracle", "seconds": dt,
            "sample": f"{steps_pairs} {what} of the FP64 oracle on the z < {zslab} slab of the "
                      f"256^3 bed ({T.N} fluid nodes)"}


# ---------------------------------------------------------------------------------------------
# Suites: the other measured configurations (one JSON line each).  They time the library only;
# GPU-vs-oracle comparisons of the same configurations live in tests/.
# ---------------------------------------------------------------------------------------------

def _time_variant(lbm, torch, lat, prec, params, form, ria, pairs, warm=2, s=None, init=True):
    sv = lbm.Solver(lat, prec, params, form=form, ria=ria, s=s)
    if init:
        sv.init_equilibrium(1.0)
    sv.step(2 * warm)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    sv.step(2 * pairs)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    return sv, 2 * lat.N * pairs / (ms / 1e3) / 1e9


def suite_channel(args, lbm, torch):
    """The paper's channel (Sect. 5.1): 100 x 100 x 500, long axis z, 1-voxel walls, periodic z."""
    solid = geometry.square_channel(100, 100, 500)
    lat = lbm.Lattice(solid, periodic=(0, 0, 1), enum="lex", B=1).upload(
        lbm.LBM_TABLES_ADJ | lbm.LBM_TABLES_RIA | lbm.LBM_TABLES_ET)
    r = lat.R / lat.N
    r_et = (len(lat.et_runs()[0]) - 1) / lat.N
    hbm, kind = peaks()
    out = {"suite": "channel", "fluid_nodes": lat.N, "runs": lat.R, "r": r, "r_times_98": r * 98, "r_et": r_et,
           "paper_table2_channel_B_l": [376, 306, 340, 305], "variants": {}}
    w = WORKLOAD
    for prec, pb in (("f64", 8), ("f64df", 8), ("f32", 4), ("f16s", 2)):
        params = lbm.Params(omega_plus=w["omega_plus"], magic=w["magic"], g=(0.0, 0.0, 1e-6),
                            shifted=prec in ("f32", "f16s"))
        for form, ria in (("osnt", False), ("osnt", True), ("aa", False), ("aa", True), ("et", False), ("et", True)):
            name = f"{form}{'_r' if ria else ''}"
            sv, g = _time_variant(lbm, torch, lat, prec, params, form, ria, args.steps)
            bl = loop_balance(name, pb, r_et if name == "et_r" else r)
            out["variants"][f"{name}_{prec}"] = {"GFLUPs": g, "B_l": bl, "frac_hbm": g * bl / hbm,
                                                  "roof_GFLUPs": hbm / bl}
            del sv
            torch.cuda.empty_cache()
    out["hbm_peak_GBs"] = hbm
    return out


def suite_sweep(args, lbm, torch):
    """Enumeration sweep on the bed (Sect. 5.6): LS with B = 1, 8, 16, 32, 64 and the Hilbert curve."""
    solid = make_geometry(args.box)
    w = WORKLOAD
    hbm, kind = peaks()
    out = {"suite": "sweep", "workload": WORKLOAD["name"] if not args.box else f"packed_bed_{args.box}",
           "enumerations": {}}
    for enum, B in (("lex", 1), ("lex", 8), ("lex", 16), ("lex", 32), ("lex", 64), ("hilbert", 1)):
        lat = lbm.Lattice(solid, periodic=w["periodic"], enum=enum, B=B).upload()
        r = lat.R / lat.N
        runs = np.diff(lat.tables(node_xyz=False, adj=False)["run_start"].astype(np.int64))
        rec = {"runs": lat.R, "r": r, "nodes_in_runs_ge_4": float(runs[runs >= 4].sum() / lat.N),
               "nodes_in_runs_ge_32": float(runs[runs >= 32].sum() / lat.N),
               "run_hist_log2": [int(x) for x in lat.run_hist[:16]]}
        for prec, pb in (("f64df", 8), ("f32", 4)):
            params = lbm.Params(omega_plus=w["omega_plus"], magic=w["magic"], g=w["g"], shifted=(prec == "f32"))
            for form, ria in (("osnt", True), ("aa", False), ("aa", True)):
                name = f"{form}{'_r' if ria else ''}"
                sv, g = _time_variant(lbm, torch, lat, prec, params, form, ria, args.steps)
                bl = loop_balance(name, pb, r)
                rec[f"{name}_{prec}"] = {"GFLUPs": g, "B_l": bl, "frac_hbm": g * bl / hbm}
                del sv
                torch.cuda.empty_cache()
        out["enumerations"][f"{enum}{B if enum == 'lex' else ''}"] = rec
        del lat
        torch.cuda.empty_cache()
    return out


def suite_foam(args, lbm, torch):
    """Precision study on an open-cell foam with pressure faces in x (AA-R, FP64 / FP32 / FP16S)."""
    n = args.box or 512
    seeds = max(3, round(400 * (n / 512) ** 3))
    radius = args.radius or 2.5
    t0 = time.time()
    solid = geometry.voronoi_foam(n, n, n, seeds, radius, 3)
    gen_s = time.time() - t0
    lat = lbm.Lattice(solid, periodic=(0, 0, 0), x_pressure=True, enum="lex", B=1).upload(lbm.LBM_TABLES_RIA)
    w = WORKLOAD
    out = {"suite": "foam", "box": n, "seeds": seeds, "strut_radius": radius, "porosity": geometry.porosity(solid),
           "fluid_nodes": lat.N, "r": lat.R / lat.N, "geometry_s": gen_s, "steps": args.foam_steps, "variants": {}}
    x = torch.as_tensor(lat.tables(adj=False, runs=False)["node_xyz"][:, 0].astype(np.int64), device="cuda")
    inlet, outlet = x < 4, x >= n - 4
    ref = None
    for prec in ("f64", "f64df", "f32", "f16s"):
        params = lbm.Params(omega_plus=w["omega_plus"], magic=w["magic"], rho_in=1.0 + 5e-4, rho_out=1.0 - 5e-4,
                            shifted=prec in ("f32", "f16s"))
        sv = lbm.Solver(lat, prec, params, form="aa", ria=True)
        sv.init_equilibrium(1.0)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        sv.step(args.foam_steps)
        b.record()
        torch.cuda.synchronize()
        g = lat.N * args.foam_steps / (a.elapsed_time(b) / 1e3) / 1e9
        rho, u, _ = sv.macroscopic(sums=False)
        dp = float((rho[inlet].mean() - rho[outlet].mean()) / 3.0)
        rec = {"GFLUPs": g, "dP": dp, "mean_ux": float(u[0].mean())}
        if ref is None:
            ref = (u.clone(), dp)
        else:
            du = (u - ref[0]).abs()
            rec.update({"u_err_max_rel": float(du.max() / ref[0].abs().max()),
                        "u_err_l2_rel": float(du.norm() / ref[0].norm()),
                        "dP_err_rel": abs(dp - ref[1]) / abs(ref[1])})
        out["variants"][prec] = rec
        del sv, rho, u
        torch.cuda.empty_cache()
    return out


def suite_adjoint(args, lbm, torch):
    """Adjoint cost: 128^3 periodic box, Brinkman field, FP32 storage, T steps, checkpoint every K."""
    return adjoint_box(lbm, torch, args.box or 128, args.adj_T, args.adj_K, fd=args.fd)


ADJ_VARIANTS = (("f32", "f32", True), ("f64df", "f64df", True), ("f64", "f64", True), ("f64_full", "f64", False))


def adjoint_box(lbm, torch, n=128, T=2000, K=45, variants=ADJ_VARIANTS, fd=0, fd_h=(1e-4, 2e-4, 4e-4)):
    """The differentiation configuration: an n^3 periodic box with a Brinkman
    field (smoothed noise, sigma 3, seed 2), objective the mean x-flux after T
    steps, checkpoints every K; forward and backward timed per storage, and
    optionally central differences of the FP64 forward at ``fd`` nodes."""
    solid = geometry.empty_box(n, n, n)
    lat = lbm.Lattice(solid, periodic=(1, 1, 1)).upload()
    s = torch.as_tensor(geometry.smooth_noise(n, n, n, 3.0, 2).reshape(-1), device="cuda")
    out = {"suite": "adjoint", "box": n, "fluid_nodes": lat.N, "T": T, "K": K, "variants": {}}
    # deviation (shifted) storage in every precision, plus FP64 with full-f
    # storage, the form that takes the fixed-point pair update in its forward
    for name, prec, shifted in variants:
        params = lbm.Params(omega_plus=1.0, magic=3 / 16, g=(1e-5, 0.0, 0.0), shifted=shifted)
        G0 = lat.new_grid(prec)
        lbm.lbm_init_equilibrium(lat, prec, params, G0, lbm.LBM_LAYOUT_OSNT, 1.0)
        nb = lbm.lbm_ckpt_workspace_bytes(lat, prec, T, K)
        ws = torch.empty((nb + 7) // 8, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        J = lbm.lbm_flux_forward(lat, prec, params, G0, s, T, K, ws, ria=False)
        e[1].record()
        grad = lbm.lbm_flux_backward(lat, prec, params, s, T, K, ws, ria=False)
        e[2].record()
        torch.cuda.synchronize()
        fwd, bwd = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
        out["variants"][name] = {"J": float(J), "forward_ms": fwd, "backward_ms": bwd,
                                 "backward_over_forward": bwd / fwd, "workspace_GB": nb / 1e9,
                                 "grad_norm": float(grad.norm()), "grad": grad.cpu()}
        del ws, G0
        torch.cuda.empty_cache()
    ref = out["variants"]["f64"]["grad"]
    for name in [v[0] for v in variants if v[0] != "f64"]:
        gv = out["variants"][name]["grad"]
        out["variants"][name]["grad_err_max_rel"] = float((gv - ref).abs().max() / ref.abs().max())
    if fd:
        # central differences of the FP64 forward (shifted storage) at args.fd
        # nodes, at h, 2h and 4h.  Truncation error (O(h^2), below 1e-8 here)
        # is far below round-off, so the spread of the quotients between h and
        # 2h estimates the round-off noise of the quotient at h: the noise
        # floor printed beside each comparison at h
        rng = np.random.default_rng(4)
        params = lbm.Params(omega_plus=1.0, magic=3 / 16, g=(1e-5, 0.0, 0.0), shifted=True)
        G0 = lat.new_grid("f64")
        lbm.lbm_init_equilibrium(lat, "f64", params, G0, lbm.LBM_LAYOUT_OSNT, 1.0)
        nb = lbm.lbm_ckpt_workspace_bytes(lat, "f64", T, K)
        ws = torch.empty((nb + 7) // 8, dtype=torch.float64, device="cuda")
        nodes = rng.choice(lat.N, fd, replace=False)
        g = np.array([float(ref[int(nd)]) for nd in nodes])
        gmax = float(ref.abs().max())
        fds = {}
        for h in fd_h:
            vals = []
            for node in nodes:
                Jv = []
                for sign in (1, -1):
                    sp = s.clone()
                    sp[node] = float(s[node]) + sign * h
                    hh = float(sp[node].double() - s[node].double())
                    Jv.append((float(lbm.lbm_flux_forward(lat, "f64", params, G0, sp, T, K, ws)), hh))
                vals.append((Jv[0][0] - Jv[1][0]) / (Jv[0][1] - Jv[1][1]))
            fds[h] = np.array(vals)
        for h, h2 in zip(fd_h[:-1], fd_h[1:]):
            err = np.abs(fds[h] - g) / np.abs(g)
            floor = np.abs(fds[h] - fds[h2]) / np.abs(g)
            out[f"fd_h{h:g}"] = {"max_rel_err": float(err.max()), "median_rel_err": float(np.median(err)),
                                 "noise_floor_max_rel": float(floor.max()),
                                 "noise_floor_median_rel": float(np.median(floor)),
                                 "max_err_over_max_grad": float(np.max(np.abs(fds[h] - g)) / gmax)}
        out["fd_nodes"] = fd
        out["fd_note"] = ("central differences of the FP64 forward (shifted storage) against the FP64 adjoint "
                          "gradient; noise_floor = |FD(h) - FD(2h)| / |dJ/ds_n|, the round-off spread of the "
                          "quotient (truncation is O(h^2), far below it)")
        del ws
    for v in out["variants"].values():
        v.pop("grad", None)
    return out


def suite_large(args, lbm, torch):
    """Large production run: 768^3 Voronoi foam, Hilbert order, pressure faces in x, FP32 AA-R."""
    return production_run(lbm, torch, args.box or 768, args.radius or 3.0, args.large_steps)


def production_run(lbm, torch, n=768, radius=3.0, steps=5000):
    """The production configuration: an n^3 Voronoi-edge foam (1500 seeds at
    768^3, strut radius 3), Hilbert-ordered, pressure faces in x, FP32 AA-R for
    ``steps`` steps; sustained GFLUP/s and the fraction of the B_l roofline."""
    seeds = max(3, round(1500 * (n / 768) ** 3))
    t0 = time.time()
    solid = geometry.voronoi_foam(n, n, n, seeds, radius, 5)
    gen_s = time.time() - t0
    t0 = time.time()
    lat = lbm.Lattice(solid, periodic=(0, 0, 0), x_pressure=True, enum="hilbert")
    build_s = time.time() - t0
    del solid
    lat.upload(lbm.LBM_TABLES_RIA)
    hbm, kind = peaks()
    w = WORKLOAD
    params = lbm.Params(omega_plus=w["omega_plus"], magic=w["magic"], rho_in=1.0 + 5e-4, rho_out=1.0 - 5e-4,
                        shifted=True)
    sv = lbm.Solver(lat, "f32", params, form="aa", ria=True)
    sv.init_equilibrium(1.0)
    sv.step(4)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(torch.cuda.current_device()) as clk:
        a.record()
        sv.step(steps)
        b.record()
        torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3
    g = lat.N * steps / sec / 1e9
    r = lat.R / lat.N
    bl = loop_balance("aa_r", 4, r)
    _, _, sums = sv.macroscopic(fields=False)
    out = {"suite": "large", "box": n, "seeds": seeds, "strut_radius": radius, "fluid_nodes": lat.N, "r": r,
           "enumeration": "hilbert", "geometry_s": gen_s, "lattice_build_s": build_s, "steps": steps,
           "seconds": sec, "GFLUPs": g, "B_l": bl, "GBs_model": g * bl, "frac_hbm": g * bl / hbm,
           "state_GB": 19 * lat.Npad * 4 / 1e9, "mass": float(sums[0]), "clocks": clk.summary()}
    del sv, lat
    torch.cuda.empty_cache()
    return out


def suite_bandwidth(args, lbm, torch):
    """Pattern-specific bandwidths (the paper's Table 3) and the roofline they predict (Table 4)."""
    solid = make_geometry(args.box)
    w = WORKLOAD
    lat = lbm.Lattice(solid, periodic=w["periodic"], enum="lex", B=1).upload()
    r = lat.R / lat.N
    out = {"suite": "bandwidth", "fluid_nodes": lat.N, "r": r, "bandwidth_GBs": {}, "predicted_vs_measured": {}}
    for p_bytes in (8, 4, 2):
        nb = 19 * lat.Npad * p_bytes
        src = torch.empty(nb // 4, dtype=torch.float32, device="cuda").fill_(1.0)
        dst = torch.empty_like(src)
        for name, kind, arrays in (("CNT-1A", 0, 1), ("CNT-19A", 0, 19), ("U-1A", 1, 1), ("U-19A", 1, 19)):
            for _ in range(3):
                lbm.lbm_bandwidth_kernel(kind, dst, src, arrays)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 20
            a.record()
            for _ in range(reps):
                lbm.lbm_bandwidth_kernel(kind, dst, src, arrays)
            b.record()
            torch.cuda.synchronize()
            gbs = 2 * nb * reps / (a.elapsed_time(b) / 1e3) / 1e9
            out["bandwidth_GBs"][f"{name}_{nb / 1e9:.2f}GB"] = gbs
            out["bandwidth_GBs"].setdefault(f"{name}_p{p_bytes}", gbs)
        del src, dst
        torch.cuda.empty_cache()
    for prec, p_bytes in (("f64df", 8), ("f32", 4), ("f16s", 2)):
        params = lbm.Params(omega_plus=w["omega_plus"], magic=w["magic"], g=w["g"], shifted=(prec != "f64df"))
        for form, ria in (("osnt", False), ("osnt", True), ("aa", False), ("aa", True)):
            name = f"{form}{'_r' if ria else ''}"
            sv, g = _time_variant(lbm, torch, lat, prec, params, form, ria, args.steps)
            b = out["bandwidth_GBs"][f"{'CNT-19A' if form == 'osnt' else 'U-19A'}_p{p_bytes}"]
            bl = loop_balance(name, p_bytes, r)
            out["predicted_vs_measured"][f"{name}_{prec}"] = {"B_l": bl, "b_GBs": b, "predicted_GFLUPs": b / bl,
                                                              "measured_GFLUPs": g, "ratio": g / (b / bl)}
            del sv
            torch.cuda.empty_cache()
    return out


def suite_partition(args, lbm, torch):
    """Partitioning and two-stage renumbering (Sect. 6, 6.1): ghost PDFs per chunk and single-GPU speed."""
    solid = make_geometry(args.box)
    w = WORKLOAD
    out = {"suite": "partition", "workload": WORKLOAD["name"] if not args.box else f"packed_bed_{args.box}",
           "orders": {}}
    base = {"lex1": lbm.Lattice(solid, periodic=w["periodic"], enum="lex", B=1),
            "lex16": lbm.Lattice(solid, periodic=w["periodic"], enum="lex", B=16),
            "hilbert": lbm.Lattice(solid, periodic=w["periodic"], enum="hilbert")}
    for P in (16, 64):
        base[f"hilbert_renum{P}"] = lbm.Lattice.from_order(solid, base["hilbert"].renumber_partitions(P),
                                                           periodic=w["periodic"])
    for name, lat in base.items():
        rec = {"runs": lat.R, "r": lat.R / lat.N}
        for P in (16, 64):
            g = lat.partition_ghosts(P)
            rec[f"ghost_pdfs_P{P}"] = {"max": int(g.max()), "mean": float(g.mean()),
                                       "max_MiB_f64": float(g.max()) * 8 / 2 ** 20}
        lat.upload()
        for prec in ("f32", "f64df"):
            params = lbm.Params(omega_plus=w["omega_plus"], magic=w["magic"], g=w["g"], shifted=(prec == "f32"))
            sv, gf = _time_variant(lbm, torch, lat, prec, params, "aa", True, args.steps)
            rec[f"aa_r_{prec}_GFLUPs"] = gf
            del sv
            torch.cuda.empty_cache()
        out["orders"][name] = rec
    return out


def suite_exchange(args, lbm, torch):
    """P chunks with a ghost-PDF exchange every step, all on one GPU (Sect. 6): the partitioned
    AA-R and OS-NT-R steps against the whole-lattice ones, and the exchange kernel alone."""
    solid = make_geometry(args.box)
    w = WORKLOAD
    hbm, kind = peaks()
    out = {"suite": "exchange", "workload": WORKLOAD["name"] if not args.box else f"packed_bed_{args.box}",
           "pairs": args.steps, "cases": {}}
    hil = lbm.Lattice(solid, periodic=w["periodic"], enum="hilbert")
    cases = [("lex1", lbm.Lattice(solid, periodic=w["periodic"], enum="lex", B=1), 16),
             ("hilbert", hil, 16)]
    for P in (16, 64):
        cases.append((f"hilbert_renum{P}", lbm.Lattice.from_order(solid, hil.renumber_partitions(P),
                                                                   periodic=w["periodic"]), P))
    for name, lat, P in cases:
        lat.upload()
        part = lbm.Partitioning(lat, P).upload()
        E = int(sum(part.ghost_pdfs))
        rec = {"P": P, "r": lat.R / lat.N, "r_chunks": sum(q.R for q in part.parts) / lat.N,
               "ghost_pdfs": E, "ghost_share": E / (18 * lat.N)}
        for prec, pb in (("f32", 4), ("f64df", 8)):
            params = lbm.Params(omega_plus=w["omega_plus"], magic=w["magic"], g=w["g"], shifted=(prec == "f32"))
            for form in ("aa", "osnt"):
                sv, whole = _time_variant(lbm, torch, lat, prec, params, form, True, args.steps)
                del sv
                ps = lbm.PartitionedSolver(part, prec, params, form=form, ria=True)
                ps.init_equilibrium(1.0)
                ps.step(4)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                ps.step(2 * args.steps)
                b.record()
                torch.cuda.synchronize()
                ms = a.elapsed_time(b)
                # the exchange alone: the two copies of one pair (gather + scatter, or two OS-NT fills)
                modes = ((lbm.LBM_HALO_AA_GATHER, lbm.LBM_HALO_AA_SCATTER) if form == "aa"
                         else (lbm.LBM_HALO_OSNT, lbm.LBM_HALO_OSNT))
                ptrs = lbm.Partitioning.pointers(ps.grids)
                a.record()
                for _ in range(args.steps):
                    for m in modes:
                        lbm.lbm_halo_exchange(part, prec, ptrs, m)
                b.record()
                torch.cuda.synchronize()
                ex_ms = a.elapsed_time(b) / args.steps
                ex_bytes = 2 * E * (2 * pb + 8)
                rec[f"{form}_r_{prec}"] = {
                    "whole_GFLUPs": whole, "partitioned_GFLUPs": 2 * lat.N * args.steps / (ms / 1e3) / 1e9,
                    "exchange_ms_per_pair": ex_ms, "exchange_GBs": ex_bytes / (ex_ms / 1e3) / 1e9,
                    "exchange_bytes_per_pair": ex_bytes, "pair_ms": ms / args.steps}
                del ps
                torch.cuda.empty_cache()
        out["cases"][name] = rec
        del part
        torch.cuda.empty_cache()
    out["hbm_peak_GBs"] = hbm
    return out


def suite_bed40(args, lbm, torch):
    """The porosity-0.4 bed (about 6.7 M nodes) that random sequential addition cannot reach:
    radius-12 spheres on a jittered, randomly rotated FCC lattice in the same 256^3 box, every
    storage form and precision, with the loop balance of each."""
    solid = geometry.packed_bed_fcc_256(1)
    w = WORKLOAD
    hbm, kind = peaks()
    lat = lbm.Lattice(solid, periodic=w["periodic"], enum="lex", B=1).upload(
        lbm.LBM_TABLES_ADJ | lbm.LBM_TABLES_RIA | lbm.LBM_TABLES_ET)
    N = lat.N
    r = lat.R / N
    r_et = (len(lat.et_runs()[0]) - 1) / N
    out = {"suite": "bed40", "fluid_nodes": N, "porosity": geometry.porosity(solid), "runs": lat.R, "r": r,
           "r_et": r_et, "phantoms": lat.et_info()[0] - N, "pairs": args.steps, "variants": {}}
    for prec, pb in (("f64", 8), ("f64df", 8), ("f32", 4), ("f16s", 2)):
        params = lbm.Params(omega_plus=w["omega_plus"], magic=w["magic"], g=w["g"],
                            shifted=prec in ("f32", "f16s"))
        for form, ria in (("osnt", False), ("osnt", True), ("aa", False), ("aa", True), ("et", False),
                          ("et", True)):
            name = f"{form}{'_r' if ria else ''}"
            sv, g = _time_variant(lbm, torch, lat, prec, params, form, ria, args.steps)
            bl = loop_balance(name, pb, r_et if name == "et_r" else r)
            out["variants"][f"{name}_{prec}"] = {"GFLUPs": g, "B_l": bl, "frac_hbm": g * bl / hbm}
            del sv
            torch.cuda.empty_cache()
    dp = COLL_DP_INSTR_UNIT_OMEGA if w["omega_plus"] == 1.0 else COLL_DP_INSTR_GENERAL
    fp = fp64_pipe_peak(lbm, torch, torch.device("cuda", 0), torch.cuda.current_stream())
    out["aa_r_f64_fp64_pipe_frac"] = out["variants"]["aa_r_f64"]["GFLUPs"] * dp / fp["G_dfma_per_s"]
    out["hbm_peak_GBs"] = hbm
    return out


def suite_graph(args, lbm, torch):
    """Launch overhead on the small sphere box (64x32x32, ~46k nodes): direct launches vs CUDA graph replay."""
    solid = geometry.sphere_box_64x32x32(0)
    lat = lbm.Lattice(solid, periodic=(1, 0, 0)).upload()
    out = {"suite": "graph", "fluid_nodes": lat.N, "steps": 2000, "variants": {}}
    w = WORKLOAD
    for prec in ("f64", "f32"):
        params = lbm.Params(omega_plus=1.0, magic=3 / 16, g=(1e-6, 0, 0), shifted=(prec == "f32"))
        for form in ("osnt", "aa"):
            rec = {}
            for mode in ("direct", "graph"):
                sv = lbm.Solver(lat, prec, params, form=form, ria=True)
                sv.init_equilibrium(1.0)
                run = sv.step if mode == "direct" else sv.step_graph
                run(20)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                run(2000)
                b.record()
                torch.cuda.synchronize()
                ms = a.elapsed_time(b)
                rec[mode] = {"us_per_step": 1000 * ms / 2000, "GFLUPs": lat.N * 2000 / (ms / 1e3) / 1e9}
            out["variants"][f"{form}_r_{prec}"] = rec
    return out


SUITES = {"bandwidth": suite_bandwidth, "partition": suite_partition, "exchange": suite_exchange, "bed40": suite_bed40,
          "graph": suite_graph, "channel": suite_channel, "sweep": suite_sweep, "foam": suite_foam, "adjoint": suite_adjoint,
          "large": suite_large}


def run_reference(args):
    """--impl reference: the oracle on a bounded sample, same metric and unit.

    The sample is a z-slab of the same bed, its tables built once.  One pair on
    an 8-layer slab measures the oracle's speed on this host; the slab is then
    sized so that each of the W + K steps (one AA even + odd pair) takes an
    equal share of about 150 s, between 4 and 64 layers.
    """
    import torch
    from oracle import lbm as olbm, tables as otables

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    solid = make_geometry()
    torch.set_num_threads(len(os.sched_getaffinity(0)))
    w = WORKLOAD
    p = olbm.Params(omega_plus=w["omega_plus"], magic=w["magic"], g=w["g"])

    def slab(z):
        T = otables.Tables(np.ascontiguousarray(solid[:z]), periodic=w["periodic"], enum="lex", B=1)
        A = olbm.from_canonical(olbm.uniform_state(T.N, p), 1, T.adj, p)
        return T, A, torch.as_tensor(T.adj.astype(np.int64))

    def pair(A, adj):
        t0 = time.perf_counter()
        A = olbm.aa_odd(olbm.aa_even(A, p), adj, p)
        return A, time.perf_counter() - t0

    T, A, adj = slab(8)
    _, t8 = pair(A, adj)
    budget = 150.0 / max(1, args.steps + args.warmup)
    zslab = int(max(4, min(64, 8 * budget / max(t8, 1e-6))))
    T, A, adj = slab(zslab)
    for _ in range(args.warmup):
        A, _ = pair(A, adj)
    total = 0.0
    for _ in range(args.steps):
        A, dt = pair(A, adj)
        total += dt
    value = 2 * T.N * args.steps / total / 1e9
    sample = (f"z < {zslab} slab of the 256^3 bed ({T.N} fluid nodes), one AA even+odd pair of the FP64 "
              f"oracle per step")
    line = {"impl": "reference", "metric": "sparse D3Q19 TRT AA-R FP64 lattice updates per second",
            "value": value, "unit": "GFLUP/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "sample": f"z < {zslab} slab", "step": "AA even+odd pair"},
            "cpu_baseline": {"value": value, "unit": "GFLUP/s", "cores": torch.get_num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GFLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 768^3 production-run leg")
    ap.add_argument("--box", type=int, default=None, help="smaller cubic bed (profiling only)")
    ap.add_argument("--suite", default=None, choices=sorted(["bandwidth", "channel", "sweep", "foam", "adjoint", "exchange", "bed40",
                                                             "large", "partition", "graph"]),
                    help="measure another configuration instead of the headline (one JSON line)")
    ap.add_argument("--radius", type=float, default=None, help="foam strut radius (suites foam/large)")
    ap.add_argument("--foam-steps", type=int, default=2000)
    ap.add_argument("--large-steps", type=int, default=5000)
    ap.add_argument("--adj-T", type=int, default=2000)
    ap.add_argument("--adj-K", type=int, default=45)
    ap.add_argument("--fd", type=int, default=0, help="adjoint suite: finite-difference nodes")
    ap.add_argument("--prec", default="f64", choices=["f64", "f64df", "f32", "f16s"],
                    help="storage/arithmetic of the timed AA-R pair (the headline is f64)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    import paper_1410_0412_gb300 as lbm

    if args.suite:
        torch.cuda.set_device(0)
        out = SUITES[args.suite](args, lbm, torch)
        print(json.dumps(out))
        return 0

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w = WORKLOAD
    t0 = time.time()
    solid = make_geometry(args.box)
    lat = lbm.Lattice(solid, periodic=w["periodic"], enum="lex", B=1)
    lat.upload(lbm.LBM_TABLES_ADJ | lbm.LBM_TABLES_RIA | lbm.LBM_TABLES_ET, device=dev)
    setup_s = time.time() - t0
    N, R = lat.N, lat.R
    r = R / N
    hp = args.prec
    params = lbm.Params(omega_plus=w["omega_plus"], magic=w["magic"], g=w["g"], shifted=hp in ("f32", "f16s"))
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # ---- headline: AA-R FP64, one even+odd pair per step ---------------------------------------------
    solver = lbm.Solver(lat, hp, params, form="aa", ria=True)
    solver.init_equilibrium(1.0)
    for _ in range(args.warmup):
        solver.step(2)
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with Clocks(local) as clk:
        start.record(stream)
        for k in range(K):
            ev[k][0].record(stream)
            lbm.lbm_step_aa(lat, hp, params, solver.pdf, 0, None, True)
            ev[k][1].record(stream)
            lbm.lbm_step_aa(lat, hp, params, solver.pdf, 1, None, True)
            ev[k][2].record(stream)
        stop.record(stream)
        barrier()
    solver.t += 2 * (args.warmup + K)
    clock_summary = clk.summary()
    ms, value = job_time_and_value(start.elapsed_time(stop), K, N, world, dev)
    even_ms = sum(e[0].elapsed_time(e[1]) for e in ev) / K
    odd_ms = sum(e[1].elapsed_time(e[2]) for e in ev) / K
    # mass check of the timed run (walls + periodic faces conserve mass)
    _, _, sums = solver.macroscopic(fields=False)
    mass = float(sums[0])

    hbm, hbm_kind = peaks()
    p = {"f64": 8, "f64df": 8, "f32": 4, "f16s": 2}[hp]
    odd_dom = odd_ms >= even_ms
    dom_ms = odd_ms if odd_dom else even_ms
    dom_name = f"aa_{'odd_ria' if odd_dom else 'even'}_{hp}"
    dom_bl = loop_balance("aa_odd_r" if odd_dom else "aa_even", p, r)
    achieved_gbs = dom_bl * N / (dom_ms / 1e3) / 1e9
    prof = TRAFFIC_PROFILED.get((dom_name, N)) if args.box is None else None
    roofline = {"kernel": dom_name, "bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
                "frac": achieved_gbs / hbm, "traffic": prof[0] if prof else None,
                "traffic_source": prof[1] if prof else None,
                "peak_kind": f"{hbm_kind} copy bandwidth (STREAM-style), burst",
                "bytes_per_node": dom_bl, "units_per_launch": N,
                "kernel_ms": {"even": even_ms, "odd": odd_ms},
                "step_GBs": (loop_balance("aa_r", p, r) * 2 * N) / (ms / K / 1e3) / 1e9}
    if hp == "f64":
        # the native FP64 step's second roof: its FP64-pipe work against the
        # pipe's measured throughput (DFMA chains, CUDA events, clock sampled)
        fp = fp64_pipe_peak(lbm, torch, dev, stream)
        dp_instr = COLL_DP_INSTR_UNIT_OMEGA if w["omega_plus"] == 1.0 else COLL_DP_INSTR_GENERAL
        dp_rate = dp_instr * N / (dom_ms / 1e3) / 1e9
        roofline["fp64_pipe"] = {"bound": "alu", "achieved": dp_rate, "peak": fp["G_dfma_per_s"],
                                 "unit": "G FP64-instr/s", "frac": dp_rate / fp["G_dfma_per_s"],
                                 "dp_instr_per_node": dp_instr, "peak_measured": fp}

    # ---- the same pair with the double-float collision (FP64 grids, same FP64 parity bar) -------------
    companion = None
    if hp == "f64" and not args.no_variants:
        sdf = lbm.Solver(lat, "f64df", params, form="aa", ria=True)
        sdf.init_equilibrium(1.0)
        for _ in range(args.warmup):
            sdf.step(2)
        evd = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
                torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        barrier()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for k in range(K):
            evd[k][0].record(stream)
            lbm.lbm_step_aa(lat, "f64df", params, sdf.pdf, 0, None, True)
            evd[k][1].record(stream)
            lbm.lbm_step_aa(lat, "f64df", params, sdf.pdf, 1, None, True)
            evd[k][2].record(stream)
        c1.record(stream)
        barrier()
        cms = c0.elapsed_time(c1)
        e_ms = sum(e[0].elapsed_time(e[1]) for e in evd) / K
        o_ms = sum(e[1].elapsed_time(e[2]) for e in evd) / K
        cval = world * 2 * N * K / (cms / 1e3) / 1e9
        cbl = loop_balance("aa_odd_r", 8, r)
        companion = {"value": cval, "unit": "GFLUP/s", "ms_per_step": cms / K,
                     "what": "the timed AA-R pair on the same FP64 grids with the collision in double-float "
                             "(FP32-pair, 48-bit) arithmetic; held to the same 1e-12 FP64 parity bar",
                     "kernel_ms": {"even": e_ms, "odd": o_ms},
                     "roofline_hbm": {"kernel": "aa_odd_ria_f64df", "bound": "hbm",
                                      "achieved": cbl * N / (o_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                                      "frac": cbl * N / (o_ms / 1e3) / 1e9 / hbm}}
        del sdf
        torch.cuda.empty_cache()

    # ---- end to end through host buffers: H2D state, one pair, D2H state -------------------------------
    # Three independent states are in flight, each on its own stream: a step of
    # a state copies it in from pinned host memory, runs the AA pair on it and
    # copies it back out.  One state's copies overlap the others' pairs, and the
    # two copy directions run at the same time.
    e2e = None
    if rank == 0 or world > 1:
        nstate = 3
        hosts = [torch.empty((19, lat.Npad), dtype=solver.pdf.dtype, pin_memory=True) for _ in range(nstate)]
        devs = [solver.pdf] + [torch.empty_like(solver.pdf) for _ in range(nstate - 1)]
        for h in hosts:
            h.copy_(solver.pdf)
        side = [torch.cuda.Stream(dev) for _ in range(nstate)]
        Ke = nstate * max(2, K // (2 * nstate))
        barrier()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for st in side:
            st.wait_stream(stream)
        for k in range(Ke):
            j = k % nstate
            with torch.cuda.stream(side[j]):
                devs[j].copy_(hosts[j], non_blocking=True)
                lbm.lbm_step_aa(lat, hp, params, devs[j], 0, None, True, stream=side[j])
                lbm.lbm_step_aa(lat, hp, params, devs[j], 1, None, True, stream=side[j])
                hosts[j].copy_(devs[j], non_blocking=True)
        for st in side:
            stream.wait_stream(st)
        s1.record(stream)
        barrier()
        ems = s0.elapsed_time(s1)
        nb = 19 * lat.Npad * p
        e2e = {"value": world * 2 * N * Ke / (ems / 1e3) / 1e9, "unit": "GFLUP/s", "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": nb,
               "what": "per step: pinned-host -> device copy of an FP64 state, AA even+odd, device -> "
                       "pinned-host copy of the state; three independent states in flight on three streams"}
        del hosts, devs

    # ---- per-variant numbers ------------------------------------------------------------------------
    variants = {}
    r_et = (len(lat.et_runs()[0]) - 1) / max(N, 1)
    if not args.no_variants:
        del solver
        torch.cuda.empty_cache()
        Kv = max(4, K // 2)
        for prec, pb in (("f64", 8), ("f64df", 8), ("f32", 4), ("f16s", 2)):
            vp = lbm.Params(omega_plus=w["omega_plus"], magic=w["magic"], g=w["g"],
                            shifted=(prec in ("f32", "f16s")))
            for form, ria in (("osnt", False), ("osnt", True), ("aa", False), ("aa", True), ("et", False),
                              ("et", True)):
                name = f"{form}{'_r' if ria else ''}"
                sv = lbm.Solver(lat, prec, vp, form=form, ria=ria)
                sv.init_equilibrium(1.0)
                sv.step(4)
                barrier()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sv.step(2 * Kv)
                b.record(stream)
                barrier()
                vms = a.elapsed_time(b)
                g = 2 * N * Kv / (vms / 1e3) / 1e9
                bl = loop_balance(name, pb, r_et if name == "et_r" else r)
                variants[f"{name}_{prec}"] = {"GFLUPs": g, "B_l": bl, "GBs_model": g * bl,
                                              "frac_hbm": g * bl / hbm, "roof_GFLUPs_8TBs": 8000 / bl}
                del sv
                torch.cuda.empty_cache()

    # ---- the metric's comparisons: FP32 / FP16S against FP64, the adjoint's cost, energy -------------
    def leg(fn, *a, **k):
        # a comparison leg is reported, and never hides the headline if it fails
        try:
            return fn(*a, **k)
        except Exception as e:
            return {"error": f"{type(e).__name__}: {e}"}

    vs_f64 = adjoint = energy = adjoint_cfg = None
    if not args.no_variants:
        vs_f64 = leg(precision_leg, lbm, torch, lat, dev, stream)
        adjoint = leg(adjoint_leg, lbm, torch, solid, dev)
        energy = leg(energy_leg, lbm, torch, lat, dev, stream)
        # the differentiation configuration itself (128^3 box, T = 2000, K = 45): FP32 and FP64
        # backward/forward, and FD of the FP64 forward at 6 nodes with the noise floor
        adjoint_cfg = leg(adjoint_box, lbm, torch, 128, 2000, 45, variants=(("f32", "f32", True), ("f64", "f64", True)),
                          fd=6, fd_h=(1e-4, 2e-4))

    # ---- the production configuration: 768^3 foam, FP32 AA-R, 5000 steps (one GPU only) -------------
    production = None
    if world == 1 and not args.no_variants and not args.no_large and args.box is None:
        production = leg(production_run, lbm, torch)

    cpu = None
    if rank == 0 and not args.no_cpu:
        try:
            import torch as _t
            _t.set_num_threads(len(os.sched_getaffinity(0)))
            cpu = cpu_oracle_sample(solid, 3, zslab=64)
            cpu.pop("seconds", None)
            # the same oracle's OS-NT step on the same slab
            osnt = cpu_oracle_sample(solid, 2, zslab=64, form="osnt")
            osnt.pop("seconds", None)
            cpu["osnt"] = osnt
            # the same oracle on one host thread, one pair on a thin slab
            _t.set_num_threads(1)
            one = cpu_oracle_sample(solid, 1, zslab=8)
            one.pop("seconds", None)
            cpu["one_thread"] = one
            _t.set_num_threads(len(os.sched_getaffinity(0)))
        except Exception as e:  # the baseline must never hide the GPU number
            cpu = {"error": str(e)}

    line = {
        "metric": "sparse D3Q19 TRT AA-R FP64 lattice updates per second" if hp == "f64"
                  else f"sparse D3Q19 TRT AA-R lattice updates per second ({hp} storage)",
        "value": value, "unit": "GFLUP/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f64": "f64", "f64df": "f64 storage, f32-pair arithmetic", "f32": "f32",
                  "f16s": "f16 storage, f32 arithmetic"}[hp], "data": "synthetic",
        "config": {"workload": WORKLOAD["name"] if not args.box else f"packed_bed_{args.box}_rsa_r12",
                   "box": [solid.shape[2], solid.shape[1], solid.shape[0]], "fluid_nodes": N, "runs": R, "et_runs_per_node": r_et,
                   "r": r, "porosity": geometry.porosity(solid), "enumeration": "lex B=1",
                   "step": "AA even + odd with RIA (2 lattice updates)", "parallelism": "replicas" if world > 1
                   else "single GPU", "l2": "inputs larger than L2 (state %.2f GB)" % (19 * lat.Npad * 8 / 1e9),
                   "setup_s": setup_s, "mass_after": mass},
        "roofline": roofline, "f64_double_float": companion,
        "variants": variants, "vs_f64": vs_f64, "adjoint": adjoint, "cpu_baseline": cpu,
        "e2e": e2e, "gpu_launches": 2 * K, "clocks": clock_summary, "energy": energy,
        "production_run": production, "adjoint_box_128": adjoint_cfg,
        "paper_context": {"what": "the paper's roofline predictions, FP64 on 7 Haswell cores of one ccNUMA domain "
                                  "(Table 4, channel, 2.6 GHz), MFLUP/s; context, not a target",
                          "OS-NT": 63.8, "OS-NT-R": 78.4, "AA": 73.8, "AA-R": 82.2},
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
