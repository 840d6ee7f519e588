"""Benchmark: cell-updates/s per TVD-RK3 step on the 128^3 Taylor-Green
vortex (WENO5-JS characteristic + HLLC + 4th-order viscous, CFL 0.5), FP64
(headline) and mixed FP32 side by side, on one GB300 per rank.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl jxf|reference]

One step = one full RK3 step of the whole hot path (3 x [3 face sweeps +
cell update] + CFL/dt/sums finalisation) on the device-resident state.
``value`` is whole-job throughput (all ranks' cells x steps / max time over
ranks); with N > 1 ranks the grid is 128 x 128 x 128N, one z-slab per rank,
with the halo exchange and the dt all-reduce inside every step (weak
scaling).  ``--impl reference`` times the CPU oracle instead, on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "cell-updates/s per RK3 step (FP64 vs FP32, 1 GB300) and % of roofline"
UNIT = "cell-updates/s"
N_TGV = 128


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="jxf", choices=["jxf", "reference"])
    p.add_argument("--size", type=int, default=N_TGV)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--precision", default="both", choices=["both", "fp64", "fp32"])
    p.add_argument("--no-extras", action="store_true",
                   help="skip the batched-drops and adjoint measurements")
    p.add_argument("--workload", default="tgv", choices=["tgv", "drops", "kh-adjoint", "shock-bubble", "weno5z", "teno6a",
                                                              "levelset", "levelset-step", "levelset-step-launches"],
                   help="tgv: the benchmark line; drops / kh-adjoint / shock-bubble / weno5z / teno6a / "
                        "levelset / levelset-step: that workload alone; levelset-step-launches: one "
                        "level-set step, untimed (for a launch list)")
    p.add_argument("--tiling", default=None,
                   help="drops: fixed 'tile_faces,blocks_per_sm' instead of the autotuner")
    return p.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------- clocks --
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t0, t1):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, line in self.lines:
            if ts < t0 - 0.05 or ts > t1 + 0.15:
                continue
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ roofline ----
def _sm_count():
    """Streaming multiprocessors of the current device (152 on a GB300)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    except Exception:  # no device: the nominal count
        pass
    return 152


def _peaks():
    """Denominators: HBM from the measured copy; plain-ALU peaks derived from
    the unit counts and the maximum SM clock (the device's SM count, 2.07
    GHz): FP32 128 lanes x 2 flop (FMA) per SM per clock; FP64 the GB300's
    1.25 TFLOP/s nominal (about 4 flop per SM per clock)."""
    p = {"hbm_gbs": 6781.8, "source": "fallback"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            m = json.load(f)
        p["hbm_gbs"] = m.get("hbm_gbs", p["hbm_gbs"])
        p["source"] = "measured"
    sms, clk = _sm_count(), 2.07e9
    p["sms"] = sms
    p["fp32_tflops"] = sms * 128 * 2 * clk / 1e12
    p["fp64_tflops"] = 1.25
    return p


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the dominant kernel from an ncu capture of the x face sweep on this
# workload, together with the hash of the device
# code it was measured on (_kernel_sha): reported only while that code still
# matches.
TRAFFIC = {"fp64": (205.15e6, "3469826877e13720ecfadfe98350b9d6f0ecfc0fe2ab8b714f434e86fe6dcb0f"),
           "fp32": (88.06e6, "3469826877e13720ecfadfe98350b9d6f0ecfc0fe2ab8b714f434e86fe6dcb0f")}


def _kernel_sha():
    """Hash of the device code the face sweeps are built from: the kernel
    headers, the precision/model instantiation units and the C header, with
    comments and blank lines removed (the host runtime units jxf_host.cu,
    jxf_batch.cu, jxf_static.cu are left out)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2402_05193_gb300", "csrc")
    files = [os.path.join(csrc, f) for f in sorted(os.listdir(csrc))
             if f.endswith(".cuh") or (f.endswith(".cu") and f.startswith(("jxf_f32_", "jxf_f64_")))]
    files.append(os.path.join(ROOT, "include", "jxf.h"))
    import re
    h = hashlib.sha256()
    for p in files:
        with open(p) as fh:
            src = fh.read()
        # comments and blank runs do not change the kernels
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        src = "\n".join(line.rstrip() for line in src.splitlines() if line.strip())
        h.update(os.path.basename(p).encode() + b"\0" + src.encode())
    return h.hexdigest()


def _traffic(prec):
    nbytes, sha = TRAFFIC[prec]
    return nbytes if nbytes is not None and sha == _kernel_sha() else None


def _flop_counts():
    with open(os.path.join(ROOT, "tests", "golden", "flop_counts.json")) as f:
        return json.load(f)["tgv_32"]


# ------------------------------------------------------------- our arm ----
def run_jxf(args):
    import torch
    import torch.distributed as dist

    import paper_2402_05193_gb300 as jxf
    from paper_2402_05193_gb300 import workloads as wl

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    case = wl.tgv(args.size, steps=args.steps)
    ncell = args.size ** 3
    stream = torch.cuda.current_stream()
    flops = _flop_counts()
    peaks = _peaks()

    def barrier():
        if ws > 1:
            dist.barrier()

    def max_over_ranks(x):
        from paper_2402_05193_gb300.dist import max_over_ranks as mor
        return mor(x, device="cuda")

    results = {}
    probe = {"fp64": jxf.jxf_peak_probe(jxf.JXF_FP64), "fp32": jxf.jxf_peak_probe(jxf.JXF_MIXED32)}
    precs = ("fp64", "fp32") if args.precision == "both" else (args.precision,)
    for prec in precs:
        esize = 8 if prec == "fp64" else 4
        s = jxf.Solver(case, prec)
        s.set_primitive(case["W"])
        if ws > 1:
            # one grid of size x size x (size * ranks) split into one slab per
            # rank (the TGV is 2 pi periodic in z: every slab starts from the
            # same field); halo exchange and dt all-reduce inside the steps
            from paper_2402_05193_gb300.decomp import DistSlab
            gcase = dict(case, n=[args.size, args.size, args.size * ws])
            runner = DistSlab(gcase, prec)
            runner.set_primitive(case["W"])
            advance = runner.step
        else:
            runner = s
            advance = lambda k: s.step(k, sync=False)  # noqa: E731
        advance(args.warmup)
        sampler = ClockSampler(local) if prec == precs[0] else None
        if sampler:
            sampler.start()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.time()
        e0.record(stream)
        for _ in range(args.steps):
            advance(1)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        t1 = time.time()
        ms = max_over_ranks(e0.elapsed_time(e1))
        clocks = sampler.stop(t0, t1) if sampler else None
        if ws > 1:
            runner.stats()  # raises on a non-admissible state
        else:
            s.step(0)  # status check
        # per-kernel device times of the same steps, launched one by one
        prof = s.step_profiled(args.steps)
        # end to end through the C interface: host state in, steps, host state out
        host = torch.empty(s.shape, dtype=s.dtype, pin_memory=True)
        jxf.jxf_get_state(s.h, host)
        barrier()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        for _ in range(args.steps):
            if ws > 1:
                runner.set_state(host)
                runner.step(1)
                jxf.jxf_get_state(runner.h, host)
            else:
                jxf.jxf_set_state(s.h, host)
                jxf.jxf_step(s.h, 1, sync=False)
                jxf.jxf_get_state(s.h, host)
        torch.cuda.synchronize()
        barrier()
        e2e_ms = max_over_ranks((time.perf_counter() - t2) * 1e3)
        state_bytes = s.nv * ncell * esize
        if ws > 1:
            runner.close()
        s.close()

        flux_ms = sum(prof[k][0] for k in ("flux_x", "flux_y", "flux_z"))
        flux_n = sum(prof[k][1] for k in ("flux_x", "flux_y", "flux_z"))
        x_ms, x_n = prof["flux_x"]
        step_dev_ms = sum(v[0] for v in prof.values()) / args.steps
        # dominant kernel: the x face sweep (one of three equal sweeps)
        alg_flops_launch = flops["face_x"] * ncell
        achieved = alg_flops_launch / (x_ms / x_n * 1e-3) / 1e12
        peak = peaks["fp64_tflops"] if prec == "fp64" else peaks["fp32_tflops"]
        results[prec] = {
            "value": ws * ncell * args.steps / (ms * 1e-3),
            "ms_per_step": ms / args.steps,
            "clocks": clocks,
            "e2e": {"value": ws * ncell * args.steps / (e2e_ms * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes},
            "roofline": {"bound": "alu", "kernel": "k_flux (x sweep)", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": _traffic(prec),
                         "flops_per_launch": alg_flops_launch,
                         "avg_launch_ms": x_ms / x_n,
                         "peak_source": "derived: FP64 1.25 TFLOP/s nominal" if prec == "fp64"
                         else "derived: %d SM x 128 lanes x 2 x 2.07 GHz" % peaks["sms"],
                         "measured_fma_peak": probe[prec],
                         "frac_of_measured_fma_peak": achieved / probe[prec]},
            "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
            "flux_share": flux_ms / (step_dev_ms * args.steps),
            "step_roofline_frac": (flops["per_step"] * ncell / (ms / args.steps * 1e-3) / 1e12) / peak,
            "gpu_launches": sum(v[1] for v in prof.values()),
        }
        del flux_n
    if ws > 1:
        dist.destroy_process_group()
    return results


# ------------------------------------------------------- extra workloads --
def run_batched_drops(steps=200, tiling=None, with_cpu=True):
    """The batched workload: 96 drops (N in {64,128,192,256}), FP32, `steps`
    RK3 steps of every simulation in one graph launch, tile shape from the
    autotuner.  cell-updates/s = sum of cells x steps / time."""
    import torch

    import paper_2402_05193_gb300 as jxf
    from paper_2402_05193_gb300 import autotune
    from paper_2402_05193_gb300 import workloads as wl
    from paper_2402_05193_gb300.dist import max_over_ranks, shard_by_cost
    cases = wl.drop_batch()
    ws, rank, _ = _dist()
    total_cells = sum(int(np.prod(c["n"])) for c in cases)
    if ws > 1:  # independent simulations: split by cost, no collective on the data path
        cases = [cases[k] for k in shard_by_cost([int(np.prod(c["n"])) for c in cases], ws, rank)]
    B = jxf.Batch(cases, "fp32")
    B.set_primitives()
    if tiling:
        choice = tuple(int(x) for x in tiling.split(","))
        B.set_tiling(*choice)
    else:
        choice, timings = autotune.tune(B, steps=3)
    B.set_primitives()
    B.step(steps)  # builds the graph of `steps` steps
    B.set_primitives()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    B.step(steps)
    e1.record()
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), device="cuda")
    cells = total_cells
    for k in range(len(cases)):
        B.stats(k)  # raises on a non-admissible state
    B.close()
    value = cells * steps / (ms * 1e-3)
    with open(os.path.join(ROOT, "tests", "golden", "flop_counts.json")) as f:
        fl = json.load(f)["drop_128"]["per_step"]
    peaks = _peaks()
    out = {"workload": "96 water drops, N in {64,128,192,256}, five-equation model, FP32",
           "value": value, "unit": UNIT, "steps": steps, "ranks": ws,
           "ms_total": ms, "launches": 1, "cells": cells,
           "tiling": {"tile_faces": choice[0], "blocks_per_sm": choice[1]},
           "flops_per_cell_step": fl,
           "roofline": {"bound": "alu", "achieved": value * fl / 1e12, "peak": peaks["fp32_tflops"],
                        "unit": "TFLOP/s", "frac": value * fl / 1e12 / peaks["fp32_tflops"],
                        "flops_source": "oracle count on a 128^2 drop of the batch's ranges"}}
    if with_cpu and ws == 1:
        out["cpu_baseline"] = run_oracle_drops()
    return out


def run_oracle_drops(budget_s=10.0):
    """The oracle on a bounded sample of the batch: one RK3 step of each
    simulation in turn (the batch order) until about budget_s seconds."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle
    from case_tools import oracle_config
    from paper_2402_05193_gb300 import workloads as wl
    cells, k, t0 = 0, 0, time.perf_counter()
    for case in wl.drop_batch():
        if time.perf_counter() - t0 > budget_s:
            break
        c = oracle_config(case)
        U = oracle.prim_to_cons(c, case["W"])
        oracle.run(c, U, 1)
        cells += int(np.prod(case["n"]))
        k += 1
    sec = time.perf_counter() - t0
    return {"value": cells / sec, "unit": UNIT, "cores": _cores(), "kind": "oracle",
            "sample": "1 RK3 step of each of the first %d simulations of the batch, %.1f s" % (k, sec)}


def run_shock_bubble(steps32=1000, steps64=100, steps_thinc32=200, steps_thinc64=20):
    """The 256 x 128 x 128 air-helium shock-bubble workload (five-equation
    model, characteristic WENO5-JS, limiters, CFL 0.4): the full 1000 steps in
    mixed FP32, 100 steps in FP64, and the same with THINC (200 / 20 steps),
    each as one graph-captured jxf_step call after 3 warm-up steps;
    cell-updates/s and the fraction of the ALU roofline (the oracle's flop
    count per cell and step of this workload)."""
    import torch

    import paper_2402_05193_gb300 as jxf
    from paper_2402_05193_gb300 import workloads as wl
    base = wl.shock_bubble()
    ncell = int(np.prod(base["n"]))
    with open(os.path.join(ROOT, "tests", "golden", "flop_counts.json")) as f:
        counts = json.load(f)
    peaks = _peaks()
    out = {"workload": "shock-bubble 256x128x128, five-equation model, limiters, CFL 0.4",
           "cells": ncell,
           "flops_per_cell_step": counts["shock_bubble_64x32x32"]["per_step"],
           "flops_per_cell_step_thinc": counts["shock_bubble_thinc_64x32x32"]["per_step"]}
    for key, prec, steps, thinc in (("fp32", "fp32", steps32, False), ("fp64", "fp64", steps64, False),
                                    ("fp32_thinc", "fp32", steps_thinc32, True),
                                    ("fp64_thinc", "fp64", steps_thinc64, True)):
        if steps <= 0:
            continue
        case = dict(base, thinc=thinc)
        fl = counts["shock_bubble_thinc_64x32x32" if thinc else "shock_bubble_64x32x32"]["per_step"]
        s = jxf.Solver(case, prec)
        try:
            s.set_primitive(case["W"])
            s.step(3)
            s.set_primitive(case["W"])
            s.set_time(0.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            s.step(steps, sync=False)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            t = s.step(0)
            _, dt_last, lim = s.stats()
            prof = s.step_profiled(10)
            peak = peaks["fp64_tflops"] if prec == "fp64" else peaks["fp32_tflops"]
            out[key] = {"steps": steps, "t_final": t, "value": ncell * steps / (ms * 1e-3),
                        "unit": UNIT, "ms_per_step": ms / steps,
                        "step_roofline_frac": fl * ncell / (ms / steps * 1e-3) / 1e12 / peak,
                        "limited_il_sides_fl_faces": list(lim),
                        "kernel_ms_per_step": {k: v[0] / 10 for k, v in prof.items()}}
        except Exception as ex:  # a non-admissible state is reported, not hidden
            out[key] = {"error": str(ex)}
        finally:
            s.close()
    return out


def run_scheme_tgv(n=N_TGV, steps=20, weno="z", visc_order=4, key="tgv_32_weno5z",
                   label="WENO5-Z characteristic"):
    """The 128^3 TGV workload with another reconstruction or viscous order:
    cell-updates/s and the ALU-roofline fractions of the x sweep and of the
    whole step, FP64 and mixed FP32 (the oracle's flop count of that scheme,
    tests/golden/flop_counts.json)."""
    import torch

    import paper_2402_05193_gb300 as jxf
    from paper_2402_05193_gb300 import workloads as wl
    case = dict(wl.tgv(n), weno=weno, visc_order=visc_order)
    ncell = n ** 3
    with open(os.path.join(ROOT, "tests", "golden", "flop_counts.json")) as f:
        fl = json.load(f)[key]
    peaks = _peaks()
    out = {"workload": "taylor_green_vortex_%d^3, %s" % (n, label), "cells": ncell,
           "flops_per_cell_step": fl["per_step"]}
    for prec in ("fp64", "fp32"):
        s = jxf.Solver(case, prec)
        s.set_primitive(case["W"])
        s.step(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s.step(steps, sync=False)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        s.step(0)
        prof = s.step_profiled(steps)
        s.close()
        peak = peaks["fp64_tflops"] if prec == "fp64" else peaks["fp32_tflops"]
        x_ms, x_n = prof["flux_x"]
        out[prec] = {"value": ncell * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
                     "x_sweep_frac": fl["face_x"] * ncell / (x_ms / x_n * 1e-3) / 1e12 / peak,
                     "step_roofline_frac": fl["per_step"] * ncell / (ms / steps * 1e-3) / 1e12 / peak}
    return out


def run_weno5z_tgv(n=N_TGV, steps=20):
    """The TGV with the WENO5-Z weights (Borges et al.; the paper's default
    scheme) in place of Jiang-Shu."""
    return run_scheme_tgv(n, steps)


def run_teno6a_tgv(n=N_TGV, steps=10):
    """The TGV with the paper's single-phase scheme: TENO6-A characteristic
    reconstruction and 6th-order central viscous fluxes."""
    return run_scheme_tgv(n, steps, weno="teno6a", visc_order=6, key="tgv_32_teno6a_visc6",
                          label="TENO6-A characteristic + 6th-order viscous")


def run_levelset(n=N_TGV, steps=10, with_cpu=True):
    """The level-set model's data-parallel parts (§3.5, App. D) on the
    level-set transport workload (a sphere in a solid-body rotation on n^3
    cubic cells, FP64).  One step = one TVD-RK3 step of the level-set
    advection, ten reinitialisation steps (the paper's count; threshold
    5e-2) and the interface geometry (apertures, volume fraction, interface
    segment, normal).  Throughput in cell-updates/s and the FP64
    ALU-roofline fraction at the oracle's flop count of that step
    (tests/golden/flop_counts.json, counted at 128^3); the oracle timed
    beside it on one step."""
    import torch

    import paper_2402_05193_gb300 as jxf
    from paper_2402_05193_gb300 import workloads as wl
    case = wl.levelset_sphere(n)
    bcode = {"periodic": jxf.JXF_BC_PERIODIC, "zerograd": jxf.JXF_BC_ZEROGRAD, "symmetry": jxf.JXF_BC_SYMMETRY}
    bc = [(bcode[a], bcode[b]) for a, b in case["bc"]]
    h, dt = case["h"], case["dt"]
    grid = jxf.ls_grid(3, case["n"], h, bc)
    ncell = n ** 3
    with open(os.path.join(ROOT, "tests", "golden", "flop_counts.json")) as f:
        fl = json.load(f)["levelset_sphere_128"]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    phi, u = dev(case["phi"]), dev(case["vel"])
    scratch = torch.zeros((2, n, n, n), dtype=torch.float64, device="cuda")
    ap = torch.zeros(jxf.jxf_ls_nface(grid), dtype=torch.float64, device="cuda")
    al = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    dg = torch.zeros_like(al)
    nr = torch.zeros((3, n, n, n), dtype=torch.float64, device="cuda")

    def step(ev=None):
        if ev:
            ev[0].record()
        jxf.jxf_ls_advect(grid, phi, u, dt, 1, scratch)
        if ev:
            ev[1].record()
        jxf.jxf_ls_reinit(grid, phi, 10, 5e-2, scratch)
        if ev:
            ev[2].record()
        jxf.jxf_ls_geometry(grid, phi, ap, al, dg, nr)
        if ev:
            ev[3].record()

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    parts = [0.0, 0.0, 0.0]
    for _ in range(steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        step(ev)
        torch.cuda.synchronize()
        for k in range(3):
            parts[k] += ev[k].elapsed_time(ev[k + 1]) / steps
    peak = _peaks()["fp64_tflops"]
    achieved = fl["per_step"] * ncell / (ms * 1e-3) / 1e12
    out = {"workload": "level-set sphere (R = 1/4) in a solid-body rotation, %d^3 cubic cells, FP64" % n,
           "cells": ncell, "flops_per_cell_step": fl["per_step"],
           "value": ncell / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
           "kernel_ms_per_step": {"advect_rk3": parts[0], "reinit_10": parts[1], "geometry": parts[2]},
           "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak,
                        "reinit_frac": 20 * fl["reinit_stage"] * ncell / (parts[1] * 1e-3) / 1e12 / peak,
                        "geometry_frac": fl["geometry"] * ncell / (parts[2] * 1e-3) / 1e12 / peak}}
    if with_cpu:
        import oracle as orc
        cfg = orc.ls_config(ndim=3, n=case["n"], h=h, bc=bc)
        t0 = time.time()
        p = orc.ls_advect(cfg, case["phi"], case["vel"], dt, 1)
        p = orc.ls_reinit(cfg, p, 10, 5e-2)
        orc.ls_geometry(cfg, p)
        dtc = time.time() - t0
        out["cpu_baseline"] = {"value": ncell / dtc, "unit": UNIT, "cores": _cores(), "kind": "oracle",
                               "sample": "1 level-set step of the same workload, %.1f s" % dtc}
    return out


def run_levelset_step(n=N_TGV, steps=5, with_cpu=True, cpu_n=64):
    """The level-set model's time step (Alg. 2, inviscid, two phases) through
    jxf_ls_step on the two-phase drop workload (a stiffened-gas drop in an
    ideal gas, uniform flow, n^3 periodic cubic cells, FP64).  One step =
    three TVD-RK3 stages of the cut-cell right-hand sides of both phases, the
    level-set advection, the stage combinations, the reinitialisation (after
    the last stage), the geometry, the mixing, the primitives and the three
    extensions.  Throughput in cell-updates/s; the oracle timed beside it on
    one step of the same workload at cpu_n^3."""
    import torch

    import paper_2402_05193_gb300 as jxf
    from paper_2402_05193_gb300 import workloads as wl
    case = wl.levelset_drop(n)
    h, dt = case["h"], case["dt"]
    ncell = n ** 3
    ls = jxf.LevelSet(3, case["n"], h, [(jxf.JXF_BC_PERIODIC, jxf.JXF_BC_PERIODIC)] * 3, case["mat1"], case["mat2"],
                      "js_char")
    ls.set_state(case["phi"], case["W1"], case["W2"])
    ls.step(dt, 3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ls.step(dt, steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    if not bool(torch.isfinite(ls.aU1).all() and torch.isfinite(ls.aU2).all()):
        raise RuntimeError("level-set step: non-finite state")
    grid, eos, sch, W2, qg = ls.grid, ls.eos, ls.scheme, ls.W2, ls.qg
    # the dominant kernels: the cut-cell right-hand side of the ideal-gas
    # phase (its three face-flux launches and the update) on the state the
    # steps left, timed alone; algorithmic flops = the oracle's count per
    # face flux (tests/golden/flop_counts.json) x the faces the phase wets
    nf = jxf.jxf_ls_nface(grid)
    ap, al, dg, nr = ls.geometry()
    dU = torch.zeros_like(W2)
    scr = torch.zeros(5 * nf, dtype=torch.float64, device="cuda")
    ug, pg = qg[:3], qg[3]
    for _ in range(2):
        jxf.jxf_ls_cut_rhs(grid, eos[1], sch, ap, dg, nr, W2, 2, ug, pg, dU, scr)
    torch.cuda.synchronize()
    reps = 10
    e0.record()
    for _ in range(reps):
        jxf.jxf_ls_cut_rhs(grid, eos[1], sch, ap, dg, nr, W2, 2, ug, pg, dU, scr)
    e1.record()
    torch.cuda.synchronize()
    ms_cut = e0.elapsed_time(e1) / reps
    with open(os.path.join(ROOT, "tests", "golden", "flop_counts.json")) as f:
        ff = json.load(f)["levelset_drop_faces"]
    per_axis = nf // 3
    wet = [int((ap[d * per_axis:(d + 1) * per_axis] < 1.0).sum()) for d in range(3)]
    flops = sum(w * ff["face_" + "xyz"[d]] for d, w in enumerate(wet))
    peak = _peaks()["fp64_tflops"]
    achieved = flops / (ms_cut * 1e-3) / 1e12
    out = {"workload": "two-phase level-set drop (stiffened gas in ideal gas, R = 1/4, uniform flow), "
                       "%d^3 periodic cubic cells, FP64, WENO5-JS characteristic + HLLC" % n,
           "cells": ncell, "value": ncell / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
           "warmup": 3,
           "roofline": {"bound": "alu", "kernel": "cut-cell right-hand side of the ideal-gas phase "
                        "(k_ls_cut_faces x 3 + k_ls_cut_update)", "achieved": achieved, "peak": peak,
                        "unit": "TFLOP/s", "frac": achieved / peak, "ms_per_launch": ms_cut,
                        "wet_faces": wet, "flops_per_face": ff["face_x"],
                        "note": "face-flux flops only (the update's aperture weighting and interface "
                                "terms are not counted)"}}
    if with_cpu:
        import oracle as orc
        c = wl.levelset_drop(cpu_n)
        obc = [(orc.PERIODIC, orc.PERIODIC)] * 3
        c1, c2 = (orc.make_config(ndim=3, n=c["n"], dx=[c["h"]] * 3, bc=obc, gamma=(g_, g_), pinf=(pi, pi),
                                  recon=orc.CHAR) for g_, pi in (c["mat1"], c["mat2"]))
        st = orc.ls_init(c1, c2, c["phi"], c["W1"], c["W2"])
        t0 = time.time()
        orc.ls_step(c1, c2, st, c["dt"], 1)
        dtc = time.time() - t0
        out["cpu_baseline"] = {"value": cpu_n ** 3 / dtc, "unit": UNIT, "cores": _cores(), "kind": "oracle",
                               "sample": "1 step of the same workload at %d^3, %.1f s" % (cpu_n, dtc)}
    return out


def run_levelset_step_launches(n=N_TGV):
    """The launches of one level-set step, for a launch-list capture: the
    two-phase drop workload's state built on the device, jxf_ls_init and one
    jxf_ls_step (dt = 0.1 h), nothing timed."""
    import torch

    import paper_2402_05193_gb300 as jxf
    from paper_2402_05193_gb300 import workloads as wl
    case = wl.levelset_drop(n)
    ls = jxf.LevelSet(3, case["n"], case["h"], [(jxf.JXF_BC_PERIODIC, jxf.JXF_BC_PERIODIC)] * 3, case["mat1"],
                      case["mat2"], "js_char")
    ls.set_state(case["phi"], case["W1"], case["W2"])
    ls.step(0.1 * case["h"], 1)
    torch.cuda.synchronize()
    return {"workload": "one level-set step of the two-phase drop, %d^3" % n,
            "finite": bool(torch.isfinite(ls.aU1).all() and torch.isfinite(ls.aU2).all())}


def run_adjoint_kh(n=256, steps=2000, ckpt=100, with_cpu=True):
    """Gradient of the final kinetic energy w.r.t. the initial density of the
    256^2 Kelvin-Helmholtz workload through the hand-written adjoint (FP64):
    forward (with checkpoints) and backward (recomputation + step adjoints)
    wall times, after a short warm-up rollout that loads every kernel the
    timed one uses (the loss itself is formed outside the timed windows)."""
    import torch

    import paper_2402_05193_gb300 as jxf
    from paper_2402_05193_gb300 import workloads as wl
    from paper_2402_05193_gb300.autograd import rollout
    case = wl.kelvin_helmholtz(n, steps=steps)
    W = case["W"]
    c = np.sqrt(1.4 * W[3] / W[0])
    dt = 0.5 / ((np.abs(W[1]) + c) / case["dx"][0] + (np.abs(W[2]) + c) / case["dx"][1]).max()
    case = dict(case, fixed_dt=dt, t_end=0.0)
    vol = case["dx"][0] * case["dx"][1]
    s = jxf.Solver(case, "fp64")

    def loss(UT):
        return 0.5 * torch.sum((UT[1] ** 2 + UT[2] ** 2) / UT[0]) * vol

    s.set_primitive(W)
    U0 = s.state().clone().requires_grad_(True)
    loss(rollout(U0, s, 4, dt, 2)).backward()  # warm-up
    s.set_primitive(W)
    U0 = s.state().clone().requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    UT = rollout(U0, s, steps, dt, ckpt)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    J = loss(UT)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    J.backward()
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    s.close()
    fwd = n * n * steps / (t1 - t0)
    with open(os.path.join(ROOT, "tests", "golden", "flop_counts.json")) as f:
        fl = json.load(f)["kh_256"]["per_step"]
    peak = _peaks()["fp64_tflops"]
    out = {"workload": "KH %d^2, %d fixed-dt steps, checkpoints every %d, FP64" % (n, steps, ckpt),
           "forward_s": t1 - t0, "backward_s": t3 - t2,
           "forward_cell_updates_per_s": fwd,
           "backward_cell_updates_per_s": n * n * steps / (t3 - t2),
           "flops_per_cell_step": fl,
           "forward_roofline": {"bound": "alu", "achieved": fwd * fl / 1e12, "peak": peak, "unit": "TFLOP/s",
                                "frac": fwd * fl / 1e12 / peak},
           "backward_note": "the reverse sweep (recomputation + step adjoints) has no oracle flop count: "
                            "the oracle has forward (dual-number) mode only"}
    if with_cpu:
        out["cpu_baseline"] = run_oracle_kh(case, dt)
    return out


def run_oracle_kh(case, dt, budget_s=10.0):
    """The oracle on a bounded sample of the KH workload: fixed-dt RK3 steps
    of the value, then of the dual-number tangent along one direction (the
    oracle's derivative mode), each for about half of budget_s."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle
    from case_tools import oracle_config
    c = oracle_config(case)
    U = oracle.prim_to_cons(c, case["W"])
    ncell = int(np.prod(case["n"]))
    out = {}
    for mode in ("value", "tangent"):
        k, t0 = 0, time.perf_counter()
        Uk, Ud = U, np.zeros_like(U)
        Ud[0] = 1.0
        while time.perf_counter() - t0 < budget_s / 2:
            if mode == "value":
                Uk, _, _, _, _ = oracle.run(c, Uk, 5)
            else:
                Uk, Ud = oracle.run_tangent(c, Uk, Ud, 5, dt)
            k += 5
        sec = time.perf_counter() - t0
        out[mode] = {"value": ncell * k / sec, "unit": UNIT, "steps": k, "s": sec}
    return {"value": out["value"]["value"], "unit": UNIT, "cores": _cores(), "kind": "oracle",
            "tangent_value": out["tangent"]["value"],
            "sample": "%d fixed-dt RK3 steps of the %d^2 KH workload (value), %d with the dual-number "
                      "tangent along one direction" % (out["value"]["steps"], case["n"][0],
                                                        out["tangent"]["steps"])}


# ----------------------------------------------------- oracle (CPU) arm ----
def _oracle_setup(n):
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle
    from case_tools import oracle_config
    from paper_2402_05193_gb300 import workloads as wl
    case = wl.tgv(n)
    c = oracle_config(case)
    return oracle, c, oracle.prim_to_cons(c, case["W"])


def _cores():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_oracle_sample(n=N_TGV, budget_s=10.0, max_steps=30):
    """The oracle as it stands on a bounded sample of the workload: RK3 steps
    of the same n^3 TGV, one at a time, until about budget_s seconds."""
    oracle, c, U = _oracle_setup(n)
    t, k, t0 = 0.0, 0, time.perf_counter()
    while k < max_steps and time.perf_counter() - t0 < budget_s:
        U, t, kk, _, _ = oracle.run(c, U, 1, t)
        k += kk
    sec = time.perf_counter() - t0
    return {"value": n ** 3 * k / sec, "unit": UNIT, "cores": _cores(), "kind": "oracle",
            "sample": "%d RK3 steps of the %d^3 TGV workload, %.1f s" % (k, n, sec)}


def run_reference(args):
    """Reference arm: the CPU oracle, on the same workload (128^3 TGV), one
    RK3 step per timed step, on the host cores of rank 0."""
    ws, rank, local = _dist()
    if rank != 0:
        return None
    oracle, c, U = _oracle_setup(args.size)
    t = 0.0
    for _ in range(args.warmup):
        U, t, _, _, _ = oracle.run(c, U, 1, t)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U, t, _, _, _ = oracle.run(c, U, 1, t)
    sec = time.perf_counter() - t0
    value = args.size ** 3 * args.steps / sec
    cb = {"value": value, "unit": UNIT, "cores": _cores(), "kind": "oracle",
          "sample": "each step: 1 RK3 step of the %d^3 TGV workload" % args.size}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(args), "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return line


def _config(args):
    return {"workload": "taylor_green_vortex_%d^3" % args.size, "cells": args.size ** 3,
            "scheme": "WENO5-JS characteristic + HLLC + 4th-order viscous + TVD-RK3, CFL 0.5",
            "physics": "single-phase ideal gas, Ma 0.1, Re 1600, Pr 0.72, periodic",
            "precision": "FP64 headline; mixed FP32 under 'fp32'",
            "parallelism": ("one %dx%dx%d grid in %d z-slabs (halo exchange + dt all-reduce)"
                            % (args.size, args.size, args.size * args.gpus, args.gpus))
            if args.gpus > 1 else "single GPU",
            "l2": "working set (state, stage state, primitives, face fluxes) > L2, no flush"}


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload != "tgv":
        import torch
        import torch.distributed as dist
        ws, rank, local = _dist()
        torch.cuda.set_device(local)
        if ws > 1 and args.workload == "drops":  # simulations split across ranks
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        if args.workload == "drops":
            r = run_batched_drops(steps=args.steps, tiling=args.tiling)
        elif args.workload == "shock-bubble":
            r = run_shock_bubble(steps32=args.steps, steps64=args.steps)
        elif args.workload == "weno5z":
            r = run_weno5z_tgv(n=args.size, steps=args.steps)
        elif args.workload == "teno6a":
            r = run_teno6a_tgv(n=args.size, steps=args.steps)
        elif args.workload == "levelset":
            r = run_levelset(n=args.size, steps=args.steps)
        elif args.workload == "levelset-step":
            r = run_levelset_step(n=args.size, steps=args.steps)
        elif args.workload == "levelset-step-launches":
            r = run_levelset_step_launches(n=args.size)
        else:
            r = run_adjoint_kh(steps=args.steps)
        if dist.is_initialized():
            dist.destroy_process_group()
        if rank == 0:
            print(json.dumps(r))
        return
    ws, rank, local = _dist()
    res = run_jxf(args)
    if rank != 0:
        return
    head = "fp64" if "fp64" in res else "fp32"
    r64 = res[head]
    r32 = res.get("fp32") if head == "fp64" else None
    cb = None
    if ws == 1 and not args.no_cpu_baseline:
        cb = run_oracle_sample(n=args.size)
    extras = {}
    if ws == 1 and not args.no_extras:
        extras["batched_drops"] = run_batched_drops()
        extras["adjoint_kh"] = run_adjoint_kh()
        extras["shock_bubble"] = run_shock_bubble()
        extras["weno5z_tgv"] = run_weno5z_tgv(n=args.size)
        extras["teno6a_visc6_tgv"] = run_teno6a_tgv(n=args.size)
        extras["levelset"] = run_levelset(n=args.size)
        extras["levelset_step"] = run_levelset_step(n=args.size)
    line = {
        "metric": METRIC, "value": r64["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r64["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if head == "fp64" else "f32",
        "data": "synthetic",
        "config": _config(args), "clocks": r64["clocks"], "e2e": r64["e2e"],
        "gpu_launches": r64["gpu_launches"], "roofline": r64["roofline"],
        "cpu_baseline": cb,
        "fp32": {k: r32[k] for k in ("value", "ms_per_step", "e2e", "roofline", "kernel_ms_per_step",
                                     "flux_share", "step_roofline_frac")} if r32 else None,
        head + "_detail": {k: r64[k] for k in ("kernel_ms_per_step", "flux_share", "step_roofline_frac")},
        "paper_context": "JAX-Fluids 2.0 single phase, A100 FP64: 58.01 ns/cell/step = 1.72e7 "
                         "cell-updates/s per device (WENO5-Z, inviscid, 2x2x2 ranks)",
    }
    line.update(extras)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
