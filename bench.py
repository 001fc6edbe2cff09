"""Benchmark: GSM solves/s at 31^3 harmonics to relative residual 1e-8 on one
B300 (woodpile of rods eps 11.9, Lambda = 0.35 lambda, 64^3 FFT grid).

One step = one batched solve of B incident points (kappa over [0.70, 0.90] k0,
x and y polarisation, normal incidence) with the complex64 FFT matvec inside
FP64 iterative refinement, fields left in HBM.  Reported beside it: the plain
FP64 GPU path on the same batch, the end-to-end rate through the C ABI with
host buffers, the dominant kernel's roofline position and the CPU oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--impl reference]

With N > 1 (torchrun) every rank solves its own batch (independent points:
replicas, weak scaling); the max over ranks of the timed region is used.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1501_01752_b300 import workloads as wl  # noqa: E402

METRIC = "solves/s at 31^3 harmonics, residual 1e-8: FP32+refine vs FP64 on B300; HBM % peak"
N_HARM = (31, 31, 31)
TOL = 1e-8
L2_BYTES = 126 * 1024 * 1024
L_FFT = 64
# Algorithmic bytes of one complex64 product of one instance (the unit of the
# roofline): read x and write y (3 N^3 complex each), the 3 L^2 N
# intermediate written and read twice, and the L^3 real multiplier,
#   B_mv = 8 * 3 (2 N^3 + 4 L^2 N) + 4 L^3 = 14.67 MB at N = 31, L = 64.
B_MV = 8 * 3 * (2 * N_HARM[0] ** 3 + 4 * L_FFT ** 2 * N_HARM[0]) + 4 * L_FFT ** 3
# Bytes this implementation's x-first layout actually moves per instance and
# product (3 L N^2 intermediate): x-forward s_c (U + 3 L N^2), yz pass
# 2 s_c 3 L N^2, x-inverse + Green s_c (3 L N^2 + 2 U) + 4 N^3, plus the
# multiplier once per launch.  The preconditioned product of the solves adds
# the per-harmonic denominators read by its three-component pass 1 (4 N^3).
_U = 3 * N_HARM[0] ** 3
_TSZ = 3 * L_FFT * N_HARM[1] * N_HARM[2]
OWN_MV = 8 * (_U + _TSZ) + 16 * _TSZ + 8 * (_TSZ + 2 * _U) + 4 * N_HARM[0] ** 3
OWN_MV_PC = OWN_MV + 4 * N_HARM[0] ** 3
# FP32-pipe operations (an FMA counts once) of the complex64 yz pass for one
# instance: per (r_x, c) plane N_z y transforms with inputs pruned to the
# harmonics, L_z z columns of forward transform, times the real D(r) and
# inverse transform, and N_z inverse y transforms with pruned outputs.  Per
# lane of a 64-point transform (radix 8 x 8, seven twiddle products of four
# operations): forward 36 (8-point DFT of four nonzero inputs) + 28 + 52,
# inverse 52 + 28 + 44 (four kept outputs); D is two operations per value.
_YZ_T = 8 * ((36 + 28 + 52) + (52 + 28 + 44))
OPS_YZ = 3 * L_FFT * ((N_HARM[0] + L_FFT) * _YZ_T + 2 * L_FFT * L_FFT)
# dram__bytes_read.sum + dram__bytes_write.sum of the three kernels of one
# product launch at the bench batch (512 instances), from one ncu capture of
# the current kernels, per operator; None where no capture of the current
# kernels exists.
NCU_TRAFFIC = {"precond": 4.1069e9, "plain": 4.0693e9}
# FP64 work of one FP64 product of one instance on this grid, from one ncu
# count of the three FP64 product kernels at 32 instances: floating-point
# operations (2 DFMA + DADD + DMUL) and FP64-pipe instructions (DFMA + DADD +
# DMUL, each one issue of the pipe); None until counted for the current kernels.
FP64_FLOP_PER_PRODUCT = 55.347e6
FP64_INSTR_PER_PRODUCT = 44.70e6


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                for n, v in zip(names, r[3:7]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
            except Exception:
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(points, budget_s=20.0, fields=None):
    """The oracle (FP64 GMRES, scipy FFT on all host cores) on a bounded sample
    of the batch: as many points as fit in about budget_s seconds.  The
    oracle's fields are appended to `fields` when a list is given."""
    from oracle import operator as oop
    from oracle import retrieval as ort
    cores = os.cpu_count() or 1
    oop.WORKERS = cores
    st = wl.woodpile()
    ost = ort.Structure(st["periods"], st["eps_host"], st["shapes"])
    Delta = ost.delta(N_HARM, 1.0)
    done, t0 = 0, time.perf_counter()
    for p in points:
        Eo, _ = ort.solve_point(ost, N_HARM, 1.0, p["k0"], p["kdir"], p["kappa"], p["pol"], tol=TOL, Delta=Delta)
        if fields is not None:
            fields.append(np.asarray(Eo).ravel())
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": "%d of the %d woodpile points, 31^3 harmonics, FP64 GMRES(60) to 1e-8, scipy FFT on %d threads"
                      % (done, len(points), cores)}


def workload_config(args, ws):
    """The config object of the JSON line, the same for both arms."""
    return {"workload": "woodpile eps 11.9 in eps_b 1, Lambda 0.35, 31^3 harmonics, 64^3 FFT grid",
            "global_batch": args.batch * ws, "tol": TOL, "krylov": args.krylov, "form": args.form.upper(),
            "precond": args.precond, "l2": "flushed between steps (inputs+basis > L2)",
            "parallelism": "replicas" if ws > 1 else "single"}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl != "reference" else "gloo")
    return ws, rank, local


def run_reference(args, ws, rank):
    if rank != 0:
        return
    pts = wl.woodpile_batch(args.batch)
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; its first solve is timed like the rest
    vals = []
    t_all = time.perf_counter()
    for s in range(args.steps):
        cb = cpu_baseline(pts[s % len(pts):] + pts[:s % len(pts)], budget_s=max(5.0, 60.0 / max(1, args.steps)))
        vals.append(cb["value"])
    dt = time.perf_counter() - t_all
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128 (fp64)",
            "data": "synthetic", "config": workload_config(args, ws),
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=512,
                    help="points per batched solve (measured on one B300: 128: 3685, 256: 3877, 512: 4165-4174, "
                         "1024: 4204 solves/s)")
    ap.add_argument("--impl", default="ours")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--alt-steps", type=int, default=5,
                    help="timed steps of the other Krylov method on the same batch (0 skips it)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--inner-tol", type=float, default=0.0,
                    help="relative tolerance of the complex64 inner GMRES cycles (0 = library default 1e-4)")
    ap.add_argument("--form", default="e", choices=["e", "h"],
                    help="E-field (Eq. 4) or H-field (Eq. 5) formulation; points keep their polarisation as H amplitude")
    ap.add_argument("--krylov", default="gmres", choices=["gmres", "bicgstab"],
                    help="Krylov method of the refined solve (and of the FP64 plain path)")
    ap.add_argument("--residual", default="auto", choices=["auto", "fp64"],
                    help="outer-residual arithmetic of the refined solve (double-float where available, or FP64)")
    ap.add_argument("--precond", default="auto", choices=["auto", "none"],
                    help="averaged-medium right preconditioner of the Krylov solves (auto) or none")
    ap.add_argument("--mv-batch", type=int, default=32,
                    help="instances per product of the matvec workload")
    ap.add_argument("--sweep-batch", type=int, default=256,
                    help="instances per batch of the sweep workload (batches span truncations; measured on one "
                         "B300, solves/s: 64: 6097, 128: 6761, 256: 7309, 512: 7071)")
    ap.add_argument("--workload", default="woodpile",
                    choices=["woodpile", "matvec", "sweep", "gyroid", "adjoint", "optimise", "nearpole"])
    args = ap.parse_args()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload != "woodpile":
        from paper_1501_01752_b300 import bench_workloads
        bench_workloads.run(args.workload, args)
        return
    import torch
    from paper_1501_01752_b300 import build
    build.build()
    from paper_1501_01752_b300 import gsm
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    st = wl.woodpile()
    B = args.batch
    pts = wl.woodpile_batch(B)
    U = 3 * N_HARM[0] * N_HARM[1] * N_HARM[2]
    stream = torch.cuda.current_stream(dev)

    def make_plan(prec):
        return gsm.plan_for(st, N_HARM, precision=prec, tol=TOL, max_batch=B, device=local,
                            stream=stream.cuda_stream, inner_tol=args.inner_tol,
                            krylov=gsm.BICGSTAB if args.krylov == "bicgstab" else gsm.GMRES,
                            form=gsm.FORM_H if args.form == "h" else gsm.FORM_E,
                            residual=gsm.RESID_FP64 if args.residual == "fp64" else gsm.RESID_AUTO,
                            precond=gsm.PRECOND_NONE if args.precond == "none" else gsm.PRECOND_AUTO)

    plan = make_plan(gsm.FP32_REFINE)
    E = torch.empty(B * U, dtype=torch.complex128, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    def timed(p, steps, out):
        """Per-step CUDA events on the plan's stream; the L2 flush between steps
        sits outside the events.  Returns summed device seconds."""
        tot = 0.0
        infos = None
        for _ in range(steps):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _, infos, s = p.solve(pts, out=out)
            b.record(stream)
            b.synchronize()
            if s:
                raise RuntimeError("solve did not converge: %s" % infos)
            tot += a.elapsed_time(b) / 1000.0
        return tot, infos

    for _ in range(args.warmup):
        plan.solve(pts, out=E)
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    plan.profile(False)          # resets the launch counter; no event records in this region
    torch.cuda.synchronize()
    barrier()
    t_dev, infos = timed(plan, args.steps, E)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = plan.profile_get(7)[0]
    # per-kernel CUDA-event durations: the same steps again with an event pair
    # around every launch on the plan's stream (the roofline and shares)
    plan.profile(True)
    t_prof, _ = timed(plan, args.steps, E)
    kinds = {}
    for k, name in enumerate(["fwd_x", "yz_conv", "inv_x_green", "krylov_dots", "krylov_update", "other",
                              "outer_residual"]):
        n, ms, by = plan.profile_get(k)
        kinds[name] = (n, ms, by)
    plan.profile(False)
    if ws > 1:
        t = torch.tensor([t_dev], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_dev = float(t.item())
    value = ws * B * args.steps / t_dev

    # end to end through the C ABI: points from host memory, fields copied
    # back into pinned host memory inside every step
    Eh = torch.empty(B * U, dtype=torch.complex128, pin_memory=True)
    ee_steps = max(2, args.steps // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ee_steps):
        plan.solve(pts, host_out=Eh)
    e2e = B * ws * ee_steps / (time.perf_counter() - t0)
    h2d = B * 96  # per-point parameter block copied to the device: k_inc, k_b^2, polarisation, preconditioner (12 doubles)
    d2h = B * U * 16
    # the retrieval workflow's call: gsm_sweep returns only the 0th-order
    # amplitudes E_0 (3 complex128 per point) to the host
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ee_steps):
        plan.sweep(pts)
    e2e_sweep = B * ws * ee_steps / (time.perf_counter() - t0)

    # the other Krylov method on the same batch (few steps; not the headline)
    alt = "bicgstab" if args.krylov == "gmres" else "gmres"
    alt_line = None
    if args.alt_steps > 0:
        palt = gsm.plan_for(st, N_HARM, precision=gsm.FP32_REFINE, tol=TOL, max_batch=B, device=local,
                            stream=stream.cuda_stream, inner_tol=args.inner_tol,
                            form=gsm.FORM_H if args.form == "h" else gsm.FORM_E,
                            krylov=gsm.BICGSTAB if alt == "bicgstab" else gsm.GMRES,
                            residual=gsm.RESID_FP64 if args.residual == "fp64" else gsm.RESID_AUTO,
                            precond=gsm.PRECOND_NONE if args.precond == "none" else gsm.PRECOND_AUTO)
        palt.solve(pts, out=E)
        talt, infos_alt = timed(palt, args.alt_steps, E)
        alt_line = {"krylov": alt, "value": B * args.alt_steps / talt, "unit": "solves/s",
                    "steps": args.alt_steps, "iters_mean": float(np.mean([i["iters"] for i in infos_alt])),
                    "rel_residual_max": float(max(i["rel_residual"] for i in infos_alt))}
        palt.close()

    # plain FP64 GPU path on the same batch (--fp64-steps 0 skips it)
    fp64_value, infos64, fp64_roof = None, None, None
    if args.fp64_steps > 0:
        p64 = make_plan(gsm.FP64)
        p64.solve(pts, out=E)
        t64, infos64 = timed(p64, args.fp64_steps, E)
        fp64_value = B * args.fp64_steps / t64
        p64.close()
        # the FP64 path against the measured FP64 FMA rate: every product of
        # every instance (Krylov products + FP64 residuals) per second
        fp64_peak = gsm.probe_fma(0, local, stream.cuda_stream)
        prods = sum(i["iters"] + i["refine_steps"] for i in infos64) * args.fp64_steps / t64
        fp64_roof = {"bound": "alu (FP64 pipe)", "peak": fp64_peak, "unit": "TFLOP/s",
                     "peak_kind": "measured (gsm_probe_fma FP64)", "instance_products_per_s": prods,
                     "achieved": None if FP64_FLOP_PER_PRODUCT is None else prods * FP64_FLOP_PER_PRODUCT / 1e12,
                     "flop_per_product": FP64_FLOP_PER_PRODUCT,
                     "scope": "product flops over the whole FP64 solve time (Gram-Schmidt not counted)"}
        if FP64_FLOP_PER_PRODUCT is not None:
            fp64_roof["frac"] = fp64_roof["achieved"] / fp64_peak
            # issue share of the FP64 pipe (an FMA-only kernel at the probe's rate = 1)
            fp64_roof["pipe_frac"] = prods * FP64_INSTR_PER_PRODUCT / (fp64_peak * 1e12 / 2)

    peak, peak_kind = peaks()
    # The complex64 product on the full batch with every instance active,
    # R products through gsm_apply, each pass timed with CUDA events on the
    # plan's stream: first the right-preconditioned operator A M^-1 that the
    # Krylov solves iterate with (three-component pass 1 with the scaled input
    # written back, M^-1 x in pass 3: the kernels of the timed solves), then
    # the plain Eq. 4 operator.  (Inside a solve, instances that have
    # converged are masked, so a launch there moves less than B instances'
    # bytes.)
    xd = torch.from_numpy(wl.random_field(N_HARM, 11, batch=B)).to(dev)
    R_MV = 5

    def product_roofline(precond, own_bytes, nvtx):
        plan.apply(pts, xd, precision=gsm.FP32_REFINE, precond=precond)
        plan.profile(True)
        torch.cuda.nvtx.range_push(nvtx)   # lets ncu select these launches (--nvtx-include)
        for _ in range(R_MV):
            plan.apply(pts, xd, precision=gsm.FP32_REFINE, precond=precond)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        mvk = {name: plan.profile_get(k) for k, name in enumerate(["fwd_x", "yz_conv", "inv_x_green"])}
        plan.profile(False)
        n_mv = mvk["fwd_x"][0]
        t_mv = sum(v[1] for v in mvk.values()) / max(1, n_mv) / 1000.0   # s per product
        achieved = B * B_MV / t_mv / 1e9 if t_mv > 0 else 0.0
        own = (B * own_bytes + 4 * L_FFT ** 3) / t_mv / 1e9 if t_mv > 0 else 0.0
        traffic = NCU_TRAFFIC["precond" if precond else "plain"]
        return {"kernel": "c64_product (%s + k_yz_t8x2r + k_inv_x_t8c)" % ("k_fwd_x_t8h" if precond else "k_fwd_x_t8"),
                "operator": "A M^-1 (as in the solves)" if precond else "A (Eq. 4)",
                "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": peak_kind + " (copy, burst)", "traffic": traffic,
                "algorithmic_bytes_per_launch": B * B_MV, "launches": n_mv, "avg_us": 1e6 * t_mv,
                "passes_us": {k: 1000.0 * v[1] / max(1, v[0]) for k, v in mvk.items()},
                "own_layout_bytes_per_launch": B * own_bytes + 4 * L_FFT ** 3,
                "own_layout_GBps": own, "own_layout_frac": own / peak,
                "traffic_over_own_layout": None if traffic is None else traffic / (B * own_bytes + 4 * L_FFT ** 3)}

    # the preconditioner exists for Eq. 4 only: an Eq. 5 solve iterates with the plain operator
    pc_solve = args.precond != "none" and args.form == "e"
    roof = product_roofline(pc_solve, OWN_MV_PC if pc_solve else OWN_MV, "roofline_product")
    fma32 = gsm.probe_fma(1, local, stream.cuda_stream)
    # the yz pass, compute-bound: FP32-pipe operations against the measured
    # FMA instruction rate (the probe's flop rate / 2)
    t_yz = roof["passes_us"]["yz_conv"] * 1e-6
    roof_yz = {"kernel": "k_yz_t8x2r", "bound": "alu", "unit": "Top/s (FP32-pipe lane operations)",
               "ops_per_instance": OPS_YZ, "achieved": B * OPS_YZ / t_yz / 1e12 if t_yz > 0 else None,
               "peak": fma32 / 2, "peak_kind": "measured (gsm_probe_fma FP32 / 2)",
               "frac": (B * OPS_YZ / t_yz / 1e12) / (fma32 / 2) if t_yz > 0 else None, "avg_us": 1e6 * t_yz}
    roof_plain = product_roofline(False, OWN_MV, "roofline_product_plain") if pc_solve else None
    # Gram-Schmidt passes (dots + update) inside the profiled solve, at the
    # algorithmic bytes of the instances still iterating at each step
    kr_ms = kinds["krylov_dots"][1] + kinds["krylov_update"][1]
    kr_by = kinds["krylov_dots"][2] + kinds["krylov_update"][2]
    iters = [i["iters"] for i in infos]
    tot_ms = sum(v[1] for v in kinds.values())
    # the whole solve: the algorithmic bytes B_mv of every product of every
    # instance (the Krylov products; one certified residual per solve, whose
    # 16-byte arithmetic counts twice; one complex64 product per later
    # refinement step, which updates the residual recursively) plus the
    # Gram-Schmidt bytes, over the device time of one step
    n_cert = sum(1 for i in infos if i["refine_steps"] > 0)
    n_rec = sum(max(0, i["refine_steps"] - 1) for i in infos)
    solve_bytes = (sum(iters) + 2 * n_cert + n_rec) * B_MV + kr_by / args.steps
    t_step = t_dev / args.steps
    prof_by = sum(v[2] for v in kinds.values()) / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64 matvec + c128 refinement", "data": "synthetic",
        "config": workload_config(args, ws),
        "fp64_plain": None if fp64_value is None else
        {"value": fp64_value, "unit": "solves/s", "iters_mean": float(np.mean([i["iters"] for i in infos64])),
         "roofline": fp64_roof},
        "measured_fma_tflops": {"fp32": fma32,
                                "fp32x2": gsm.probe_fma(2, local, stream.cuda_stream)},
        "speedup_vs_fp64": None if fp64_value is None else value / ws / fp64_value,
        "alt_krylov": alt_line,
        "iters_mean": float(np.mean(iters)), "refine_steps_mean": float(np.mean([i["refine_steps"] for i in infos])),
        "rel_residual_max": float(max(i["rel_residual"] for i in infos)),
        "roofline": roof,
        "roofline_plain_operator": roof_plain,
        "roofline_yz": roof_yz,
        "roofline_krylov": {"kernel": "k_dots + k_update", "bound": "hbm",
                            "achieved": kr_by / (kr_ms / 1000.0) / 1e9 if kr_ms > 0 else None,
                            "peak": peak, "unit": "GB/s",
                            "frac": (kr_by / (kr_ms / 1000.0) / 1e9) / peak if kr_ms > 0 else None,
                            "bytes": "active instances per step",
                            },
        "roofline_solve": {"bytes_per_step": solve_bytes, "ms_per_step": 1000 * t_step,
                           "achieved": solve_bytes / t_step / 1e9, "peak": peak, "unit": "GB/s",
                           "frac": solve_bytes / t_step / 1e9 / peak,
                           "bytes": "B_mv per Krylov product, 2 B_mv per certified residual (one per solve), B_mv per recursive residual update, + Gram-Schmidt",
                           "own_layout_GBps_profiled": prof_by / (1e-3 * tot_ms / args.steps) / 1e9 if tot_ms else None},
        "kernel_shares": {k: {"launches": v[0], "ms": v[1], "share": v[1] / tot_ms if tot_ms else None}
                          for k, v in kinds.items()},
        "profiled_ms_per_step": 1000 * t_prof / args.steps,
        "e2e": {"value": e2e, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "e2e_sweep": {"value": e2e_sweep, "unit": "solves/s", "call": "gsm_sweep (E_0 only)",
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": B * 48},
        "gpu_launches": int(launches),
        "autotuned_blocks": list(plan.tuned_blocks(gsm.FP32_REFINE)),
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu:
        oracle_fields = []
        line["cpu_baseline"] = cpu_baseline(pts, fields=oracle_fields)
        # the refined complex64 fields of the e2e solves against the oracle's
        # FP64 fields of the same points (both to relative residual 1e-8)
        Eg = Eh.numpy()
        errs = [float(np.linalg.norm(Eg[i * U:(i + 1) * U] - f) / np.linalg.norm(f)) for i, f in enumerate(oracle_fields)]
        line["oracle_parity"] = {"points": len(errs), "field_rel_err_max": max(errs) if errs else None,
                                 "note": "GPU FP32+refine vs oracle FP64 GMRES, both to residual 1e-8"}
    plan.close()
    # the C3 resonance sweep of the retrieval (512 points of truncations
    # 15/21/31 through gsm_sweep, batches across truncations), end to end
    # with the pole fits: a secondary figure, not the headline
    from paper_1501_01752_b300 import bench_workloads
    sw = bench_workloads.sweep_c3(args)
    line["sweep_c3"] = {k: sw[k] for k in ("workload", "solves_per_s", "seconds", "seconds_each", "retrieval_host_ms", "iters_mean",
                                           "rel_residual_max", "max_batch", "batches")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
