"""Benchmark of the GB300 SBCI library on the H10 singlet workload.

Workload: linear H10 chain, STO-3G, Loewdin basis, 1.2 A spacing, 10 orbitals,
5 alpha / 5 beta electrons, 252 x 252 = 63,504 determinants; the ground state
and 3 excited states in the c = c^T (singlet) sector; SBCI1 with the paper's
thresholds.  One step = one complete solve of the 4 states.

Default arm: the CUDA library (device-resident integrals, CUDA-event timing on
the library stream, L2 flushed between steps), plus an end-to-end number
through the C ABI with host buffers, a roofline entry for the dominant kernel
and the CPU oracle timed on the host cores.  ``--impl reference`` times the
oracle alone (bounded samples).  Under torchrun every rank runs independent
solves (replicas); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FCI solves/sec (H10 STO-3G 1.2 A, 4 singlet-sector states, SBCI1)"
WORKLOAD = "h10_sto3g_1.2A_4states_singlet"
NSTATES = 4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--prec", default="tf32x3", choices=["fp64", "fp32", "tf32x3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ncu", action="store_true",
                    help="one solve, no warm-up and no extra legs (for an ncu launch list)")
    ap.add_argument("--sigma-only", default=None, choices=["h10", "h12", "n14", "n16"],
                    help="only run sigma products of one workload (for ncu captures)")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--serving", action="store_true",
                    help="serving stream: batched mixed precision vs sequential FP64, p50/p99")
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--batch", type=int, default=16,
                    help="H10 solves per step, solved together by the batched persistent kernels "
                         "(1: one solve per step through its own graph loop)")
    ap.add_argument("--slots", type=int, default=16)
    ap.add_argument("--davidson", action="store_true",
                    help="SBCI1 vs block Davidson-Liu on the same FP64 sigma: time, H-products, memory")
    return ap.parse_args()


def workload():
    from paper_2603_06101_gb300 import inputs

    return inputs.h_chain(10, 1.2)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            with open(self.path) as f:
                for row in csv.reader(f):
                    if len(row) < 9:
                        continue
                    try:
                        sm.append(float(row[1]))
                        smax.append(float(row[2]))
                    except ValueError:
                        continue
                    for nm, v in zip(names, row[5:9]):
                        if "Active" in v and "Not" not in v:
                            reasons.add(nm)
            os.unlink(self.path)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def source_sha(*rel):
    h = hashlib.sha256()
    for r in rel:
        with open(os.path.join(ROOT, r), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_for(kernel: str):
    """DRAM bytes per launch from a committed ncu summary, if the kernel source
    is unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get(kernel)
    if not e:
        return None
    if e.get("source_sha") != source_sha(*e["sources"]):
        return None
    return e.get("dram_bytes_per_launch_full")


# ----------------------------------------------------------------------------
def oracle_solve_time(I, nstates, max_steps=None):
    """Times the oracle's SBCI1 on the workload; returns (seconds, steps, done)."""
    from oracle import sbci as osb
    from oracle import sigma as osg
    from oracle import slater_condon as osc

    sig = osg.StringSigma(I.h1, I.eri, I.nalpha, I.nbeta)
    D = osc.diagonal_by_occupation(I.h1, I.eri, I.nalpha, I.nbeta)

    class Capped(osb.SBCI1):
        steps = 0

        def H(self, v):
            if max_steps is not None and self.n_sigma >= max_steps:
                raise StopIteration
            return super().H(v)

    run = Capped(sig.apply, D, (sig.Na, sig.Nb), osb.SBCIParams(sector=1))
    t0 = time.perf_counter()
    done = True
    try:
        run.solve(nstates)
    except StopIteration:
        done = False
    return time.perf_counter() - t0, run.n_sigma, done


def max_over_ranks(x: float, dist=None, device: str = "cuda") -> float:
    """The largest of every rank's x (the job ends when its slowest rank does);
    x itself with one rank."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: float, seconds_max: float) -> float:
    """Units all ranks processed per second of the slowest rank (weak scaling:
    every rank runs the same independent replicas)."""
    return world * units_per_rank / seconds_max


def run_reference(args, rank, world):
    if rank != 0:
        return
    I = workload()
    # one untimed full solve fixes the number of H-products per solve
    t_full, nsig_full, _ = oracle_solve_time(I, NSTATES)
    sample = 12  # H-products per bounded sample (initial guess + first SB steps)
    for _ in range(args.warmup):
        oracle_solve_time(I, NSTATES, max_steps=sample)
    times = []
    for _ in range(args.steps):
        t, n, _ = oracle_solve_time(I, NSTATES, max_steps=sample)
        times.append(t / n)
    per_sigma = float(np.mean(times))
    value = 1.0 / (per_sigma * nsig_full)
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "norb": 10, "ndet": 63504, "states": NSTATES, "sector": "c=c^T"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": f"each step: the first {sample} H-products of the oracle SBCI1 solve "
                                   f"(time per H-product incl. its SB work), scaled by the "
                                   f"{nsig_full} H-products of one full oracle solve ({t_full:.1f} s)"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gb300(args, rank, world, local_rank):
    import torch

    from paper_2603_06101_gb300 import sbci

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

    I = workload()
    prec = {"fp64": sbci.SBCI_FP64, "fp32": sbci.SBCI_FP32, "tf32x3": sbci.SBCI_TF32X3}[args.prec]
    stream = torch.cuda.Stream()
    ctx = sbci.Context.from_integrals(I, stream=stream.cuda_stream)
    p = sbci.params(sector=1, prec=prec)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    B = max(1, args.batch) if args.prec == "tf32x3" else 1
    batch_ctx = [ctx] + [sbci.Context.from_integrals(I, stream=stream.cuda_stream) for _ in range(B - 1)]

    def one_solve():
        if B == 1:
            E, _, R, st = ctx.solve(NSTATES, p)
            return E, R, st
        E, R, st = sbci.solve_batch(batch_ctx, NSTATES, p)
        one_solve.launches += sbci.solve_batch.last_launches
        return E[0], R[:NSTATES], st

    one_solve.launches = 0

    for _ in range(max(args.warmup, 3)):
        E, R, st = one_solve()
    nsig = sum(r.n_sigma for r in R)
    # ---------------- timed region: device-resident, CUDA events on the library
    # stream, each solve's SB steps running in the library's CUDA-graph loop
    sampler = ClockSampler(local_rank)
    ctx.profile(False)  # reset the launch counters; graphs stay on
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    one_solve.launches = 0
    t_ms = 0.0
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)  # L2 flush: 256 MB > 129 MB L2
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        E, R, st = one_solve()
        e1.record(stream)
        e1.synchronize()
        t_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    stats = ctx.profile_read()
    launches = sum(v[0] for v in stats.values()) if B == 1 else one_solve.launches
    t_max = max_over_ranks(t_ms, dist)
    value = whole_job_rate(world, B * args.steps, t_max / 1000.0)
    # ---------------- one solve alone (latency), same event timing
    single = None
    if B > 1:
        ts = 0.0
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.solve(NSTATES, p)
            e1.record(stream)
            e1.synchronize()
            ts += e0.elapsed_time(e1)
        single = {"solves_per_s": args.steps / (ts / 1000.0), "ms_per_solve": ts / args.steps,
                  "engine": "one graph loop per solve"}
    # ---------------- kernel timing pass: the same solves with each step kernel
    # launched on its own and bracketed by CUDA events on the launching stream
    kt0 = torch.cuda.Event(enable_timing=True)
    kt1 = torch.cuda.Event(enable_timing=True)
    if B == 1:
        ctx.profile(True)
        kt0.record(stream)
        for _ in range(2):
            ctx.solve(NSTATES, p)
        kt1.record(stream)
        kt1.synchronize()
        kstats = ctx.profile_read()
        ctx.profile(False)
        kpass_ms = kt0.elapsed_time(kt1)
        units = 1
    else:
        sbci.batch_profile(True)
        t0 = time.perf_counter()
        sbci.solve_batch(batch_ctx, NSTATES, p)
        torch.cuda.synchronize()
        kpass_ms = (time.perf_counter() - t0) * 1000.0
        kstats = sbci.batch_profile_read()
        sbci.batch_profile(False)
        units = B  # every batched launch serves the B solves (same Hamiltonian: they halt together)
    # ---------------- roofline of the dominant kernel
    pk, pk_kind = peaks()
    dom = max(kstats.items(), key=lambda kv: kv[1][1])
    name, (nl, ms) = dom
    npair, ndet = ctx.npair, ctx.ndet
    avg_s = ms / 1000.0 / max(nl, 1)
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    flops = 2.0 * npair * npair * ndet * units
    base = name[len("batch_"):] if name.startswith("batch_") else name
    base = {"update": "sb_update", "project": "sb_project", "scatter": "sigma_scatter"}.get(base, base)
    if base == "gather_contract_tc" or base == "sigma_gather_contract_tc":
        # two ceilings: the contraction on the tensor pipe and the HBM traffic the
        # kernel must move (G written, 4 B per pair, and the FP32 z read, 4 B, per
        # determinant); the larger ideal time is the binding one
        tpeak = pk.get("bf16_tflops", 1900.0) * 0.5  # TF32 dense = half the BF16 rate (1.1 vs 2.25 PF)
        bytes_alg = float(4 * npair + 4) * ndet * units
        t_tensor = flops / (tpeak * 1e12)
        t_hbm = bytes_alg / (pk["hbm_gbs"] * 1e9)
        tensor = {"achieved": flops / avg_s / 1e12, "peak": tpeak, "unit": "TFLOP/s",
                  "frac": flops / avg_s / 1e12 / tpeak, "algorithmic_per_launch": flops,
                  "peak_kind": f"{pk_kind} bf16 x nominal TF32/BF16 ratio 0.5; algorithmic 2 npair^2 flops "
                               "per determinant (the 3-term split executes 3x)"}
        hbm = {"achieved": bytes_alg / avg_s / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
               "frac": bytes_alg / avg_s / 1e9 / pk["hbm_gbs"], "algorithmic_per_launch": bytes_alg,
               "peak_kind": pk_kind, "algorithmic_note": f"{4 * npair + 4} B per determinant (G write + z read)"}
        if t_hbm >= t_tensor:
            roof = {"bound": "hbm", **hbm, "other_ceiling": {"bound": "tensor", **tensor}}
        else:
            roof = {"bound": "tensor", **tensor, "other_ceiling": {"bound": "hbm", **hbm}}
    elif base == "sigma_gather_contract_os":
        # FP64 contraction by exact BF16 slices: the HBM traffic it must move (G
        # written in FP64, 8 B per pair, and c read, 8 B, per determinant) and the
        # tensor work it executes (34 slice products of 2 Kp Np flops, Kp = Np = 64)
        bytes_alg = float(8 * npair + 8) * ndet * units
        xflops = 34.0 * 2 * 64 * 64 * ndet * units
        tpeak = pk.get("bf16_tflops", 1900.0)
        hbm = {"achieved": bytes_alg / avg_s / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
               "frac": bytes_alg / avg_s / 1e9 / pk["hbm_gbs"], "algorithmic_per_launch": bytes_alg,
               "peak_kind": pk_kind, "algorithmic_note": f"{8 * npair + 8} B per determinant (FP64 G write + c read)"}
        tensor = {"achieved": xflops / avg_s / 1e12, "peak": tpeak, "unit": "TFLOP/s",
                  "frac": xflops / avg_s / 1e12 / tpeak, "algorithmic_per_launch": xflops,
                  "peak_kind": f"{pk_kind} bf16; executed slice products (34 of 2 x 64 x 64 flops per determinant)"}
        if bytes_alg / (pk["hbm_gbs"] * 1e9) >= xflops / (tpeak * 1e12):
            roof = {"bound": "hbm", **hbm, "other_ceiling": {"bound": "tensor", **tensor}}
        else:
            roof = {"bound": "tensor", **tensor, "other_ceiling": {"bound": "hbm", **hbm}}
    elif base == "sigma_gather_contract" and args.prec == "fp64":
        peak = 4.0 * 152 * sm_mhz * 1e6 / 1e12  # 2 FP64 FMA per clock per SM (1.25 TF/s at 2.07 GHz)
        roof = {"bound": "alu", "achieved": flops / avg_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                "peak_kind": "FP64: 152 SMs x 2 FMA/clk x 2 flop x median SM clock (the 1.25 TFLOP/s nominal)",
                "algorithmic_per_launch": flops}
    elif base == "sigma_gather_contract":
        peak = 2.0 * 152 * 128 * sm_mhz * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": flops / avg_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                "peak_kind": "FP32: 152 SMs x 128 lanes x 2 flop x median SM clock",
                "algorithmic_per_launch": flops}
    else:
        gsz = 8 if args.prec == "fp64" else 4
        per_det = {"sigma_scatter": npair * gsz + 8, "sb_update": 12 * 8, "sb_project": 4 * 8}.get(base, 16)
        bytes_alg = float(per_det) * ndet * units
        roof = {"bound": "hbm", "achieved": bytes_alg / avg_s / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "peak_kind": pk_kind, "algorithmic_per_launch": bytes_alg,
                "algorithmic_note": f"{per_det} B per determinant x {units} solves"}
    roof["kernel"] = name
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = traffic_for(name)
    roof["avg_launch_us"] = avg_s * 1e6
    roof["share_of_timing_pass"] = ms / max(kpass_ms, 1e-9)
    # ---------------- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        h1 = np.ascontiguousarray(I.h1)
        eri = np.ascontiguousarray(I.eri)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d2h = 0
        for _ in range(args.steps):
            cs = [sbci.Context(I.norb, I.nalpha, I.nbeta, h1, eri, I.e_core, stream=stream.cuda_stream)
                  for _ in range(B)]
            if B == 1:
                E2, V2, _, _ = cs[0].solve(NSTATES, p, want_vectors=True)
                d2h = E2.nbytes + V2.nbytes
            else:
                E2, _, _ = sbci.solve_batch(cs, NSTATES, p)
                d2h = E2.nbytes
            for c2 in cs:
                c2.close()
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, dist)
        e2e = {"value": whole_job_rate(world, B * args.steps, te), "unit": "solves/s",
               "h2d_bytes_per_step": int(B * (h1.nbytes + eri.nbytes)),
               "d2h_bytes_per_step": int(d2h)}
    # ---------------- CPU oracle on the host cores (rank 0, N = 1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_full, nsig_o, _ = oracle_solve_time(I, NSTATES)
        cpu = {"value": 1.0 / t_full, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one full oracle SBCI1 solve of the same workload ({nsig_o} H-products, "
                         f"{t_full:.1f} s, numpy/OpenBLAS on all host cores)"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "tf32x3": "tf32x3+f64"}[args.prec],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "norb": 10, "ndet": ndet, "states": NSTATES,
                       "solves_per_step": B, "engine": "batched persistent kernels, one graph loop" if B > 1
                       else "one graph loop per solve",
                       "sector": "c=c^T", "sigma_precision": args.prec, "l2": "flushed (256 MB write) between steps",
                       "parallelism": f"replicas x{world}", "sigma_per_solve": nsig,
                       "sigma_per_state": [int(r.n_sigma) for r in R],
                       "fp64_sigma_per_state": [int(r.n_sigma_fp64) for r in R],
                       "controller_us_per_step": sum(r.ctl_cycles for r in R) / max(nsig, 1) / (clocks.get("sm_mhz") or 2070.0),
                       "energies": [float(e) for e in E]},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "single_solve": single,
            "autotuner": sbci.batch_classes() if B > 1 else None,
            "launches_timed": {k: v[0] for k, v in stats.items() if v[0]},
            "kernels_timing_pass": {k: {"launches": v[0], "ms": v[1]} for k, v in kstats.items() if v[0]},
            "clocks": clocks, "wall_s_timed": wall,
        }
        print(json.dumps(line), flush=True)


def sigma_only(args):
    """A few sigma products of one workload: the small cases of the ncu captures."""
    import torch

    from paper_2603_06101_gb300 import inputs, sbci

    I = {"h10": lambda: inputs.h_chain(10, 1.2), "h12": lambda: inputs.h_chain(12, 1.2),
         "n14": lambda: inputs.random_df(14, 14), "n16": lambda: inputs.random_df(16, 16)}[args.sigma_only]()
    ctx = sbci.Context.from_integrals(I)
    prec = {"fp64": sbci.SBCI_FP64, "fp32": sbci.SBCI_FP32, "tf32x3": sbci.SBCI_TF32X3}[args.prec]
    c = torch.from_numpy(inputs.random_vector(ctx.na, ctx.nb, 1)).cuda()
    out = torch.empty_like(c)
    for _ in range(args.reps):
        ctx.sigma(c, out, prec=prec)
    torch.cuda.synchronize()
    print(json.dumps({"sigma_only": args.sigma_only, "ndet": ctx.ndet, "reps": args.reps,
                      "norm": float(out.norm())}))


def run_ncu_solve(args):
    """One solve of the bench workload with nothing else (ncu launch lists)."""
    import torch

    from paper_2603_06101_gb300 import sbci

    I = workload()
    ctx = sbci.Context.from_integrals(I)
    prec = {"fp64": sbci.SBCI_FP64, "fp32": sbci.SBCI_FP32, "tf32x3": sbci.SBCI_TF32X3}[args.prec]
    p = sbci.params(sector=1, prec=prec)
    B = max(1, args.batch) if args.prec == "tf32x3" else 1
    if B == 1:
        E, _, R, st = ctx.solve(NSTATES, p)
    else:
        ctxs = [ctx] + [sbci.Context.from_integrals(I) for _ in range(B - 1)]
        EB, RB, st = sbci.solve_batch(ctxs, NSTATES, p)
        E, R = EB[0], RB[:NSTATES]
    torch.cuda.synchronize()
    print(json.dumps({"ncu_solve": WORKLOAD, "solves": B, "energies": [float(e) for e in E],
                      "sigma": sum(r.n_sigma for r in R)}))


def run_davidson(args):
    """The paper's comparison (Fig. 4, Tables S2-S19: time, steps and memory of
    SBCI vs the Davidson method) on the bench workload, one GPU: SBCI1 with FP64
    and with TF32x3 sigma and SBCI2 with FP64 sigma against block Davidson-Liu
    with FP64 sigma at two subspace limits.  Times are host wall-clock per solve (best of --reps after
    one warm-up solve); the vectors are the device buffers each solver holds."""
    import torch

    from paper_2603_06101_gb300 import sbci

    I = workload()
    ctx = sbci.Context.from_integrals(I)
    ndet = ctx.ndet
    k = NSTATES

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        best, out = None, None
        for _ in range(max(1, args.reps)):
            t0 = time.perf_counter()
            out = fn()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        return best, out

    rows = {}
    for name, prec in [("sbci1_fp64", sbci.SBCI_FP64), ("sbci1_tf32x3", sbci.SBCI_TF32X3)]:
        p = sbci.params(sector=1, prec=prec)
        dt, (E, _, R, st) = timed(lambda: ctx.solve(k, p))
        # x, X, y, Y, w, z[2], Z[2], the k stored states and the preconditioner:
        # 10 + k FP64 vectors, plus the FP32 copy of z in the split mode
        nb = (10 + k) * 8 * ndet + (4 * ndet if prec != sbci.SBCI_FP64 else 0)
        rows[name] = {"ms_per_solve": 1e3 * dt, "status": st, "energies": [float(e) for e in E],
                      "sigma_per_solve": int(sum(r.n_sigma for r in R)),
                      "fp64_sigma_per_solve": int(sum(r.n_sigma_fp64 for r in R)),
                      "steps": int(sum(r.n_step for r in R)), "vector_bytes": int(nb)}
    p2 = sbci.params(sector=1)
    dt, (E, _, R, st) = timed(lambda: ctx.solve_sbci2(k, p2))
    # SBCI1's vectors plus the pair's x, X, y, Y, z, Z (two each) and the k
    # start vectors with their H-images
    nb = (10 + k) * 8 * ndet + (12 + 2 * k) * 8 * ndet
    rows["sbci2_fp64"] = {"ms_per_solve": 1e3 * dt, "status": st, "energies": [float(e) for e in E],
                          "sigma_per_solve": int(sum(r.n_sigma for r in R)),
                          "steps": int(sum(r.n_step for r in R)), "vector_bytes": int(nb)}
    for ms in (0, 40):
        p = sbci.params(sector=1)
        dt, (E, _, R, st, nb) = timed(lambda: ctx.davidson(k, p, max_space=ms))
        rows[f"davidson_max_space_{ms or max(12, 4 * k)}"] = {
            "ms_per_solve": 1e3 * dt, "status": st, "energies": [float(e) for e in E],
            "sigma_per_solve": int(R[0].n_sigma), "iterations": int(R[0].n_step),
            "collapses": int(R[0].n_restart[0]), "vector_bytes": int(nb)}
    # kernel families of one solve each (launch counts and CUDA-event time)
    kernels = {}
    for name, fn in [("sbci1_fp64", lambda: ctx.solve(k, sbci.params(sector=1))),
                     ("davidson_max_space_16", lambda: ctx.davidson(k, sbci.params(sector=1)))]:
        ctx.profile(True)
        fn()
        torch.cuda.synchronize()
        kernels[name] = {f: {"launches": n, "ms": round(ms, 3)} for f, (n, ms) in ctx.profile_read().items() if n}
        ctx.profile(False)
    ref = np.sort(rows["sbci1_fp64"]["energies"])
    for r in rows.values():
        r["max_energy_diff_vs_sbci1_fp64"] = float(np.abs(np.sort(r["energies"]) - ref).max())
    print(json.dumps({"comparison": "SBCI1 and SBCI2 vs block Davidson-Liu (same FP64 sigma, same thresholds)",
                      "workload": WORKLOAD, "states": k, "ndet": int(ndet), "rows": rows,
                      "kernels_one_solve": kernels}))


def run_serving(args):
    """Serving stream over H6/H8/H10/H12 chains (1-4 states, spacing 0.7-3.0 A).

    1. saturation run of the batched mixed-precision server (all arrivals at
       t = 0) -> capacity;  2. Poisson arrivals at 0.7 x capacity through the
    server -> p50/p99 latency;  3. the same Poisson trace served by plain FP64
    one solve at a time (each solve alone, in arrival order) -> p50/p99 and
    solves/s.  Latency = completion - arrival.
    """
    import torch

    from paper_2603_06101_gb300 import inputs, sbci

    n = args.requests
    base = inputs.serving_trace(n, seed=4, rate_per_s=float("inf"))
    ints = [inputs.h_chain(r.natoms, r.spacing_angstrom) for r in base]
    ks = [r.nstates for r in base]
    # a seeded full-symmetry component in every start (start_noise): symmetric
    # chains would otherwise let rounding decide which symmetry a state search
    # explores, and the two precisions could meet different states
    p_mixed = sbci.params(prec=sbci.SBCI_TF32X3, start_noise=1e-2, noise_seed=2603)
    p_fp64 = sbci.params(prec=sbci.SBCI_FP64, start_noise=1e-2, noise_seed=2603)
    budget = 64 << 30

    def serve(arrivals, p, slots):
        server = sbci.Server(budget, slots)
        t0 = time.perf_counter()
        tickets, done, lat = {}, {}, {}
        serve.errors = {}
        order = np.argsort(arrivals, kind="stable")
        nxt = 0
        while len(done) < n:
            now = time.perf_counter() - t0
            while nxt < n and arrivals[order[nxt]] <= now:
                i = int(order[nxt])
                tickets[i] = server.submit(ints[i], ks[i], p)
                nxt += 1
            server.progress()
            for i, t in tickets.items():
                if i in done:
                    continue
                r = server.poll(t)
                if r is not None:
                    done[i] = r
                    if r[3] != 0:
                        serve.errors[i] = sbci.last_error()
                    lat[i] = (time.perf_counter() - t0) - arrivals[i]
        makespan = time.perf_counter() - t0
        server.close()
        return makespan, np.array([lat[i] for i in range(n)]), done

    # warm-up: one of each size through the server (graph builds, module loads)
    warm = sbci.Server(budget, 4)
    for sz in (6, 8, 10, 12):
        t = warm.submit(inputs.h_chain(sz, 1.0), 1, p_mixed)
        while warm.poll(t) is None:
            warm.progress()
    warm.close()
    torch.cuda.synchronize()
    sat_span, sat_lat, _ = serve(np.zeros(n), p_mixed, args.slots)
    capacity = n / sat_span
    rate = 0.7 * capacity
    gaps = np.random.default_rng(4).exponential(1.0 / rate, size=n)
    arrivals = np.cumsum(gaps) - gaps[0]
    span_m, lat_m, done_m = serve(arrivals, p_mixed, args.slots)
    errors_m = dict(serve.errors)
    # plain FP64, one solve per launch, in arrival order
    t0 = time.perf_counter()
    lat_f = np.zeros(n)
    E_f, st_f = {}, {}
    for i in np.argsort(arrivals, kind="stable"):
        while time.perf_counter() - t0 < arrivals[i]:
            pass
        ctx = sbci.Context.from_integrals(ints[i])
        E, _, _, st = ctx.solve(ks[i], p_fp64)
        ctx.close()
        E_f[int(i)] = E
        st_f[int(i)] = int(st)
        lat_f[i] = (time.perf_counter() - t0) - arrivals[i]
    span_f = time.perf_counter() - t0
    err = max(float(np.abs(np.sort(done_m[i][0]) - np.sort(E_f[i])).max()) for i in range(n))
    err0 = max(float(abs(done_m[i][0][0] - E_f[i][0])) for i in range(n))
    bad = [i for i in range(n) if np.abs(np.sort(done_m[i][0]) - np.sort(E_f[i])).max() > 1e-6]
    nbad = len(bad)
    details = [{"request": i, "natoms": base[i].natoms, "spacing": base[i].spacing_angstrom, "k": ks[i],
                "E_mixed": [float(e) for e in done_m[i][0]], "status_mixed": int(done_m[i][3]),
                "converged_mixed": [int(r.converged) for r in done_m[i][1]],
                "n_sigma_mixed": [int(r.n_sigma) for r in done_m[i][1]],
                "E_fp64": [float(e) for e in E_f[i]], "status_fp64": st_f[i],
                "error_mixed": errors_m.get(i)} for i in bad]
    line = {
        "serving": f"{n} requests, H6/H8/H10/H12 STO-3G, spacing U(0.7, 3.0) A, 1-4 states (seed 4)",
        "saturation_solves_per_s": capacity, "poisson_rate_per_s": rate,
        "batched_tf32x3": {"solves_per_s": n / span_m, "p50_s": float(np.percentile(lat_m, 50)),
                           "p99_s": float(np.percentile(lat_m, 99)), "slots": args.slots},
        "sequential_fp64": {"solves_per_s": n / span_f, "p50_s": float(np.percentile(lat_f, 50)),
                            "p99_s": float(np.percentile(lat_f, 99))},
        "max_energy_diff_mixed_vs_fp64_hartree": err, "max_ground_state_diff_hartree": err0,
        "requests_differing_by_more_than_1e-6": nbad, "differing": details,
        "sizes": {str(sz): int(sum(1 for r in base if r.natoms == sz)) for sz in (6, 8, 10, 12)},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.serving:
        run_serving(args)
        return
    if args.davidson:
        run_davidson(args)
        return
    if args.sigma_only:
        sigma_only(args)
        return
    if args.ncu:
        run_ncu_solve(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist

            dist.init_process_group("gloo")
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_gb300(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
