"""Benchmark of the GB300 SBCI library.

Headline workload: linear H10 chain, STO-3G, Loewdin basis, 1.2 A spacing, 10
orbitals, 5 alpha / 5 beta electrons, 252 x 252 = 63,504 determinants; the
ground state and 3 excited states in the c = c^T (singlet) sector; SBCI1 with
the paper's thresholds, TF32x3 sigma with FP64 refinement.  One step = 16
such solves through the batched engine, each solve's context on its own CUDA
stream (CUDA-event timing around the call, L2 flushed between steps).

Legs of the default line (rank 0, one GPU): an end-to-end number through the
C ABI with host buffers (each step creates its 16 contexts from the host
integrals with sbci_init_integrals_many, solves them and destroys them); per-step latency percentiles; the same workload one
solve per launch, mixed and plain FP64; the roofline of the dominant kernel
(16 B per determinant per sigma, 2 npair^2 flops) and of every step kernel;
the per-state energy error against the oracle's exact sector energies
(tests/golden); a short serving stream (H6-H12, batched mixed precision
against FP64 one solve per launch, p50/p99); random density-fitted n = 14
(TF32x3, BF16x3 and FP64 sigma with rooflines, a 2-state mixed solve) and
n = 16 (BF16x3 sigma); the CPU oracle timed on the host cores.
``--impl reference`` times the oracle alone (bounded samples).  Under
torchrun every rank runs independent solves (replicas); rank 0 prints one
JSON line.
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
    ap.add_argument("--prec", default="tf32x3", choices=["fp64", "fp32", "tf32x3", "bf16x3"])
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
    ap.add_argument("--serving-requests", type=int, default=24,
                    help="requests of the short serving stream in the default bench line")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-n14", action="store_true")
    ap.add_argument("--no-n16", action="store_true")
    ap.add_argument("--init-stage", type=int, default=0, choices=[0, 1],
                    help="sbci_params.init_stage of the mixed-precision solves: the initial guess's "
                         "H-products in the stage precision instead of FP64")
    ap.add_argument("--large-solve", action="store_true",
                    help="only the n = 16 random density-fitted space: one ground-state solve, BF16x3 stage "
                         "on the tensor cores with FP64 refinement")
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
        res = run.solve(nstates)
        oracle_solve_time.energies = [r.energy for r in res]
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


GOLDEN_H10 = os.path.join(ROOT, "tests", "golden", "h10_sector_energies.json")


def golden_energies():
    """Exact H10 sector energies (total, hartree) written by the committed
    oracle script tests/golden/make_sector_energies.py, or None."""
    if not os.path.exists(GOLDEN_H10):
        return None
    with open(GOLDEN_H10) as f:
        return np.array(json.load(f)["total"])


def energy_errors(E, ref):
    """Per-state |E - ref| of the sorted energies (None without a reference)."""
    if ref is None:
        return None
    return [float(x) for x in np.abs(np.sort(np.asarray(E)) - np.sort(ref))]


def percentiles(ms):
    ms = np.asarray(ms, dtype=float)
    return {"p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
            "samples": int(ms.size)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    I = workload()
    # one untimed full solve fixes the number of H-products per solve
    t_full, nsig_full, _ = oracle_solve_time(I, NSTATES)
    sample = 12  # H-products per bounded sample (initial guess + first SB steps)
    for _ in range(args.warmup):
        oracle_solve_time(I, NSTATES, max_steps=sample)
    times, per = [], []
    for _ in range(args.steps):
        t, n, _ = oracle_solve_time(I, NSTATES, max_steps=sample)
        times.append(t)
        per.append(t / n)
    per_sigma = float(np.mean(per))
    value = 1.0 / (per_sigma * nsig_full)
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        # measured wall time of one timed step (one bounded sample), not 1/value
        "ms_per_step": 1000.0 * float(np.mean(times)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "norb": 10, "ndet": 63504, "states": NSTATES, "sector": "c=c^T"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": f"each timed step: the first {sample} H-products of the oracle SBCI1 solve "
                                   f"with their SB work ({1000.0 * float(np.mean(times)):.0f} ms); solves/s = 1 / "
                                   f"(time per H-product x the {nsig_full} H-products of one full oracle "
                                   f"solve, measured untimed before the steps: {t_full:.1f} s)"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


TF32_OF_BF16 = 0.5  # nominal dense TF32 / BF16 tensor rate (1.1 vs 2.25 PFLOP/s)
SIGMA_FAMILIES = ("gather_contract_tc", "gather_contract_os", "gather_contract", "gather_contract_lr",
                  "gather_contract_bf16", "gather_contract_tc_lr", "scatter", "symfinish", "fused_column")


def family_of(name: str) -> str:
    base = name[len("batch_"):] if name.startswith("batch_") else name
    base = base[len("sigma_"):] if base.startswith("sigma_") else base
    return {"update": "sb_update", "project": "sb_project"}.get(base, base)


def roofline(name, launches, ms, dets_per_launch, npair, prec, pk, pk_kind, sm_mhz, alpha_avg=0.0):
    """Roofline entry of one kernel family from its CUDA-event time.

    Algorithmic counts of the measurement plan: one sigma moves 16 B per
    determinant (c read, sigma written, FP64) and does 2 npair^2 flops per
    determinant (packed pairs); one SB update sweep moves 96 B per determinant,
    the projection 16 + 8 alpha.  The D/G scratch a kernel writes or reads is
    not algorithmic: it is what the DRAM traffic figure shows on top."""
    fam = family_of(name)
    avg_s = ms / 1000.0 / max(launches, 1)
    flops = 2.0 * npair * npair * dets_per_launch
    hbm_peak = pk["hbm_gbs"]
    if fam in SIGMA_FAMILIES:
        bytes_alg = 16.0 * dets_per_launch
        hbm = {"bound": "hbm", "achieved": bytes_alg / avg_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
               "peak_kind": f"{pk_kind} copy bandwidth", "algorithmic_per_launch": bytes_alg,
               "algorithmic_note": f"16 B per determinant per sigma (c read + sigma written, FP64) x "
                                   f"{dets_per_launch} determinants"}
        hbm["frac"] = hbm["achieved"] / hbm_peak
        other = None
        if fam in ("gather_contract_tc", "fused_column", "gather_contract_os", "gather_contract_bf16",
                   "gather_contract_tc_lr"):
            tf32 = fam in ("gather_contract_tc", "fused_column", "gather_contract_tc_lr")
            tpeak = pk.get("bf16_tflops", 1900.0) * (TF32_OF_BF16 if tf32 else 1.0)
            note = ("TF32: measured bf16 x nominal TF32/BF16 ratio 0.5" if tf32
                    else "BF16 operands (BF16x3 split, or the exact slices of the FP64 contraction): measured bf16")
            anote = "2 npair^2 flops per determinant (the split precisions execute more)"
            if fam == "gather_contract_tc_lr":
                anote += "; the factored form executes 4 npair (r + 2) products' worth, r + 2 the factor's rank"
            other = {"bound": "tensor", "achieved": flops / avg_s / 1e12, "peak": tpeak, "unit": "TFLOP/s",
                     "peak_kind": f"{pk_kind} {note}", "algorithmic_per_launch": flops,
                     "algorithmic_note": anote}
        elif fam in ("gather_contract", "gather_contract_lr"):
            lanes = 2.0 if prec == "fp64" else 128.0
            peak = 2.0 * lanes * 152 * sm_mhz * 1e6 / 1e12
            other = {"bound": "alu", "achieved": flops / avg_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                     "peak_kind": f"{'FP64' if prec == 'fp64' else 'FP32'}: 152 SMs x {lanes:.0f} FMA/clk x 2 x "
                                  f"median SM clock", "algorithmic_per_launch": flops}
        if other:
            other["frac"] = other["achieved"] / other["peak"]
            hbm["other_ceiling"] = other
        roof = hbm
    else:
        per_det = {"sb_update": 96.0, "sb_project": 16.0 + 8.0 * alpha_avg}.get(fam, 16.0)
        bytes_alg = per_det * dets_per_launch
        roof = {"bound": "hbm", "achieved": bytes_alg / avg_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                "peak_kind": f"{pk_kind} copy bandwidth", "algorithmic_per_launch": bytes_alg,
                "algorithmic_note": f"{per_det:g} B per determinant x {dets_per_launch} determinants"}
        roof["frac"] = roof["achieved"] / hbm_peak
    roof["kernel"] = name
    roof["avg_launch_us"] = avg_s * 1e6
    roof["launches"] = int(launches)
    roof["traffic"] = traffic_for(name)
    return roof


def serving_leg(n, slots, quiet=True):
    """Serving stream over H6/H8/H10/H12 chains (1-4 states, spacing 0.7-3.0 A,
    seed 4): (1) saturation run of the batched mixed-precision server (every
    arrival at t = 0) -> capacity; (2) Poisson arrivals at 0.7 x capacity
    through the server -> p50/p99 latency; (3) the same Poisson trace served by
    plain FP64 SBCI1 one solve per launch, in arrival order -> p50/p99.
    Latency = completion - arrival."""
    import torch

    from paper_2603_06101_gb300 import inputs, sbci

    base = inputs.serving_trace(n, seed=4, rate_per_s=float("inf"))
    ints = [inputs.h_chain(r.natoms, r.spacing_angstrom) for r in base]
    ks = [r.nstates for r in base]
    # a seeded full-symmetry component in every start (start_noise): symmetric
    # chains would otherwise let rounding decide which symmetry a state search
    # explores, and the two precisions could meet different states
    p_mixed = sbci.params(prec=sbci.SBCI_TF32X3, start_noise=1e-2, noise_seed=2603)
    p_fp64 = sbci.params(prec=sbci.SBCI_FP64, start_noise=1e-2, noise_seed=2603)
    budget = 64 << 30

    def serve(arrivals, p):
        server = sbci.Server(budget, slots)
        t0 = time.perf_counter()
        tickets, done, lat = {}, {}, {}
        errors = {}
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
                        errors[i] = sbci.last_error()
                    lat[i] = (time.perf_counter() - t0) - arrivals[i]
        makespan = time.perf_counter() - t0
        server.close()
        return makespan, np.array([lat[i] for i in range(n)]), done, errors

    # warm-up: one of each size through the server (graph builds, module loads)
    warm = sbci.Server(budget, 4)
    for sz in (6, 8, 10, 12):
        t = warm.submit(inputs.h_chain(sz, 1.0), 1, p_mixed)
        while warm.poll(t) is None:
            warm.progress()
    warm.close()
    torch.cuda.synchronize()
    sat_span, _, _, _ = serve(np.zeros(n), p_mixed)
    capacity = n / sat_span
    rate = 0.7 * capacity
    gaps = np.random.default_rng(4).exponential(1.0 / rate, size=n)
    arrivals = np.cumsum(gaps) - gaps[0]
    span_m, lat_m, done_m, errors_m = serve(arrivals, p_mixed)
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
    diff = [float(np.abs(np.sort(done_m[i][0]) - np.sort(E_f[i])).max()) for i in range(n)]
    bad = [i for i in range(n) if diff[i] > 1e-6]
    out = {
        "requests": n, "trace": "H6/H8/H10/H12 STO-3G, spacing U(0.7, 3.0) A, 1-4 states, seed 4; "
                                "Poisson arrivals at 0.7 x the saturation capacity",
        "saturation_solves_per_s": capacity, "poisson_rate_per_s": rate,
        "batched_tf32x3": {"solves_per_s": n / span_m, "p50_s": float(np.percentile(lat_m, 50)),
                           "p99_s": float(np.percentile(lat_m, 99)), "slots": slots},
        "fp64_one_solve_per_launch": {"solves_per_s": n / span_f, "p50_s": float(np.percentile(lat_f, 50)),
                                      "p99_s": float(np.percentile(lat_f, 99))},
        "max_energy_diff_mixed_vs_fp64_hartree": float(max(diff)),
        "requests_differing_by_more_than_1e-6": len(bad),
        "sizes": {str(sz): int(sum(1 for r in base if r.natoms == sz)) for sz in (6, 8, 10, 12)},
    }
    if not quiet:
        out["differing"] = [{"request": i, "natoms": base[i].natoms, "spacing": base[i].spacing_angstrom,
                             "k": ks[i], "E_mixed": [float(e) for e in done_m[i][0]],
                             "status_mixed": int(done_m[i][3]), "E_fp64": [float(e) for e in E_f[i]],
                             "status_fp64": st_f[i], "error_mixed": errors_m.get(i)} for i in bad]
    return out


def _time_sigma(ctx, c, out, prec, pname, reps, pk, pk_kind, sm_mhz):
    """One warm-up and reps sigma calls, per-kernel CUDA-event times on the
    library stream; the roofline of the dominant kernel."""
    import torch

    ctx.sigma(c, out, prec=prec)  # warm-up (scratch allocation)
    torch.cuda.synchronize()
    ctx.profile(True)
    t0 = time.perf_counter()
    for _ in range(reps):
        ctx.sigma(c, out, prec=prec)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    st = ctx.profile_read()
    ctx.profile(False)
    st = {k: v for k, v in st.items() if v[0] and k.startswith("sigma_")}
    dom = max(st.items(), key=lambda kv: kv[1][1])
    return {"ms_per_sigma": sum(v[1] for v in st.values()) / reps, "wall_ms_per_sigma": 1e3 * wall / reps,
            "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in st.items()},
            "roofline": roofline(dom[0], dom[1][0], dom[1][1], ctx.ndet, ctx.npair, pname, pk, pk_kind, sm_mhz)}


def random_df_leg(pk, pk_kind, sm_mhz, reps=3):
    """Random density-fitted integrals, n = 14, 7 alpha / 7 beta (seed 14;
    11,778,624 determinants): one TF32x3 sigma (the full form, and the
    factored tensor-core contraction on a second context with
    SBCI_TC_LOWRANK=1), one BF16x3 and one FP64 sigma, timed per kernel
    with CUDA events on the library stream (roofline of each), then the
    2-state solve in mixed precision with FP64 refinement (solve time, FP64
    residual per state)."""
    import torch

    from paper_2603_06101_gb300 import inputs, sbci

    I = inputs.random_df(14, 14)
    ctx = sbci.Context.from_integrals(I)
    c = torch.from_numpy(inputs.random_vector(ctx.na, ctx.nb, 1)).cuda()
    out = torch.empty_like(c)
    res = {"workload": "random density-fitted integrals n=14, 7a/7b, seed 14", "ndet": ctx.ndet,
           "npair": ctx.npair}
    for tag, prec, pname in (("tf32x3", sbci.SBCI_TF32X3, "tf32x3"), ("bf16x3", sbci.SBCI_BF16X3, "bf16x3"),
                             ("fp64", sbci.SBCI_FP64, "fp64")):
        res[f"sigma_{tag}"] = _time_sigma(ctx, c, out, prec, pname, reps if prec != sbci.SBCI_FP64 else 1,
                                          pk, pk_kind, sm_mhz)
    p = sbci.params(prec=sbci.SBCI_TF32X3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    E, _, R, st = ctx.solve(2, p)
    torch.cuda.synchronize()
    res["solve_tf32x3_2_states"] = {
        "seconds": time.perf_counter() - t0, "status": int(st), "energies": [float(e) for e in E],
        "fp64_residual_per_state": [float(r.residual) for r in R],
        "converged": [int(r.converged) for r in R], "sigma_per_state": [int(r.n_sigma) for r in R],
        "fp64_sigma_per_state": [int(r.n_sigma_fp64) for r in R]}
    ctx.close()
    # the factored TF32x3 contraction on the same space, for comparison
    old = os.environ.get("SBCI_TC_LOWRANK")
    os.environ["SBCI_TC_LOWRANK"] = "1"
    try:
        fac = sbci.Context.from_integrals(I)
    finally:
        if old is None:
            del os.environ["SBCI_TC_LOWRANK"]
        else:
            os.environ["SBCI_TC_LOWRANK"] = old
    res["sigma_tf32x3_factored"] = _time_sigma(fac, c, out, sbci.SBCI_TF32X3, "tf32x3", reps, pk, pk_kind, sm_mhz)
    fac.close()
    return res


def random_df_n16_leg(pk, pk_kind, sm_mhz, reps=2):
    """The largest space: random density-fitted integrals, n = 16, 8 alpha / 8
    beta (seed 16; 165,636,900 determinants, 1.3 GB per FP64 vector): the
    BF16x3 sigma on the tensor cores, timed per kernel with CUDA events on the
    library stream, with its roofline (the TF32 operands do not fit shared
    memory at this size)."""
    import torch

    from paper_2603_06101_gb300 import inputs, sbci

    I = inputs.random_df(16, 16)
    ctx = sbci.Context.from_integrals(I)
    c = torch.from_numpy(inputs.random_vector(ctx.na, ctx.nb, 1)).cuda()
    out = torch.empty_like(c)
    ctx.sigma(c, out, prec=sbci.SBCI_BF16X3)  # warm-up (scratch allocation)
    torch.cuda.synchronize()
    ctx.profile(True)
    t0 = time.perf_counter()
    for _ in range(reps):
        ctx.sigma(c, out, prec=sbci.SBCI_BF16X3)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    st = {k: v for k, v in ctx.profile_read().items() if v[0] and k.startswith("sigma_")}
    ctx.profile(False)
    dom = max(st.items(), key=lambda kv: kv[1][1])
    res = {"workload": "random density-fitted integrals n=16, 8a/8b, seed 16", "ndet": ctx.ndet, "npair": ctx.npair,
           "sigma_bf16x3": {"ms_per_sigma": sum(v[1] for v in st.values()) / reps, "wall_ms_per_sigma": 1e3 * wall / reps,
                            "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in st.items()},
                            "roofline": roofline(dom[0], dom[1][0], dom[1][1], ctx.ndet, ctx.npair, "bf16x3", pk,
                                                 pk_kind, sm_mhz)}}
    del c, out
    ctx.close()
    torch.cuda.empty_cache()
    return res


def large_solve_leg(init_stage=0):
    """The single large solve of the n = 16 space (165,636,900 determinants):
    the ground state with the BF16x3 stage on the tensor cores, FP64 re-syncs
    and the FP64 verification to the paper's thresholds; wall time of the
    solve (context creation excluded), H-products by precision, the FP64
    residual and the GPU time per kernel family."""
    import torch

    from paper_2603_06101_gb300 import inputs, sbci

    I = inputs.random_df(16, 16)
    t0 = time.perf_counter()
    ctx = sbci.Context.from_integrals(I)
    t_ctx = time.perf_counter() - t0
    p = sbci.params(prec=sbci.SBCI_BF16X3, init_stage=init_stage)
    torch.cuda.synchronize()
    ctx.profile(True)
    t0 = time.perf_counter()
    E, _, R, st = ctx.solve(1, p)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    prof = {k: {"launches": v[0], "ms": v[1]} for k, v in ctx.profile_read().items() if v[0]}
    ctx.profile(False)
    res = {"workload": "random density-fitted integrals n=16, 8a/8b, seed 16", "ndet": ctx.ndet,
           "npair": ctx.npair, "context_seconds": t_ctx, "init_stage": init_stage,
           "solve_bf16x3_ground_state": {
               "seconds": wall, "status": int(st), "energy": float(E[0]), "converged": int(R[0].converged),
               "fp64_residual": float(R[0].residual), "r0": float(p.r0), "sigma": int(R[0].n_sigma),
               "fp64_sigma": int(R[0].n_sigma_fp64), "kernels": prof}}
    ctx.close()
    torch.cuda.empty_cache()
    return res


def run_gb300(args, rank, world, local_rank):
    import torch

    from paper_2603_06101_gb300 import sbci

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

    I = workload()
    prec = {"fp64": sbci.SBCI_FP64, "fp32": sbci.SBCI_FP32, "tf32x3": sbci.SBCI_TF32X3,
            "bf16x3": sbci.SBCI_BF16X3}[args.prec]
    stream = torch.cuda.Stream()
    ctx = sbci.Context.from_integrals(I, stream=stream.cuda_stream)
    p = sbci.params(sector=1, prec=prec, init_stage=args.init_stage)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    B = max(1, args.batch) if args.prec == "tf32x3" else 1  # (the batch engine takes TF32x3 solves)
    # one CUDA stream per solve: a solve's own work between batch rounds (its
    # initial guess, FP64 re-syncs and state transitions) then overlaps the
    # others'; the batch engine orders itself after each solve's stream
    streams = [stream] + [torch.cuda.Stream() for _ in range(B - 1)]
    batch_ctx = [ctx] + [sbci.Context.from_integrals(I, stream=streams[i].cuda_stream) for i in range(1, B)]
    ref_E = golden_energies()

    def one_solve():
        if B == 1:
            E, _, R, st = ctx.solve(NSTATES, p)
            return E, R, st
        E, R, st = sbci.solve_batch(batch_ctx, NSTATES, p)
        one_solve.launches += sbci.solve_batch.last_launches
        one_solve.all_E = E
        return E[0], R[:NSTATES], st

    one_solve.launches = 0
    one_solve.all_E = None

    def timed_solves(fn, steps):
        """CUDA-event time of each call on the library stream, L2 flushed before each."""
        out = []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)  # L2 flush: 256 MB > 129 MB L2
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        return out, r

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
    wall0 = time.perf_counter()
    step_ms, (E, R, st) = timed_solves(one_solve, args.steps)
    t_ms = float(sum(step_ms))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    stats = ctx.profile_read()
    launches = sum(v[0] for v in stats.values()) if B == 1 else one_solve.launches
    t_max = max_over_ranks(t_ms, dist)
    value = whole_job_rate(world, B * args.steps, t_max / 1000.0)
    all_E = one_solve.all_E if B > 1 else np.asarray([E])
    err_batch = None
    if ref_E is not None:
        err_batch = [max(energy_errors(Ei, ref_E)[s] for Ei in all_E) for s in range(NSTATES)]
    # ---------------- one solve per launch: the same workload with the mixed
    # sigma, and plain FP64 SBCI1 (latency per solve = its CUDA-event time)
    single = None
    fp64_arm = None
    if B > 1:
        ms1, (E1, _, R1, st1) = timed_solves(lambda: ctx.solve(NSTATES, p), args.steps)
        single = {"solves_per_s": len(ms1) / (sum(ms1) / 1000.0), "ms_per_solve": float(np.mean(ms1)),
                  "latency": percentiles(ms1), "engine": "one graph loop per solve", "sigma_precision": args.prec,
                  "energy_err_vs_oracle": energy_errors(E1, ref_E)}
    if args.prec != "fp64":
        p64 = sbci.params(sector=1, prec=sbci.SBCI_FP64)
        ctx.solve(NSTATES, p64)  # warm-up: the FP64 graph
        k64 = min(args.steps, 10)
        ms64, (E64, _, R64, st64) = timed_solves(lambda: ctx.solve(NSTATES, p64), k64)
        fp64_arm = {"solves_per_s": len(ms64) / (sum(ms64) / 1000.0), "ms_per_solve": float(np.mean(ms64)),
                    "latency": percentiles(ms64), "engine": "plain FP64 SBCI1, one graph loop per solve",
                    "status": int(st64), "sigma_per_solve": int(sum(r.n_sigma for r in R64)),
                    "energies": [float(e) for e in E64], "energy_err_vs_oracle": energy_errors(E64, ref_E)}
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
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    host_halted = kstats.pop("batch_host_halted", None)  # host time between rounds, not a kernel
    kst = {k: v for k, v in kstats.items() if v[0]}
    dom = max(kst.items(), key=lambda kv: kv[1][1])
    name, (nl, ms) = dom
    npair, ndet = ctx.npair, ctx.ndet
    alpha_avg = (NSTATES - 1) / 2.0
    roof = roofline(name, nl, ms, ndet * units, npair, args.prec, pk, pk_kind, sm_mhz, alpha_avg)
    roof["share_of_timing_pass"] = ms / max(kpass_ms, 1e-9)
    kernel_rooflines = {k: roofline(k, v[0], v[1], ndet * units, npair, args.prec, pk, pk_kind, sm_mhz, alpha_avg)
                        for k, v in kst.items() if family_of(k) not in ("end", "reduce", "dots", "lincomb")}
    # ---------------- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        h1 = np.ascontiguousarray(I.h1)
        eri = np.ascontiguousarray(I.eri)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d2h = 0
        for _ in range(args.steps):
            cs = sbci.Context.many(I.norb, I.nalpha, I.nbeta, h1, eri, I.e_core,
                                   streams=[streams[i].cuda_stream for i in range(B)])
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
    # ---------------- further workloads of the measurement plan (rank 0, N = 1)
    serving = None
    n14 = None
    n16 = None
    if rank == 0 and world == 1:
        if not args.no_serving:
            serving = serving_leg(args.serving_requests, args.slots)
        if not args.no_n14:
            n14 = random_df_leg(pk, pk_kind, sm_mhz)
        if not args.no_n16:
            n16 = random_df_n16_leg(pk, pk_kind, sm_mhz)
    # ---------------- CPU oracle on the host cores (rank 0, N = 1)
    cpu = None
    oracle_same_run = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_full, nsig_o, _ = oracle_solve_time(I, NSTATES)
        cpu = {"value": 1.0 / t_full, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one full oracle SBCI1 solve of the same workload ({nsig_o} H-products, "
                         f"{t_full:.1f} s, numpy/OpenBLAS on all host cores)"}
        oracle_same_run = energy_errors(E, np.asarray(oracle_solve_time.energies) + I.e_core)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "tf32x3": "tf32x3+f64", "bf16x3": "bf16x3+f64"}[args.prec],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "norb": 10, "ndet": ndet, "states": NSTATES,
                       "solves_per_step": B, "engine": "batched persistent kernels, one graph loop" if B > 1
                       else "one graph loop per solve",
                       "sector": "c=c^T", "sigma_precision": args.prec, "init_stage": args.init_stage,
                       "l2": "flushed (256 MB write) between steps",
                       "parallelism": f"replicas x{world}", "sigma_per_solve": nsig,
                       "sigma_per_state": [int(r.n_sigma) for r in R],
                       "fp64_sigma_per_state": [int(r.n_sigma_fp64) for r in R],
                       "controller_us_per_step": sum(r.ctl_cycles for r in R) / max(nsig, 1) / (clocks.get("sm_mhz") or 2070.0),
                       "energies": [float(e) for e in E]},
            "latency": percentiles(step_ms),
            "energy_err_vs_oracle": err_batch,
            "energy_err_vs_oracle_note": "per state, max over the step's solves, |E - E_exact| against the "
                                         "oracle's exact sector energies (tests/golden/h10_sector_energies.json)",
            "energy_err_vs_oracle_sbci1_same_run": oracle_same_run,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "single_solve": single, "fp64_one_solve_per_launch": fp64_arm,
            "serving": serving, "random_df_n14": n14, "random_df_n16": n16,
            "kernel_rooflines": kernel_rooflines,
            "autotuner": sbci.batch_classes() if B > 1 else None,
            "launches_timed": {k: v[0] for k, v in stats.items() if v[0]},
            "kernels_timing_pass": {k: {"launches": v[0], "ms": v[1]} for k, v in kstats.items() if v[0]},
            "host_between_rounds_timing_pass": ({"halted_solves": host_halted[0], "ms": host_halted[1],
                                                 "pass_ms": kpass_ms} if host_halted else None),
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
    prec = {"fp64": sbci.SBCI_FP64, "fp32": sbci.SBCI_FP32, "tf32x3": sbci.SBCI_TF32X3,
            "bf16x3": sbci.SBCI_BF16X3}[args.prec]
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
    prec = {"fp64": sbci.SBCI_FP64, "fp32": sbci.SBCI_FP32, "tf32x3": sbci.SBCI_TF32X3,
            "bf16x3": sbci.SBCI_BF16X3}[args.prec]
    p = sbci.params(sector=1, prec=prec, init_stage=args.init_stage)
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
    """The serving stream alone (``--serving``): ``--requests`` requests through
    the batched mixed-precision server against plain FP64 one solve per launch
    (see serving_leg), with the differing requests listed."""
    print(json.dumps({"serving": serving_leg(args.requests, args.slots, quiet=False)}), flush=True)


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
    if args.large_solve:
        print(json.dumps({"random_df_n16": large_solve_leg(args.init_stage)}), flush=True)
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
