"""Benchmark of the Nyström–Schur preconditioner hot path on one GB300 (per rank).

Workload (default): 3D 7-point heterogeneous diffusion on a 64^3 grid (n = 262,144),
lognormal coefficient (correlation length 8 cells, sigma = 2), 32 subdomains by recursive
coordinate bisection, k = 64, p = 16, FP32 inner solves / FP64 Nyström core and outer PCG,
outer PCG to a relative residual of 1e-8 with b = A x*, x* ~ N(0, 1).

One step = numeric rebuild of the preconditioner (device factorization of every interior
block and of A_G, sketch, inner block PCG, Nyström core, Z) + the outer PCG solve, with A's
values and b resident in device memory. The host symbolic analysis of A's pattern is done
once per pattern and reported separately (analyze_ms). e2e repeats the step through the same
public calls from pinned host buffers (values and b in, x out).

--impl reference times the FP64 CPU oracle (the program that defines correctness), on a
bounded sample per step, extrapolated to one full solve with the iteration counts the
oracle itself measures once.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solve time to 1e-8 rel. residual; Schur block-apply GB/s vs HBM peak"
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="nsp", choices=["nsp", "reference"])
    ap.add_argument("--config", type=int, default=1)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--variant", default="m2", choices=["m2", "m2_adef"],
                    help="preconditioner of the timed step (§4.3: M2 or M_2A-DEF)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--apply-reps", type=int, default=20)
    ap.add_argument("--profile", action="store_true",
                    help="one warm-up step, then one step inside the NVTX range 'timed_step' "
                         "and one S_Gamma block apply inside 'schur_apply'; no timing output")
    return ap.parse_args()


def max_over_ranks(value, pg, device):
    """The largest value over all ranks (a replicated job takes as long as its slowest rank)."""
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def schur_apply_bytes(info, s, wbytes, nnz_sub):
    """Algorithmic bytes of one S_Gamma block apply: L read by both sweeps, one round trip
    of the n_I x s interior block, X read and Y written, A_IG, A_GI, A_G read once."""
    return (2 * info["nnz_L_interior"] * wbytes + 2 * info["n_interior"] * s * wbytes
            + 2 * info["n_gamma"] * s * wbytes + nnz_sub * (wbytes + 4))


def sweep_algorithmic_bytes(info, s, wbytes):
    """Algorithmic bytes of one interior sweep X = A_I^{-1} B (n_I x s): the panels read by
    the forward and the backward pass, B read, X written, and one round trip of the n_I x s
    intermediate between the two passes."""
    return 2 * info["nnz_L_interior"] * wbytes + 4 * info["n_interior"] * s * wbytes


# DRAM bytes (read + write) of one interior-sweep launch from an ncu capture of the bench
# workload (profiles/sweep_block_lognormal3d_64.md), keyed by (configuration, s); absent
# until captured for the current kernel.
SWEEP_TRAFFIC = {(1, 80): 768.0e6}


def sub_nnz(P):
    part = P.part
    coo = P.A.tocoo()
    pr, pc = part[coo.row], part[coo.col]
    # entries of A_IG, A_GI and A_G
    return int(((pr < 0) | (pc < 0)).sum())


# --------------------------------------------------------------------------- oracle arm
def oracle_sample(P, G, b, counts=None):
    """Time the oracle on a bounded sample and extrapolate to one full solve.

    Sample: DBBD split + sparse factorizations, one block S_Gamma apply (s columns), one
    A_G solve with s columns, one single-vector S_Gamma apply and M2 apply. A full solve is
    factor + (1 + it_inner) block applies + it_inner A_G solves + it_pcg (apply + M2).
    """
    import oracle as O
    t0 = time.perf_counter()
    D = O.DBBD(P.A, P.part, P.nsub)
    t_fact = time.perf_counter() - t0
    t0 = time.perf_counter()
    D.apply_S_gamma(G)
    t_block = time.perf_counter() - t0
    t0 = time.perf_counter()
    D.solve_G(G)
    t_gsolve = time.perf_counter() - t0
    v = G[:, 0].copy()
    t0 = time.perf_counter()
    D.apply_S_gamma(v)
    D.solve_G(v)
    t_single = time.perf_counter() - t0
    if counts is None:
        M, info = O.build_m2(D, G, P.k, P.eps_inner)
        _, it_pcg, _ = O.solve(D, M.apply, b, rtol=P.rtol)
        counts = (info["it_inner"], it_pcg)
    it_inner, it_pcg = counts
    total = t_fact + (1 + it_inner) * t_block + it_inner * t_gsolve + it_pcg * t_single
    return total * 1e3, counts


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args, P, G, b):
    world, rank, _ = dist_env()
    if rank != 0:
        return None
    counts = None
    for _ in range(max(args.warmup, 0)):
        _, counts = oracle_sample(P, G, b, counts)
    if counts is None:
        _, counts = oracle_sample(P, G, b, None)
    times = []
    for _ in range(args.steps):
        ms, counts = oracle_sample(P, G, b, counts)
        times.append(ms)
    ms = float(np.mean(times))
    sample = ("per step: oracle DBBD + SuperLU factorizations, one %d-column S_Gamma apply, "
              "one A_G solve, one single-vector S_Gamma + M2 apply; extrapolated with the "
              "oracle's own counts it_inner=%d, it_pcg=%d" % (P.s, counts[0], counts[1]))
    return {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(P, args),
            "cpu_baseline": {"value": ms, "unit": "ms", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def workload_config(P, args):
    return {"workload": "lognormal3d_64: 3D 7-point diffusion 64^3 (n=262144), lognormal a "
                        "(ell=8, sigma=2), 32 subdomains, k=64, p=16" if args.config == 1
                        else P.name,
            "n": int(P.n), "n_gamma": int(P.n_gamma), "subdomains": int(P.nsub),
            "k": int(P.k), "p": int(P.p), "eps_inner": P.eps_inner, "rtol": P.rtol,
            "precision": args.precision, "parallelism": "replicas%d" % args.gpus,
            "l2": "flushed (256 MiB write) between timed steps"}


# --------------------------------------------------------------------------- nsp arm
def main():
    args = parse()
    world, rank, local = dist_env()
    import fixtures as F
    if args.config == 2 and args.impl != "reference":
        return main_batched(args, F, world, rank, local)
    P = F.make_problem(args.config, 0)
    G = F.make_sketch(P.n_gamma, P.s, args.config, rank)
    _, b = F.make_rhs(P, args.config, rank)

    if args.impl == "reference":
        if world > 1 and rank != 0:
            return
        out = run_reference(args, P, G, b)
        if out is not None:
            print(json.dumps(out))
        return

    import torch
    import paper_2101_12164_gb300 as N
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    # inputs resident in HBM
    val_d = torch.tensor(P.A.data, dtype=torch.float64, device=dev)
    b_d = torch.tensor(b, dtype=torch.float64, device=dev)
    x_d = torch.zeros_like(b_d)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    seed = 1000 + rank

    t0 = time.perf_counter()
    h = N.nsp_build(P.A, P.part, P.nsub, k=P.k, p=P.p, eps_inner=P.eps_inner,
                    precision=args.precision, seed=seed, variant=args.variant)
    torch.cuda.synchronize()
    build_first_ms = (time.perf_counter() - t0) * 1e3
    info0 = h.info()

    def step():
        h.rebuild(val_d, on_device=True)
        return h.solve(b_d, x_d, rtol=P.rtol, maxit=500)

    if args.profile:
        step()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed_step")
        step()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        X = torch.randn(P.n_gamma, P.s, device=dev,
                        dtype=torch.float32 if args.precision == "fp32" else torch.float64)
        Y = torch.empty_like(X)
        h.schur_apply(X, Y)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("schur_apply")
        h.schur_apply(X, Y)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        Bi = torch.randn(info0["n_interior"], P.s, device=dev, dtype=X.dtype)
        Xi = torch.empty_like(Bi)
        h.factor_solve(0, Bi, Xi)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("interior_sweep")
        h.factor_solve(0, Bi, Xi)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        h.destroy()
        return

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, device time by CUDA events on the launching stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    launches0 = N.nsp_kernel_launches()
    infos = []
    with ClockSampler(local) as clocks:
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            infos.append(step())
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    launches = N.nsp_kernel_launches() - launches0
    if pg:
        pg.barrier()
    step_ms = [a.elapsed_time(bb) for a, bb in ev]
    ms = max_over_ranks(float(np.mean(step_ms)), pg, dev)
    res = float(np.linalg.norm(b - P.A @ x_d.cpu().numpy()) / np.linalg.norm(b))

    # ---- Schur block apply (s = k + p columns, the handle's precision): live timing
    s = P.s
    dt = torch.float32 if args.precision == "fp32" else torch.float64
    wbytes = 4 if args.precision == "fp32" else 8
    X = torch.randn(P.n_gamma, s, dtype=dt, device=dev)
    Y = torch.empty_like(X)
    h.schur_apply(X, Y)
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(args.apply_reps):
        h.schur_apply(X, Y)
    a1.record(stream)
    torch.cuda.synchronize()
    apply_ms = a0.elapsed_time(a1) / args.apply_reps
    nbytes = schur_apply_bytes(info0, s, wbytes, sub_nnz(P))
    hbm, peak_kind = peaks()
    achieved = nbytes / (apply_ms * 1e-3) / 1e9
    flops = 4.0 * info0["nnz_L_interior"] * s
    # dominant kernel of the apply: the persistent interior sweep A_I^{-1} (n_I x s), alone
    Bi = torch.randn(info0["n_interior"], s, dtype=dt, device=dev)
    Xi = torch.empty_like(Bi)
    h.factor_solve(0, Bi, Xi)
    torch.cuda.synchronize()
    a0.record(stream)
    for _ in range(args.apply_reps):
        h.factor_solve(0, Bi, Xi)
    a1.record(stream)
    torch.cuda.synchronize()
    sweep_ms = a0.elapsed_time(a1) / args.apply_reps
    sweep_bytes = sweep_algorithmic_bytes(info0, s, wbytes)
    sweep_gbs = sweep_bytes / (sweep_ms * 1e-3) / 1e9

    # ---- e2e: same step through the public calls from pinned host buffers
    val_h = torch.tensor(P.A.data, dtype=torch.float64).pin_memory()
    b_h = torch.tensor(b, dtype=torch.float64).pin_memory()
    x_h = torch.zeros_like(b_h).pin_memory()
    e2e = []
    for i in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.rebuild(val_h, on_device=False)
        h.solve(b_h, x_h, rtol=P.rtol, maxit=500)
        torch.cuda.synchronize()
        e2e.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = float(np.mean(e2e))
    # full public path from a host CSR, analysis included
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2 = N.nsp_build(P.A, P.part, P.nsub, k=P.k, p=P.p, eps_inner=P.eps_inner,
                     precision=args.precision, seed=seed, variant=args.variant)
    h2.solve(b_h, x_h, rtol=P.rtol, maxit=500)
    torch.cuda.synchronize()
    full_ms = (time.perf_counter() - t0) * 1e3
    h2.destroy()

    # ---- the other preconditioners of §4.3 (M2 / M_2A-DEF, M3, M_3A-DEF), one power
    # iteration (§2.1 eq. (power)) and the S_I inner form (Algorithm 2 step 3 as printed) on
    # the same workload, device-timed like the step
    def time_variant(**kw):
        kw.setdefault("precision", args.precision)
        h3 = N.nsp_build(P.A, P.part, P.nsub, k=P.k, p=P.p, eps_inner=P.eps_inner,
                         seed=seed, **kw)

        def step3():
            h3.rebuild(val_d, on_device=True)
            return h3.solve(b_d, x_d, rtol=P.rtol, maxit=500)

        for _ in range(2):
            step3()
        torch.cuda.synchronize()
        v_ms, v_infos = [], []
        for i in range(args.steps):
            flush.fill_(float(i))
            a0.record(stream)
            v_infos.append(step3())
            a1.record(stream)
            torch.cuda.synchronize()
            v_ms.append(a0.elapsed_time(a1))
        v_res = float(np.linalg.norm(b - P.A @ x_d.cpu().numpy()) / np.linalg.norm(b))
        last = v_infos[-1]
        h3.destroy()
        return dict(kw, ms_per_step=float(np.mean(v_ms)), it_inner=last["it_inner"],
                    it_power=last["it_power"], it_pcg=last["it_pcg"], final_residual=v_res,
                    phase_ms={"factor": last["ms_factor"], "inner": last["ms_inner"],
                              "core": last["ms_core"], "solve": last["ms_solve"]})

    variant_line = time_variant(variant="m2_adef" if args.variant == "m2" else "m2")
    power_line = time_variant(variant=args.variant, q=1)
    si_line = time_variant(variant=args.variant, inner_form="s_i")
    m3_lines = [time_variant(variant=v) for v in ("m3", "m3_adef")]
    # the plain FP64 GPU form (FP64 factors, inner block PCG and sweeps) of the timed step
    fp64_line = time_variant(variant=args.variant, precision="fp64")

    out = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            t0 = time.perf_counter()
            o_ms, counts = oracle_sample(P, G, b, None)
            cpu = {"value": o_ms, "unit": "ms", "cores": cpu_cores(), "kind": "oracle",
                   "sample": "one oracle DBBD + SuperLU factorization, one %d-column "
                             "S_Gamma apply, one A_G solve, one single-vector S_Gamma + M2 "
                             "apply, extrapolated with the oracle's own iteration counts "
                             "(it_inner=%d, it_pcg=%d, from one full oracle run)"
                             % (s, counts[0], counts[1]),
                   "wall_s": time.perf_counter() - t0}
        last = infos[-1]
        out = {
            "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": dict(workload_config(P, args), variant=args.variant,
                           analyze_ms=info0["ms_analyze"], first_build_ms=build_first_ms,
                           it_inner=last["it_inner"], it_pcg=last["it_pcg"],
                           rank=last["rank"], final_residual=res,
                           nnz_L_interior=info0["nnz_L_interior"],
                           nnz_L_gamma=info0["nnz_L_gamma"],
                           step_ms_min=float(np.min(step_ms)),
                           phase_ms={"factor": last["ms_factor"], "inner": last["ms_inner"],
                                     "core": last["ms_core"], "solve": last["ms_solve"]}),
            "roofline": {"bound": "hbm", "achieved": sweep_gbs, "peak": hbm, "unit": "GB/s",
                         "frac": sweep_gbs / hbm, "traffic": SWEEP_TRAFFIC.get((args.config, s)),
                         "kernel": "k_sweep (s=%d, %s): persistent forward+backward supernodal "
                                   "sweep of every interior block, the dominant kernel of the "
                                   "S_Gamma block apply" % (s, args.precision),
                         "launch_ms": sweep_ms, "algorithmic_bytes": sweep_bytes,
                         "peak_kind": peak_kind,
                         "flops": flops, "tflops": flops / (sweep_ms * 1e-3) / 1e12},
            "schur_apply": {"achieved": achieved, "unit": "GB/s", "frac": achieved / hbm,
                            "apply_ms": apply_ms, "algorithmic_bytes": nbytes,
                            "what": "S_Gamma X: A_IG SpMM + interior sweep + A_G/A_GI SpMM "
                                    "(s=%d, %s)" % (s, args.precision)},
            "other_variant": variant_line,
            "power_q1": power_line,
            "inner_s_i": si_line,
            "variants_m3": m3_lines,
            "plain_fp64": fp64_line,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(8 * (P.A.nnz + P.n)),
                    "d2h_bytes_per_step": int(8 * P.n),
                    "with_analysis_ms": full_ms},
            "gpu_launches": int(launches),
            "clocks": clocks.summary(),
        }
        print(json.dumps(out))
    h.destroy()
    if pg:
        pg.barrier()
        pg.destroy_process_group()


# --------------------------------------------------------------------------- batched arm
def main_batched(args, F, world, rank, local):
    """64 independent anisotropic 2D problems in one batched handle (one step = rebuild of
    every matrix's preconditioner + the batched outer PCG of all systems)."""
    import torch
    import paper_2101_12164_gb300 as N
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    specs = F.batched_problem_specs()
    probs = [F.problem_from_spec(sp) for sp in specs]
    bs = [F.make_rhs(Pm, 2, i)[1] for i, Pm in enumerate(probs)]
    k, p = probs[0].k, probs[0].p
    vals = np.concatenate([Pm.A.data for Pm in probs])
    b = np.concatenate(bs)
    n_tot = int(sum(Pm.n for Pm in probs))
    val_d = torch.tensor(vals, dtype=torch.float64, device=dev)
    b_d = torch.tensor(b, dtype=torch.float64, device=dev)
    x_d = torch.zeros_like(b_d)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    mats = [(Pm.A, Pm.part, Pm.nsub) for Pm in probs]
    t0 = time.perf_counter()
    h = N.nsp_build_batched(mats, k=k, p=p, eps_inner=probs[0].eps_inner,
                            precision=args.precision, seed=1000 + rank)
    torch.cuda.synchronize()
    build_first_ms = (time.perf_counter() - t0) * 1e3
    info0 = h.info()
    rtol = probs[0].rtol

    def step():
        h.rebuild(val_d, on_device=True)
        return h.solve_batched(b_d, x_d, rtol=rtol, maxit=1000)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    launches0 = N.nsp_kernel_launches()
    infos = []
    with ClockSampler(local) as clocks:
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            infos.append(step())
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    launches = N.nsp_kernel_launches() - launches0
    step_ms = [a.elapsed_time(bb) for a, bb in ev]
    ms = float(np.mean(step_ms))
    x = x_d.cpu().numpy()
    off = np.concatenate([[0], np.cumsum([Pm.n for Pm in probs])])
    res = [float(np.linalg.norm(bs[m] - probs[m].A @ x[off[m]:off[m + 1]]) / np.linalg.norm(bs[m]))
           for m in range(len(probs))]
    # S_Gamma block apply of the whole batch (block diagonal), s = k + p columns
    s = k + p
    dt = torch.float32 if args.precision == "fp32" else torch.float64
    wbytes = 4 if args.precision == "fp32" else 8
    X = torch.randn(info0["n_gamma"], s, dtype=dt, device=dev)
    Y = torch.empty_like(X)
    h.schur_apply(X, Y)
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(args.apply_reps):
        h.schur_apply(X, Y)
    a1.record(stream)
    torch.cuda.synchronize()
    apply_ms = a0.elapsed_time(a1) / args.apply_reps
    nbytes = schur_apply_bytes(info0, s, wbytes, sum(sub_nnz(Pm) for Pm in probs))
    hbm, peak_kind = peaks()
    achieved = nbytes / (apply_ms * 1e-3) / 1e9
    # e2e from pinned host buffers
    val_h = torch.tensor(vals, dtype=torch.float64).pin_memory()
    b_h = torch.tensor(b, dtype=torch.float64).pin_memory()
    x_h = torch.zeros_like(b_h).pin_memory()
    e2e = []
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.rebuild(val_h, on_device=False)
        h.solve_batched(b_h, x_h, rtol=rtol, maxit=1000)
        torch.cuda.synchronize()
        e2e.append((time.perf_counter() - t0) * 1e3)
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            # oracle on the first matrices for a bounded time, scaled by unknowns
            t_start = time.perf_counter()
            done_ms, done_n = 0.0, 0
            for m, Pm in enumerate(probs):
                if time.perf_counter() - t_start > 20.0:
                    break
                Gm = F.make_sketch(Pm.n_gamma, Pm.s, 2, m)
                o_ms, _ = oracle_sample(Pm, Gm, bs[m], None)
                done_ms += o_ms
                done_n += Pm.n
            cpu = {"value": done_ms * n_tot / done_n, "unit": "ms", "cores": cpu_cores(),
                   "kind": "oracle",
                   "sample": "oracle (sample-extrapolated per matrix) on the first matrices "
                             "for ~20 s (%d unknowns), scaled to the batch's %d unknowns"
                             % (done_n, n_tot)}
        last = infos[-1]
        its = [i["it_pcg"] for i in last]
        out = {
            "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": "aniso2d_batch: 64 independent 2D 5-point anisotropic "
                                   "problems, side U{100..400}, ratio log-U[1,1e3], 8-64 "
                                   "subdomains, k=32, p=8",
                       "matrices": len(probs), "n_total": n_tot,
                       "n_gamma_total": int(info0["n_gamma"]),
                       "precision": args.precision, "parallelism": "replicas%d" % world,
                       "l2": "flushed (256 MiB write) between timed steps",
                       "first_build_ms": build_first_ms, "analyze_ms": info0["ms_analyze"],
                       "it_pcg_min": int(min(its)), "it_pcg_max": int(max(its)),
                       "it_inner_max": int(max(i["it_inner"] for i in last)),
                       "max_final_residual": float(max(res)),
                       "phase_ms": {"factor": last[0]["ms_factor"], "inner": last[0]["ms_inner"],
                                    "core": last[0]["ms_core"], "solve": last[0]["ms_solve"]}},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": None,
                         "kernel": "S_Gamma block apply of the batch (s=%d, %s)" % (s, args.precision),
                         "apply_ms": apply_ms, "algorithmic_bytes": nbytes,
                         "peak_kind": peak_kind},
            "cpu_baseline": cpu,
            "e2e": {"value": float(np.mean(e2e)), "unit": "ms",
                    "h2d_bytes_per_step": int(8 * (len(vals) + len(b))),
                    "d2h_bytes_per_step": int(8 * len(b))},
            "gpu_launches": int(launches),
            "clocks": clocks.summary(),
        }
        print(json.dumps(out))
    h.destroy()


if __name__ == "__main__":
    main()
