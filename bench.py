"""Benchmark of the Nyström–Schur preconditioner hot path on one GB300 (per rank).

Workload (default, --config 4): 3D 7-point anisotropic diffusion on a 128^3 grid
(n = 2,097,152), axis scales (1, 1, 1e-3), lognormal coefficient (sigma = 1.5, correlation
length 8 cells), 256 subdomains by recursive coordinate bisection, k = 128, p = 32 (block CG
with 160 right-hand sides), FP32 factors and inner solves / FP64 Nyström core and outer PCG,
outer PCG to a relative residual of 1e-8 with b = A x*, x* ~ N(0, 1). --config 1 runs the
64^3 lognormal workload (32 subdomains, k = 64, p = 16) the same way, --config 2 the
64-matrix batch.

One step = numeric rebuild of the preconditioner (device factorization of every interior
block and of A_G, sketch, inner block PCG, Nyström core, Z) + the outer PCG solve, with A's
values and b resident in device memory. The host symbolic analysis of A's pattern is done
once per pattern and reported separately (analyze_ms; with_analysis_ms in e2e includes it).
e2e repeats the step through the same public calls from pinned host buffers (values and b
in, x out).

Errors against the FP64 oracle are stated from tests/golden/<workload>.json (written by
tests/golden/make_golden.py, which calls only the oracle) with the same sketch and
right-hand side: the Nyström term Z Sigma Z^T and Sigma, the condition estimate of M2 S_Gamma
from the outer PCG's Lanczos coefficients, and the solution.

cpu_baseline / --impl reference time the FP64 CPU oracle (the program that defines
correctness) on a bounded sample of the same workload on this host, single-threaded: the
sparse factorization and the 160-column and single-column solves of a subset of the
interior blocks, scaled to all blocks and to the oracle's own iteration counts. The
interface (A_G) work of the oracle is not in the sample, so the value is a lower bound of
the oracle's build + solve time.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

# the oracle legs are reported single-threaded: keep BLAS to one thread (GPU work unaffected)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

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
    ap.add_argument("--config", type=int, default=4)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--variant", default="m2", choices=["m2", "m2_adef"],
                    help="preconditioner of the timed step (§4.3: M2 or M_2A-DEF)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--apply-reps", type=int, default=20)
    ap.add_argument("--variants", action="store_true",
                    help="also time q = 1, the S_I inner form, M3 and M_3A-DEF on the workload")
    ap.add_argument("--sample-blocks", type=int, default=64,
                    help="interior blocks in the oracle's timed CPU sample")
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


# DRAM bytes (read + write) of one interior-sweep launch (the scheduler the autotuner keeps)
# from an ncu capture of the bench workload (profiles/sweep_block_lognormal3d_64.md: the
# dependency-driven sweep at 64^3; profiles/sweep_bsm_lognormal3d_64.md: the column-sliced
# sweep at 128^3), keyed by (configuration, s, precision); absent until captured for the
# current kernel.
SWEEP_TRAFFIC = {(1, 80, "fp32"): 768.0e6, (4, 160, "fp32"): 11.87e9}


def sub_nnz(P):
    part = P.part
    coo = P.A.tocoo()
    pr, pc = part[coo.row], part[coo.col]
    # entries of A_IG, A_GI and A_G
    return int(((pr < 0) | (pc < 0)).sum())


# --------------------------------------------------------------------------- oracle arm
GOLDEN = os.path.join(ROOT, "tests", "golden")


def golden_for(P):
    path = os.path.join(GOLDEN, "%s.json" % P.name)
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def oracle_counts(P, G, b):
    """The oracle's own (it_inner, it_pcg) with sketch G: stored for the 128^3 workload,
    computed by one oracle run otherwise (returns the run's wall time too)."""
    gold = golden_for(P)
    if gold is not None:
        return (gold["build"]["it_inner"], gold["solve"]["it_pcg"]), None
    import oracle as O
    t0 = time.perf_counter()
    D = O.DBBD(P.A, P.part, P.nsub)
    M, info = O.build_m2(D, G, P.k, P.eps_inner)
    _, it_pcg, _ = O.solve(D, M.apply, b, rtol=P.rtol)
    return (info["it_inner"], it_pcg), time.perf_counter() - t0


def oracle_sample(P, counts, nsample):
    """Time the FP64 oracle (single thread) on a bounded sample of the workload: SuperLU
    factorization, one s-column solve and one single-column solve of `nsample` interior
    blocks spread over the subdomains. Scaled to all blocks and to the oracle's counts: the
    interior work of one build + solve is factorizing every block, 1 + it_inner s-column
    solves (the inner right-hand side and one S_Gamma apply per block-PCG iteration) and
    it_pcg + 2 single-column solves (f, one S_Gamma apply per outer iteration, x_I). The
    A_Gamma factorization and solves are left out: a lower bound of the oracle's time."""
    from oracle import nsp_oracle as NO
    A = P.A.tocsr()
    part = P.part
    blocks = np.unique(np.linspace(0, P.nsub - 1, min(nsample, P.nsub)).astype(int))
    rng = np.random.default_rng(0)
    t_fact = t_block = t_vec = 0.0
    t_start = time.perf_counter()
    for blk in blocks:
        idx = np.nonzero(part == blk)[0]
        Ab = A[idx][:, idx]
        t0 = time.perf_counter()
        lu = NO._lu(Ab)
        t_fact += time.perf_counter() - t0
        B = rng.standard_normal((len(idx), P.s))
        t0 = time.perf_counter()
        lu.solve(B)
        t_block += time.perf_counter() - t0
        v = np.ascontiguousarray(B[:, 0])
        t0 = time.perf_counter()
        lu.solve(v)
        t_vec += time.perf_counter() - t0
    sample_s = time.perf_counter() - t_start
    scale = P.nsub / len(blocks)
    it_inner, it_pcg = counts
    phases = {"factor_ms": 1e3 * scale * t_fact,
              "inner_solves_ms": 1e3 * scale * (1 + it_inner) * t_block,
              "outer_solves_ms": 1e3 * scale * (it_pcg + 2) * t_vec}
    total = sum(phases.values())
    desc = ("FP64 oracle (SciPy SuperLU, one thread) on %d of the %d interior blocks: "
            "factorization, one %d-column and one single-column solve each (%.1f s on this "
            "host), scaled to all blocks and to the oracle's counts it_inner=%d, it_pcg=%d; "
            "the A_Gamma work is not in the sample, so this is a lower bound of the oracle's "
            "build + solve" % (len(blocks), P.nsub, P.s, sample_s, it_inner, it_pcg))
    return total, phases, sample_s, desc


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args, P, G, b):
    world, rank, _ = dist_env()
    if rank != 0:
        return None
    counts, _ = oracle_counts(P, G, b)
    for _ in range(max(args.warmup, 0)):
        oracle_sample(P, counts, max(4, args.sample_blocks // 4))
    vals, samples = [], []
    for _ in range(args.steps):
        ms, phases, sample_s, desc = oracle_sample(P, counts, args.sample_blocks)
        vals.append(ms)
        samples.append(sample_s)
    ms = float(np.mean(vals))
    return {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(P, args),
            "timed_sample_s_per_step": float(np.mean(samples)),
            "cpu_baseline": {"value": ms, "unit": "ms", "cores": 1, "kind": "oracle",
                             "sample": desc, "phases": phases, "lower_bound": True},
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


WORKLOADS = {
    2: "aniso2d_batch: 64 independent 2D 5-point anisotropic problems, side U{100..400}, "
       "ratio log-U[1,1e3], 8-64 subdomains, k=32, p=8",
    4: "aniso3d_128: 3D 7-point anisotropic diffusion 128^3 (n=2097152), axis scales "
       "(1, 1, 1e-3), lognormal a (ell=8, sigma=1.5), 256 subdomains, k=128, p=32",
    1: "lognormal3d_64: 3D 7-point diffusion 64^3 (n=262144), lognormal a (ell=8, sigma=2), "
       "32 subdomains, k=64, p=16",
}


def workload_config(P, args):
    return {"workload": WORKLOADS.get(args.config, P.name),
            "n": int(P.n), "n_gamma": int(P.n_gamma), "subdomains": int(P.nsub),
            "k": int(P.k), "p": int(P.p), "eps_inner": P.eps_inner, "rtol": P.rtol,
            "precision": args.precision, "parallelism": "replicas%d" % args.gpus,
            "l2": "flushed (256 MiB write) between timed steps"}


# --------------------------------------------------------------------------- nsp arm
def time_events(stream, fn, reps):
    """Mean device time (ms) of fn() over reps calls, CUDA events on `stream`."""
    import torch
    fn()
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(reps):
        fn()
    a1.record(stream)
    torch.cuda.synchronize()
    return a0.elapsed_time(a1) / reps


def oracle_errors(N, torch, P, args, dev, b):
    """Build + solve with the stored oracle run's sketch and right-hand side; errors against
    the FP64 oracle (sampled rows of tests/golden/<workload>.json)."""
    gold = golden_for(P)
    if gold is None:
        return None
    G = F_make_sketch(P, args.config)
    x_star, _ = F_make_rhs(P, args.config)
    h = N.nsp_build(P.A, P.part, P.nsub, k=P.k, p=P.p, eps_inner=P.eps_inner,
                    precision=args.precision, sketch=G)
    bd = torch.tensor(b, dtype=torch.float64, device=dev)
    xd = torch.zeros_like(bd)
    inf = h.solve(bd, xd, rtol=P.rtol, maxit=500)
    x = xd.cpu().numpy()
    Z, S = h.get_basis()
    h.destroy()

    def sampled(full, block, rows):
        full = np.asarray(full, dtype=np.float64).reshape(full.shape[0], -1)
        ref = np.asarray(block["values"], dtype=np.float64)
        scale = np.asarray(block["colmax"], dtype=np.float64)
        return float((np.abs(full[rows] - ref).max(axis=0) / scale).max())

    import fixtures as F
    V = F.make_probe(gold["n_gamma"], 4, args.config, 2)
    g = gold["build"]
    r = min(len(S), len(g["sigma"]))
    xs = gold["solve"]
    return {
        "reference": "FP64 oracle, same sketch and right-hand side (tests/golden/%s.json, "
                     "%d sampled rows per output)" % (P.name, gold["nsample"]),
        "it_inner": [int(inf["it_inner"]), int(g["it_inner"])],
        "it_pcg": [int(inf["it_pcg"]), int(xs["it_pcg"])],
        "nystrom_term_err": sampled((Z * S) @ (Z.T @ V), g["nystrom_term"], gold["rows_gamma"]),
        "sigma_rel_err": float(np.max(np.abs(S[:r] - np.asarray(g["sigma"][:r]))
                                      / np.asarray(g["sigma"][:r]))),
        "kappa": [float(inf["kappa_est"]), float(xs["kappa"])],
        "kappa_rel_err": abs(inf["kappa_est"] - xs["kappa"]) / xs["kappa"],
        "solution_err": sampled(x, xs["x"], gold["rows_full"]),
        "x_err_vs_xstar": [float(np.linalg.norm(x - x_star) / np.linalg.norm(x_star)),
                           float(xs["err_vs_xstar"])],
        "final_residual": [float(np.linalg.norm(b - P.A @ x) / np.linalg.norm(b)),
                           float(xs["residual"])],
    }


def F_make_sketch(P, config):
    import fixtures as F
    return F.make_sketch(P.n_gamma, P.s, config, 0)


def F_make_rhs(P, config):
    import fixtures as F
    return F.make_rhs(P, config, 0)


def main():
    args = parse()
    world, rank, local = dist_env()
    import fixtures as F
    if args.config == 2 and args.impl != "reference":
        return main_batched(args, F, world, rank, local)
    P = F.make_problem(args.config, 0)
    G = F.make_sketch(P.n_gamma, P.s, args.config, 0)
    _, b = F.make_rhs(P, args.config, 0)

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
    apply_ms = time_events(stream, lambda: h.schur_apply(X, Y), args.apply_reps)
    nbytes = schur_apply_bytes(info0, s, wbytes, sub_nnz(P))
    hbm, peak_kind = peaks()
    achieved = nbytes / (apply_ms * 1e-3) / 1e9
    flops = 4.0 * info0["nnz_L_interior"] * s
    # dominant kernel of the apply: the interior sweep A_I^{-1} (n_I x s), alone
    Bi = torch.randn(info0["n_interior"], s, dtype=dt, device=dev)
    Xi = torch.empty_like(Bi)
    sweep_ms = time_events(stream, lambda: h.factor_solve(0, Bi, Xi), args.apply_reps)
    sweep_bytes = sweep_algorithmic_bytes(info0, s, wbytes)
    sweep_gbs = sweep_bytes / (sweep_ms * 1e-3) / 1e9
    del Bi, Xi
    # the block-CG Gram X^T Y (n_Gamma x s, FP32) on the tensor cores, alone
    gram = None
    if args.precision == "fp32":
        Yg = torch.randn(P.n_gamma, s, dtype=torch.float32, device=dev)
        Cg = torch.empty(s, s, dtype=torch.float64, device=dev)
        nbw = N.lib().nsp_gram_work_bytes(P.n_gamma, s, s)
        Wg = torch.empty(nbw, dtype=torch.uint8, device=dev)
        g_ms = time_events(stream, lambda: N.lib().nsp_gram(
            X.data_ptr(), Yg.data_ptr(), P.n_gamma, s, s, Cg.data_ptr(), Wg.data_ptr(),
            stream.cuda_stream), args.apply_reps)
        gbytes = 2 * P.n_gamma * s * 4
        gram = {"ms": g_ms, "GBps": gbytes / (g_ms * 1e-3) / 1e9,
                "frac_hbm": gbytes / (g_ms * 1e-3) / 1e9 / hbm,
                "tflops": 2.0 * P.n_gamma * s * s / (g_ms * 1e-3) / 1e12,
                "what": "X^T Y, n_Gamma x %d FP32, tcgen05 3xTF32 (three MMAs per product)" % s}
        del Yg, Cg, Wg

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
    h.destroy()

    errors = oracle_errors(N, torch, P, args, dev, b)

    # ---- other forms of the step on the same workload, device-timed like the step
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def time_variant(steps=2, **kw):
        kw.setdefault("precision", args.precision)
        h3 = N.nsp_build(P.A, P.part, P.nsub, k=P.k, p=P.p, eps_inner=P.eps_inner,
                         seed=seed, **kw)

        def step3():
            h3.rebuild(val_d, on_device=True)
            return h3.solve(b_d, x_d, rtol=P.rtol, maxit=500)

        step3()
        torch.cuda.synchronize()
        v_ms, v_infos = [], []
        for i in range(steps):
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
                    it_inner_gamma=last["it_inner_gamma"],
                    phase_ms={"factor": last["ms_factor"], "inner": last["ms_inner"],
                              "core": last["ms_core"], "solve": last["ms_solve"]})

    variant_line = time_variant(variant="m2_adef" if args.variant == "m2" else "m2")
    # the recursive treatment of A_Gamma: A_Gamma split into 64 blocks by coordinate
    # bisection of the interface nodes, its Schur solve M2' of rank 32 (16 oversampling)
    recursive_line = None
    if args.variant == "m2":
        g_idx = P.gamma
        part2 = F.interface_partition(P.A[g_idx][:, g_idx], P.coords[g_idx], 64)
        recursive_line = time_variant(variant="m2", gamma_part=part2, gamma_nblocks=64,
                                      gamma_k=32, gamma_p=16, gamma_eps_inner=P.eps_inner)
        recursive_line.pop("gamma_part")
        recursive_line["n_gamma2"] = int((part2 < 0).sum())
    # the plain FP64 GPU form (FP64 factors, inner block PCG and sweeps) of the timed step
    fp64_line = time_variant(variant=args.variant, precision="fp64")
    extra = {}
    if args.variants:
        extra["power_q1"] = time_variant(variant=args.variant, q=1)
        extra["inner_s_i"] = time_variant(variant=args.variant, inner_form="s_i")
        extra["variants_m3"] = [time_variant(variant=v) for v in ("m3", "m3_adef")]

    # ---- the 64^3 workload beside the 128^3 one (same step, fewer and smaller blocks)
    second = None
    if args.config == 4:
        P1 = F.make_problem(1, 0)
        _, b1 = F.make_rhs(P1, 1, 0)
        v1 = torch.tensor(P1.A.data, dtype=torch.float64, device=dev)
        b1d = torch.tensor(b1, dtype=torch.float64, device=dev)
        x1d = torch.zeros_like(b1d)
        h1 = N.nsp_build(P1.A, P1.part, P1.nsub, k=P1.k, p=P1.p, eps_inner=P1.eps_inner,
                         precision=args.precision, seed=seed)
        i1 = h1.info()

        def step1():
            h1.rebuild(v1, on_device=True)
            return h1.solve(b1d, x1d, rtol=P1.rtol, maxit=500)

        for _ in range(2):
            step1()
        torch.cuda.synchronize()
        t1 = []
        for i in range(3):
            flush.fill_(float(i))
            a0.record(stream)
            l1 = step1()
            a1.record(stream)
            torch.cuda.synchronize()
            t1.append(a0.elapsed_time(a1))
        B1 = torch.randn(i1["n_interior"], P1.s, dtype=dt, device=dev)
        X1 = torch.empty_like(B1)
        sw1 = time_events(stream, lambda: h1.factor_solve(0, B1, X1), args.apply_reps)
        sb1 = sweep_algorithmic_bytes(i1, P1.s, wbytes)
        second = {"workload": WORKLOADS[1], "ms_per_step": float(np.mean(t1)),
                  "it_inner": l1["it_inner"], "it_pcg": l1["it_pcg"],
                  "final_residual": float(np.linalg.norm(b1 - P1.A @ x1d.cpu().numpy())
                                          / np.linalg.norm(b1)),
                  "phase_ms": {"factor": l1["ms_factor"], "inner": l1["ms_inner"],
                               "core": l1["ms_core"], "solve": l1["ms_solve"]},
                  "sweep_ms": sw1, "sweep_frac_hbm": sb1 / (sw1 * 1e-3) / 1e9 / hbm}
        h1.destroy()

    # ---- the batched workload (64 independent 2D problems in one batched handle, §8(a) A8)
    # beside it: 1 warm-up + 3 timed steps of the same batched step as `--config 2`
    batched = None
    if args.config == 4:
        specs = F.batched_problem_specs()
        probs = [F.problem_from_spec(sp) for sp in specs]
        bb = np.concatenate([F.make_rhs(Pm, 2, i)[1] for i, Pm in enumerate(probs)])
        vb_d = torch.tensor(np.concatenate([Pm.A.data for Pm in probs]), dtype=torch.float64,
                            device=dev)
        bb_d = torch.tensor(bb, dtype=torch.float64, device=dev)
        xb_d = torch.zeros_like(bb_d)
        hb = N.nsp_build_batched([(Pm.A, Pm.part, Pm.nsub) for Pm in probs], k=probs[0].k,
                                 p=probs[0].p, eps_inner=probs[0].eps_inner,
                                 precision=args.precision, seed=seed)

        def stepb():
            hb.rebuild(vb_d, on_device=True)
            return hb.solve_batched(bb_d, xb_d, rtol=probs[0].rtol, maxit=1000)

        stepb()
        torch.cuda.synchronize()
        tb = []
        for i in range(3):
            flush.fill_(float(i))
            a0.record(stream)
            lb = stepb()
            a1.record(stream)
            torch.cuda.synchronize()
            tb.append(a0.elapsed_time(a1))
        xb = xb_d.cpu().numpy()
        off = np.concatenate([[0], np.cumsum([Pm.n for Pm in probs])])
        resb = [float(np.linalg.norm(bb[off[i]:off[i + 1]] - Pm.A @ xb[off[i]:off[i + 1]])
                      / np.linalg.norm(bb[off[i]:off[i + 1]])) for i, Pm in enumerate(probs)]
        batched = {"workload": WORKLOADS[2], "matrices": len(probs),
                   "unknowns": int(off[-1]), "ms_per_step": float(np.mean(tb)),
                   "it_inner_range": [int(min(d["it_inner"] for d in lb)),
                                      int(max(d["it_inner"] for d in lb))],
                   "it_pcg_range": [int(min(d["it_pcg"] for d in lb)),
                                    int(max(d["it_pcg"] for d in lb))],
                   "final_residual_max": float(max(resb))}
        hb.destroy()

    out = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            counts, full_s = oracle_counts(P, G, b)
            o_ms, phases, sample_s, desc = oracle_sample(P, counts, args.sample_blocks)
            cpu = {"value": o_ms, "unit": "ms", "cores": 1, "kind": "oracle", "sample": desc,
                   "phases": phases, "lower_bound": True, "sample_s": sample_s}
            gold = golden_for(P)
            if gold is not None:
                cpu["oracle_full_run_s_elsewhere"] = gold["oracle_seconds"]
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
                           kappa_est=last["kappa_est"],
                           nnz_L_interior=info0["nnz_L_interior"],
                           nnz_L_gamma=info0["nnz_L_gamma"],
                           step_ms_min=float(np.min(step_ms)),
                           step_ms_each=[round(float(t), 3) for t in step_ms],
                           phase_ms={"factor": last["ms_factor"], "inner": last["ms_inner"],
                                     "core": last["ms_core"], "solve": last["ms_solve"]}),
            "roofline": {"bound": "hbm", "achieved": sweep_gbs, "peak": hbm, "unit": "GB/s",
                         "frac": sweep_gbs / hbm, "traffic": SWEEP_TRAFFIC.get((args.config, s, args.precision)),
                         "kernel": "interior sweep (s=%d, %s): forward+backward supernodal "
                                   "sweep of every interior block, the dominant kernel of the "
                                   "S_Gamma block apply" % (s, args.precision),
                         "launch_ms": sweep_ms, "algorithmic_bytes": sweep_bytes,
                         "peak_kind": peak_kind,
                         "flops": flops, "tflops": flops / (sweep_ms * 1e-3) / 1e12},
            "schur_apply": {"achieved": achieved, "unit": "GB/s", "frac": achieved / hbm,
                            "apply_ms": apply_ms, "algorithmic_bytes": nbytes,
                            "what": "S_Gamma X: A_IG SpMM + interior sweep + A_G/A_GI SpMM "
                                    "(s=%d, %s)" % (s, args.precision)},
            "gram": gram,
            "errors_vs_oracle": errors,
            "other_variant": variant_line,
            "gamma_recursive": recursive_line,
            "plain_fp64": fp64_line,
            "second_workload": second,
            "batched_workload": batched,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(8 * (P.A.nnz + P.n)),
                    "d2h_bytes_per_step": int(8 * P.n),
                    "with_analysis_ms": full_ms},
            "gpu_launches": int(launches),
            "clocks": clocks.summary(),
        }
        out.update(extra)
        print(json.dumps(out))
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
            # the oracle's full build + solve on the first matrices for a bounded time (a
            # timed run, one thread), scaled by unknowns
            import oracle as O
            t_start = time.perf_counter()
            done_s, done_n = 0.0, 0
            for m, Pm in enumerate(probs):
                if time.perf_counter() - t_start > 20.0:
                    break
                Gm = F.make_sketch(Pm.n_gamma, Pm.s, 2, m)
                t0 = time.perf_counter()
                D = O.DBBD(Pm.A, Pm.part, Pm.nsub)
                M, _ = O.build_m2(D, Gm, Pm.k, Pm.eps_inner)
                O.solve(D, M.apply, bs[m], rtol=Pm.rtol)
                done_s += time.perf_counter() - t0
                done_n += Pm.n
            cpu = {"value": 1e3 * done_s * n_tot / done_n, "unit": "ms", "cores": 1,
                   "kind": "oracle",
                   "sample": "FP64 oracle build + solve of the first matrices for ~20 s "
                             "(%d unknowns, one thread), scaled to the batch's %d unknowns"
                             % (done_n, n_tot)}
        last = infos[-1]
        its = [i["it_pcg"] for i in last]
        out = {
            "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[2],
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
