"""Benchmark: converged eigenpairs per second of warm-started ChFSI sequences on GB300.

The workload is the mixed-precision sequence: n = 9300, nev = 256, blk = 320, filter
degree 20, 20 correlated problems (generated like the n = 512 case: B = I + 0.1 G^H G/n,
planted spectrum, eigenvectors rotated between problems), first problem cold, the rest
warm-started from the previous eigenvectors.  One step is one problem of this sequence,
taken cyclically (the whole hot path: reduction, Lanczos bound, Chebyshev filter,
re-orthonormalisation, Rayleigh-Ritz, locking, back-transform); the problem after the last
one is the first again and starts cold, so K = 20 timed steps solve the whole sequence once
(one cold and 19 warm problems), whatever the warm-up.  Inputs are seeded synthetic
matrices resident in HBM (27.7 GB of A and B, larger than L2).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own independent sequence (different seed): the units
(eigenpairs) of all ranks are summed and divided by the slowest rank's time ("weak").
``--impl reference`` times the CPU oracle (NumPy/SciPy FP64) on the same workload, one
filter loop per step; only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "converged eigenpairs/s per sequence & filter % tensor peak vs plain FP64 @res≤1e-10"
UNIT = "eigenpairs/s"
WORKLOAD = "c3"
WORKLOAD_TEXT = {
    "c2": "n=2600 nev=100 blk=130 deg adaptive 8-25 cond(B)=1e4",
    "c3": "n=9300 nev=256 blk=320 deg=20 B=I+0.1G^HG/n",
    "c5": "n=13400 nev=1000 blk=1200 deg adaptive 4-40 B=I+0.1G^HG/n",
}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        # raw samples: CHFSI_CLOCKS_CSV (with {rank} replaced by the GPU index), else a temp file
        tmpl = os.environ.get("CHFSI_CLOCKS_CSV")
        self.path = (tmpl.replace("{rank}", str(gpu_index)) if tmpl else
                     os.path.join(tempfile.gettempdir(), f"chfsi_clocks_gpu{gpu_index}.csv"))

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            if getattr(self, "f", None) is not None:
                self.f.close()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def combine_ranks(ms: float, units: float, device="cpu"):
    """Whole-job figures over all ranks: the slowest rank's time and the units of all
    ranks (independent sequences per rank: weak scaling, no data-path collective)."""
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    c = torch.tensor([units], dtype=torch.float64, device=device)
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        import torch.distributed as dist

        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def step_schedule(first: int, count: int, N: int):
    """Problem index and cold flag of the steps first .. first + count - 1 of the cyclic
    sequence: step s solves problem s mod N, cold when that is the first problem."""
    return [(s % N, s % N == 0) for s in range(first, first + count)]


def segments(first: int, count: int, N: int):
    """The steps first .. first + count - 1 as runs of consecutive problems
    [(start problem, length, cold start)], split where the sequence starts over."""
    out = []
    s, left = first, count
    while left > 0:
        p = s % N
        ln = min(left, N - p)
        out.append((p, ln, p == 0))
        s += ln
        left -= ln
    return out


def summary(values) -> dict:
    """Percentiles of a list of non-negative errors (every eigenpair of the timed steps)."""
    v = np.asarray(values, dtype=np.float64).ravel()
    if v.size == 0:
        return {}
    return {"count": int(v.size), "p50": float(np.percentile(v, 50)), "p90": float(np.percentile(v, 90)),
            "p99": float(np.percentile(v, 99)), "max": float(v.max())}


def load_workload(device, rank: int, name: str = WORKLOAD, N=None, keep_vectors=False):
    from paper_1206_3768_gb300 import inputs

    return inputs.planted_sequence(name, device=device, keep_vectors=keep_vectors, seed_offset=rank, N=N)


def _workload_text(name, seq, N):
    text = WORKLOAD_TEXT[name] if name in WORKLOAD_TEXT else f"n={seq.n} nev={seq.nev} blk={seq.blk}"
    return (f"{name}: {text} N={N}, "
            "planted spectrum, first problem cold, rest warm; one step = one problem of the "
            "cyclic sequence (K = N steps cover it once)")


def run_reference(args):
    """The oracle on the host cores, on the same workload: one step is one filter loop of
    the oracle's Algorithm 1 (the first loop of a problem also does its reduction, Lanczos
    bound and start-up), the loops running through the sequence in order from problem 1,
    warm-started from the planted eigenpairs of problem 0 (the state a converged solve of
    problem 0 leaves; 19 of the 20 problems of a pass are warm), each later problem from
    the oracle's own previous result; the unit count is the pairs the timed loops locked."""
    import oracle.chfsi_oracle as O

    ws, rank, _ = _dist()
    if rank != 0:
        return
    k = max(1, args.steps)
    w = max(0, args.warmup)
    n_prob = args.ref_problems
    dev = "cuda" if torch.cuda.is_available() else "cpu"   # input generation only
    seq = load_workload(dev, 0, name=args.workload, N=n_prob, keep_vectors={0})
    As = [np.tril(p.A.cpu().numpy()) for p in seq.problems]
    Bs = [np.tril(p.B.cpu().numpy()) for p in seq.problems]
    p0 = seq.problems[0]
    warm0 = O.WarmState(X=p0.X[:, :seq.blk].cpu().numpy(), lam=np.array(p0.lam[:seq.blk]))
    del p0
    del seq.problems[:]
    if dev == "cuda":
        torch.cuda.empty_cache()
    cfg = __import__("paper_1206_3768_gb300.inputs", fromlist=["CONFIGS"]).CONFIGS[args.workload]

    def loops():
        warm = warm0
        ell = 1
        while True:
            gen = O.chfsi_solve_loops(As[ell], Bs[ell], cfg["nev"], cfg["blk"], cfg["tol"],
                                      deg=cfg["deg"], deg_min=cfg["deg_min"], deg_max=cfg["deg_max"],
                                      warm=warm)
            while True:
                try:
                    yield ell, next(gen)
                except StopIteration as done:
                    _, _, warm, _ = done.value
                    break
            ell += 1
            if ell == n_prob:
                raise RuntimeError("reference sample ran past its generated problems")

    it = loops()
    for _ in range(w):
        next(it)
    t0 = time.perf_counter()
    locked, problems = 0, set()
    for _ in range(k):
        ell, nl = next(it)
        locked += nl
        problems.add(ell)
    total = time.perf_counter() - t0
    value = locked / total
    cores = os.cpu_count()
    sample = (f"{k} filter loops of the oracle after {w} warm-up loops, over problems "
              f"{sorted(problems)} of the sequence (warm: problem 1 from the planted eigenpairs of "
              f"problem 0), {locked} pairs locked, {total:.1f} s")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": k, "warmup": w, "ms_per_step": 1e3 * total / k, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": _workload_text(args.workload, None, cfg["N"]).replace(
                       "one step = one problem of the cyclic sequence (K = N steps cover it once)",
                       "one step = one filter loop of the oracle"),
                   "sample_problems": sorted(problems)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_oracle_warm_problem(seq, ell: int, budget_s: float):
    """The oracle on problem ell of the sequence, warm-started from the planted eigenvectors
    and eigenvalues of problem ell - 1 (exact input data, the state a converged previous solve
    leaves), loop by loop until it finishes or the time budget is spent.  Returns (pairs
    locked, seconds, loops, finished, eigenvalues)."""
    import oracle.chfsi_oracle as O

    prev, cur = seq.problems[ell - 1], seq.problems[ell]
    A = np.tril(cur.A.cpu().numpy())
    B = np.tril(cur.B.cpu().numpy())
    warm = O.WarmState(X=prev.X[:, :seq.blk].cpu().numpy(), lam=np.array(prev.lam[:seq.blk]))
    t0 = time.perf_counter()
    gen = O.chfsi_solve_loops(A, B, seq.nev, seq.blk, seq.tol, deg=seq.deg, deg_min=seq.deg_min,
                              deg_max=seq.deg_max, warm=warm)
    locked, loops, lam = 0, 0, None
    while True:
        try:
            locked += next(gen)
            loops += 1
        except StopIteration as done:
            lam = done.value[0]
            return int(np.isfinite(lam).sum()), time.perf_counter() - t0, loops, True, lam
        if time.perf_counter() - t0 > budget_s:
            return locked, time.perf_counter() - t0, loops, False, None


def run_ours(args):
    from paper_1206_3768_gb300 import binding as cb

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    want_cpu = rank == 0 and ws == 1 and not args.no_cpu
    t_gen = time.perf_counter()
    seq = load_workload(dev, rank, name=args.workload, N=args.problems,
                        keep_vectors={0} if want_cpu else False)
    n, nev, blk, N = seq.n, seq.nev, seq.blk, len(seq.problems)
    # lower triangles, column-major; B is common to the whole sequence (one copy)
    B_low = cb.fortran(torch.tril(seq.problems[0].B))
    As, Bs = [], []
    for p in seq.problems:
        As.append(cb.fortran(torch.tril(p.A)))
        Bs.append(B_low)
        if not (want_cpu and p is seq.problems[1]):
            p.A = None
    lam_planted = [p.lam[:nev].copy() for p in seq.problems]
    lam_scale = [float(np.max(np.abs(p.lam))) for p in seq.problems]
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    stream = torch.cuda.current_stream(dev)
    W, K = args.warmup, args.steps
    deg = seq.deg

    def barrier():
        if ws > 1:
            import torch.distributed as dist

            dist.barrier()

    def run_arm(ctx, want_vectors):
        """W untimed then K timed steps on ctx; returns (ms, evals by problem, evecs by problem,
        stats of the timed steps in order)."""
        for p, cold in step_schedule(0, W, N):
            if cold:
                cb.chfsi_reset_warm_state(ctx)
            cb.chfsi_solve_next(ctx, As[p], Bs[p], nev, blk, deg, seq.tol, want_vectors=False)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        evals, evecs, stats = {}, {}, []
        e0.record(stream)
        for p, cold in step_schedule(W, K, N):
            if cold:
                cb.chfsi_reset_warm_state(ctx)
            ev, X, st = cb.chfsi_solve_next(ctx, As[p], Bs[p], nev, blk, deg, seq.tol,
                                            want_vectors=want_vectors)
            evals[p], evecs[p] = ev, X
            st["problem"] = p
            stats.append(st)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return e0.elapsed_time(e1), evals, evecs, stats

    solver = cb.Solver(n, blk, stream=stream, deg_min=seq.deg_min, deg_max=seq.deg_max)
    ctx = solver.ctx
    sampler = ClockSampler(local)
    sampler.start()
    ms, evals, evecs, all_stats = run_arm(ctx, want_vectors=True)
    clocks = sampler.stop()
    converged = sum(int(torch.isfinite(e).sum()) for e in [evals[p] for p, _ in step_schedule(W, K, N)])
    ms_max, units = combine_ranks(ms, converged, dev)
    value = units / (ms_max / 1e3)
    max_resid = max(s["max_resid"] for s in all_stats)
    launches = sum(s["launches"] for s in all_stats)

    # ---- roofline of the dominant kernel: the filter's product kernel
    peaks, peak_kind = _peaks()
    g_ms = sum(s["t_filter_gemm_ms"] for s in all_stats)
    t_flops = sum(s["tensor_flops"] for s in all_stats)
    fp64_equiv = 8.0 * n * n * sum(s["filter_matvecs"] for s in all_stats)
    # DRAM traffic per launch: one ncu capture of the kernel (profiles/oz_gemm_tc_traffic.json)
    # gives DRAM bytes / bytes of Hs digit slices streamed (the launch's minimum traffic); the
    # step's launches are scaled by the slice bytes they stream (counted by the library).
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "oz_gemm_tc_traffic.json")
    products = sum(s["filter_products"] for s in all_stats)
    if os.path.exists(tfile) and products > 0 and os.environ.get("CHFSI_OZ_KERNEL", "tc") != "mma":
        try:
            with open(tfile) as f:
                tj = json.load(f)
            if tj.get("current", True):
                traffic = float(tj["dram_bytes_over_slice_bytes"]) * sum(
                    s["filter_slice_bytes"] for s in all_stats) / products
        except (OSError, ValueError, KeyError):
            traffic = None
    if t_flops > 0:
        achieved = t_flops / (g_ms / 1e3) / 1e12
        peak = peaks["bf16_tflops_sustained"]
        kname = ("oz_gemm_tc_kernel (split-BF16 digit products, TMA + tcgen05.mma, FP32 "
                 "accumulators in tensor memory)" if os.environ.get("CHFSI_OZ_KERNEL", "tc") != "mma"
                 else "oz_gemm_kernel (split-BF16 digit products, mma.sync bf16 -> fp32)")
        roofline = {"bound": "tensor", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": traffic,
                    "fp64_equivalent_tflops": fp64_equiv / (g_ms / 1e3) / 1e12,
                    "launches": products,
                    "algorithmic_bytes_per_launch": (sum(s["filter_slice_bytes"] for s in all_stats)
                                                     / products) if products else None,
                    "peak_note": f"bf16 dense sustained ({peak_kind}); achieved counts the "
                                 "slice-pair products the kernel issues (Gauss form: three real "
                                 "products of 2 x pairs x n x m x n flops; real embedding: 2 x pairs "
                                 "x 2n x m x 2n; unpadded) over the product kernel's CUDA-event time"}
    else:
        fp64_peak = peaks["bf16_tflops_sustained"] * 1.25 / 2250.0
        achieved = fp64_equiv / (g_ms / 1e3) / 1e12 if g_ms > 0 else None
        roofline = {"bound": "tensor", "kernel": "zgemm3m_kernel (FP64 filter step)",
                    "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": (achieved / fp64_peak) if achieved else None, "traffic": traffic,
                    "peak_note": f"FP64 = {peak_kind} bf16 sustained x 1.25/2250 (nominal FP64/bf16 "
                                 "ratio); achieved counts 8 flops per complex FMA"}
    phase_keys = ("t_reduce_ms", "t_lanczos_ms", "t_filter_ms", "t_filter_gemm_ms", "t_qr_ms", "t_small_ms",
                  "t_rr_ms", "t_eig_ms", "t_resid_ms", "t_total_ms")
    phase = {k: sum(s[k] for s in all_stats) for k in phase_keys}
    per_problem = [{"problem": s["problem"], "ms": s["t_total_ms"], "loops": s["loops"],
                    "filtered_vectors": s["filtered_vectors"]} for s in all_stats]
    cold_ms = [s["t_total_ms"] for s in all_stats if s["problem"] == 0]
    warm_ms = [s["t_total_ms"] for s in all_stats if s["problem"] != 0]

    # ---- per-eigenpair accuracy of the timed steps: eigenvalues against the planted ones and
    # generalized residuals ||A x - lam B x|| / (||A||_2 ||x||) (torch on the GPU, outside
    # the timed region; ||A||_2 = max |lam| for the planted pencil with ||B|| ~ 1)
    def pair_errors(evs, vecs):
        e_pl, res = [], []
        for p in sorted(evs):
            lam = evs[p].cpu().numpy()
            e_pl.append(np.abs(lam - lam_planted[p]) / lam_scale[p])
            if vecs.get(p) is not None:
                Af = As[p] + torch.tril(As[p], -1).mH
                Bf = B_low + torch.tril(B_low, -1).mH
                X = vecs[p]
                R = Af @ X - (Bf @ X) * evs[p].to(X.dtype).unsqueeze(0)
                anorm = torch.linalg.matrix_norm(Af, ord=2) if n <= 3000 else lam_scale[p]
                res.append((torch.linalg.vector_norm(R, dim=0) / (anorm * torch.linalg.vector_norm(X, dim=0)))
                           .cpu().numpy())
                del Af, Bf, R
        return np.concatenate(e_pl), (np.concatenate(res) if res else np.zeros(0))

    err_mixed, res_mixed = pair_errors(evals, evecs)

    # ---- deviation angles between eigenvectors of adjacent problems (Section 2.2, Fig. 1)
    dev_angles = None
    if not args.no_angles and N > 1 and all(evecs.get(p) is not None for p in range(N)):
        medians, maxs = [], []
        for ell in range(1, N):
            th, _ = cb.chfsi_deviation_angles(ctx, evecs[ell - 1], evecs[ell], Bs[ell])
            medians.append(float(th.median()))
            maxs.append(float(th.max()))
        dev_angles = {"median": medians, "max": maxs,
                      "note": "angle between x_i of problem l-1 and its associated x of problem l "
                              "(B-inner product), l = 1..N-1; a max near pi/2 marks an "
                              "eigenvalue crossing the nev boundary (its partner is not computed)"}
    del evecs

    # ---- the plain FP64 form on the same workload, same warm-up and timed steps
    plain = None
    if not args.no_plain:
        with cb.Solver(n, blk, stream=stream, deg_min=seq.deg_min, deg_max=seq.deg_max, precision=0) as s64:
            pms, ev64, vec64, st64 = run_arm(s64.ctx, want_vectors=True)
        err64, res64 = pair_errors(ev64, vec64)
        del vec64
        diff = np.concatenate([np.abs(evals[p].cpu().numpy() - ev64[p].cpu().numpy()) / lam_scale[p]
                               for p in sorted(evals)])
        conv64 = sum(int(torch.isfinite(ev64[p]).sum()) for p, _ in step_schedule(W, K, N))
        plain = {"value": conv64 / (pms / 1e3), "ms_per_step": pms / K, "steps": K, "warmup": W,
                 "max_resid": max(s["max_resid"] for s in st64),
                 "phase_ms": {k: sum(s[k] for s in st64) for k in phase_keys},
                 "per_eigenpair": {
                     "eig_diff_mixed_vs_fp64": summary(diff),
                     "eig_err_mixed_vs_planted": summary(err_mixed),
                     "eig_err_fp64_vs_planted": summary(err64),
                     "resid_mixed": summary(res_mixed),
                     "resid_fp64": summary(res64),
                     "note": "every eigenpair of the timed steps; eigenvalue errors relative to "
                             "max|lambda| of the problem; residuals ||Ax - lam Bx|| / (||A|| ||x||)"}}

    # ---- end to end through the C ABI with host buffers (pinned): the same warm-up and timed
    # steps, each problem's A and B copied from the host inside the region (the library
    # stages them), eigenvalues and eigenvectors copied back
    e2e = None
    if not args.no_e2e:
        B_h = B_low.mT.contiguous().cpu().pin_memory().mT
        A_h = [a.mT.contiguous().cpu().pin_memory().mT for a in As]
        B_hl = [B_h] * N

        def host_steps(first, count):
            conv = 0
            for p0, ln, cold in segments(first, count, N):
                if cold:
                    cb.chfsi_reset_warm_state(ctx)
                ev, _, _ = cb.chfsi_solve_sequence(ctx, A_h[p0:p0 + ln], B_hl[p0:p0 + ln], nev, blk, deg,
                                                   seq.tol, want_vectors=True)
                conv += int(torch.isfinite(ev).sum())
            return conv

        host_steps(0, W)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        conv_e2e = host_steps(W, K)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        t_e, c_e = combine_ranks(dt, conv_e2e, dev)
        e2e = {"value": c_e / t_e, "unit": UNIT,
               "h2d_bytes_per_step": 2 * n * n * 16,
               "d2h_bytes_per_step": nev * 8 + n * nev * 16, "steps": K, "warmup": W,
               "note": "host A and B of every problem staged by the library (copies of the next "
                       "problem overlap the current solve within a chfsi_solve_sequence call)"}
        del A_h, B_h, B_hl

    # ---- CPU baseline (oracle, host cores, bounded sample), rank 0 at N = 1 only
    cpu = None
    if want_cpu and N > 1:
        pairs, dt, loops, finished, lam_o = cpu_oracle_warm_problem(seq, 1, args.cpu_budget)
        cpu = {"value": pairs / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"problem 1 of the same n={n} sequence warm-started from the planted "
                         f"eigenvectors of problem 0, NumPy/SciPy FP64: {loops} loops, {pairs} pairs "
                         f"{'converged' if finished else 'locked before the time budget ran out'}, "
                         f"{dt:.1f} s"}
        if finished and 1 in evals:
            cpu["eig_diff_gpu_vs_oracle"] = summary(np.abs(evals[1].cpu().numpy() - lam_o) / lam_scale[1])

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K,
            "warmup": W, "ms_per_step": ms_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 (bf16 digit-slice tensor products)",
            "data": "synthetic",
            "config": {"workload": _workload_text(args.workload, seq, N),
                       "l2": f"inputs larger than L2 (A of {N} problems + B = "
                             f"{(N + 1) * n * n * 16 / 1e9:.1f} GB resident)",
                       "filter_arithmetic": "FP64 results from bf16 digit-slice tensor-core "
                                            "products (exact fp32 chunks, double-float sums): "
                                            "filter 2-7 slices chosen per loop, Rayleigh-Ritz, "
                                            "reduction and other large products 7-8 slices; FP32 "
                                            "Cholesky QR + FP64 Loewdin steps; FP64 Jacobi "
                                            "eigensolver, residuals and small products",
                       "tol": seq.tol, "max_resid": max_resid, "generation_s": t_gen,
                       "cold_problem_ms": cold_ms, "warm_problem_ms_mean": (sum(warm_ms) / len(warm_ms)) if warm_ms else None,
                       "per_problem": per_problem,
                       "phase_ms_timed_region": phase},
            "roofline": roofline,
            "plain_fp64": plain,
            "speedup_vs_plain_fp64": (value / plain["value"]) if plain else None,
            "cpu_baseline": cpu,
            "deviation_angles": dev_angles,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def run_heev_case(args):
    """One dense Hermitian eigensolve (the Rayleigh-Ritz Jacobi kernel) of a seeded random
    m x m Hermitian matrix through the C ABI: the small case used for the Jacobi profile."""
    from paper_1206_3768_gb300 import binding as cb

    dev = torch.device("cuda:0")
    g = torch.Generator(device="cpu").manual_seed(5)
    m = args.case_m
    M = torch.randn(m, m, dtype=torch.complex128, generator=g)
    G = (0.5 * (M + M.mH)).to(dev)
    # nearly diagonal, as the Gram matrix of a warm loop: sorted diagonal, 1e-6 coupling
    D = torch.diag(torch.linspace(-2.0, 2.0, m, dtype=torch.float64)).to(torch.complex128)
    N = torch.randn(m, m, dtype=torch.complex128, generator=g)
    Gd = (D + 0.5e-6 * (N + N.mH)).to(dev)
    out = {"case": "heev", "m": m}
    with cb.Solver(max(args.case_n, m), m) as s:
        for name, fn in (("fp64", cb.chfsi_heev), ("df", cb.chfsi_heev_df)):
            for label, A in (("random", G), ("near_diag", Gd)):
                for _ in range(args.case_reps):
                    fn(s.ctx, A)
                torch.cuda.synchronize()
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev0.record()
                w, V = fn(s.ctx, A)
                ev1.record()
                torch.cuda.synchronize()
                resid = float(((A @ V - V * w.to(V.dtype).unsqueeze(0)).abs().max() / A.abs().max()).item())
                orth = float((V.mH @ V - torch.eye(m, dtype=V.dtype, device=dev)).abs().max().item())
                out[f"{name}_{label}"] = {"ms": ev0.elapsed_time(ev1), "rel_resid": resid, "orth": orth}
    print(json.dumps(out))


def run_batch(args):
    """The batched k-point workload: K independent sequences of uneven size (n_k uniform in
    [3000, 6000], nev_k = ceil(0.04 n_k), blk_k = ceil(1.3 nev_k), degree 20), solved by a
    batch of --workers contexts on their own streams, against the same sequences solved one
    after another on one context.  Host wall time around each solve (both return only after
    their streams are synchronised)."""
    from paper_1206_3768_gb300 import binding as cb
    from paper_1206_3768_gb300 import inputs

    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    K, N = args.kpoints, args.problems or 10
    t_gen = time.perf_counter()
    seqs = inputs.kpoint_sequences(K=K, N=N, device=dev)
    data = []
    for q in seqs:  # lower triangles, column-major, one B per k-point; originals freed as we go
        B_low = cb.fortran(torch.tril(q.problems[0].B))
        As = []
        for p in q.problems:
            As.append(cb.fortran(torch.tril(p.A)))
            p.A = None
            p.B = None
        data.append((As, [B_low] * N))
    torch.cuda.empty_cache()
    t_gen = time.perf_counter() - t_gen
    nev = [q.nev for q in seqs]
    blk = [q.blk for q in seqs]
    n_max, blk_max = max(q.n for q in seqs), max(blk)
    torch.cuda.synchronize()
    pairs = sum(N * v for v in nev)
    with cb.Batch(args.workers, n_max, blk_max) as batch:
        for _ in range(max(1, args.warmup)):
            batch.solve(data[:args.workers], nev[:args.workers], blk[:args.workers], 20, 1e-10,
                        want_vectors=False)
        t0 = time.perf_counter()
        res = batch.solve(data, nev, blk, 20, 1e-10, want_vectors=False)
        t_batch = time.perf_counter() - t0
    conv_b = sum(int(torch.isfinite(ev).sum()) for ev, _, _ in res)
    max_resid = max(st["max_resid"] for _, _, sts in res for st in sts)
    with cb.Solver(n_max, blk_max) as s:
        cb.chfsi_reset_warm_state(s.ctx)
        cb.chfsi_solve_sequence(s.ctx, data[0][0], data[0][1], nev[0], blk[0], 20, 1e-10,
                                want_vectors=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        conv_s = 0
        for (As, Bs), v, b in zip(data, nev, blk):
            cb.chfsi_reset_warm_state(s.ctx)
            ev, _, _ = cb.chfsi_solve_sequence(s.ctx, As, Bs, v, b, 20, 1e-10, want_vectors=False)
            conv_s += int(torch.isfinite(ev).sum())
        torch.cuda.synchronize()
        t_seq = time.perf_counter() - t0
        # the same form on the first k-points alone, for the plain-FP64 comparison below
        ksub = min(K, 4)
        t0 = time.perf_counter()
        conv_sub = 0
        for (As, Bs), v, b in zip(data[:ksub], nev[:ksub], blk[:ksub]):
            cb.chfsi_reset_warm_state(s.ctx)
            ev, _, _ = cb.chfsi_solve_sequence(s.ctx, As, Bs, v, b, 20, 1e-10, want_vectors=False)
            conv_sub += int(torch.isfinite(ev).sum())
        t_sub = time.perf_counter() - t0
    with cb.Solver(n_max, blk_max, precision=0) as s64:
        t0 = time.perf_counter()
        conv64 = 0
        for (As, Bs), v, b in zip(data[:ksub], nev[:ksub], blk[:ksub]):
            cb.chfsi_reset_warm_state(s64.ctx)
            ev, _, _ = cb.chfsi_solve_sequence(s64.ctx, As, Bs, v, b, 20, 1e-10, want_vectors=False)
            conv64 += int(torch.isfinite(ev).sum())
        t64 = time.perf_counter() - t0
    eig_err = max(float(np.max(np.abs(ev[l].numpy() - p.lam[:q.nev]))) / float(np.max(np.abs(p.lam)))
                  for q, (ev, _, _) in zip(seqs, res) for l, p in enumerate(q.problems))
    print(json.dumps({
        "metric": "batched k-point sequences, converged eigenpairs/s", "value": conv_b / t_batch,
        "unit": UNIT, "higher_is_better": True, "n_gpus": 1,
        "sequential": {"value": conv_s / t_seq, "seconds": t_seq},
        "speedup_vs_sequential": (conv_b / t_batch) / (conv_s / t_seq), "seconds": t_batch,
        "pairs": pairs, "max_resid": max_resid, "max_eig_err_vs_planted": eig_err,
        "plain_fp64_first_kpoints": {"kpoints": ksub, "value": conv64 / t64, "seconds": t64,
                                     "mixed_same_kpoints": conv_sub / t_sub,
                                     "speedup_mixed_vs_fp64": (conv_sub / t_sub) / (conv64 / t64)},
        "config": {"workload": f"c4: K={K} k-point sequences, N={N} problems each, n_k in "
                               f"[3000, 6000] ({min(q.n for q in seqs)}..{n_max}), nev_k = "
                               f"ceil(0.04 n_k), blk_k = ceil(1.3 nev_k), deg 20, first problem "
                               f"cold, rest warm", "workers": args.workers, "generation_s": t_gen},
    }), flush=True)


def run_degree_model(args):
    """The learned per-vector degree (three hidden layers of 64, FP16 weights in the solver)
    against the closed-form rule and a fixed degree (25, the ChFSI degree of Table 3), degrees
    in [4, 40]: the model is trained by the library's CUDA kernels on the degree logs of the
    n = 512 and n = 2600 workloads (independent seeds, closed-form degrees, not timed), then
    the evaluation sequence is solved once per form, each timed with CUDA events over the
    whole sequence (first problem cold, the rest warm)."""
    from paper_1206_3768_gb300 import binding as cb
    from paper_1206_3768_gb300 import degree_model as dm
    from paper_1206_3768_gb300 import inputs

    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    name = args.workload
    N = args.problems or inputs.CONFIGS[name]["N"]
    # ---- training data: degree logs of the n = 512 and n = 2600 sequences
    logs, t0 = [], time.perf_counter()
    for tname, tN in (("c1", 6), ("c2", 6)):
        tr = inputs.planted_sequence(tname, N=tN, device=dev, keep_vectors=False, seed_offset=3)
        with cb.Solver(tr.n, tr.blk, stream=stream, deg_min=4, deg_max=40) as s:
            cb.chfsi_degree_log_start(s.ctx, 5_000_000)
            cb.chfsi_reset_warm_state(s.ctx)
            cb.chfsi_solve_sequence(s.ctx, [p.A for p in tr.problems], [p.B for p in tr.problems], tr.nev, tr.blk,
                                    0, tr.tol, want_vectors=False)
            logs.append(cb.chfsi_degree_log_read(s.ctx))
        del tr
    log = np.concatenate(logs)
    X, z = dm.training_pairs(log)
    t_logs = time.perf_counter() - t0
    evalseq = inputs.planted_sequence(name, N=N, device=dev, keep_vectors=False)
    n, nev, blk = evalseq.n, evalseq.nev, evalseq.blk
    As = [cb.fortran(torch.tril(p.A)) for p in evalseq.problems]
    B_low = cb.fortran(torch.tril(evalseq.problems[0].B))
    Bs = [B_low] * N
    for p in evalseq.problems:
        p.A = None
    scale = max(float(np.max(np.abs(p.lam))) for p in evalseq.problems)
    out = {}
    with cb.Solver(n, blk, stream=stream, deg_min=4, deg_max=40) as s:
        model = cb.chfsi_mlp_init(12063768)
        t0 = time.perf_counter()
        loss = cb.chfsi_mlp_train(s.ctx, model, X, z, epochs=args.epochs, batch=256, lr=2e-3, seed=1)
        t_train = time.perf_counter() - t0
        cb.chfsi_reset_warm_state(s.ctx)
        cb.chfsi_solve_sequence(s.ctx, As[:1], Bs[:1], nev, blk, 0, evalseq.tol, want_vectors=False)  # warm-up
        for form, mdl, deg in (("fixed_degree_25", None, 25), ("closed_form", None, 0), ("learned", model, 0)):
            cb.chfsi_set_degree_model(s.ctx, mdl)
            cb.chfsi_reset_warm_state(s.ctx)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ev, _, st = cb.chfsi_solve_sequence(s.ctx, As, Bs, nev, blk, deg, evalseq.tol, want_vectors=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            err = max(float(np.max(np.abs(ev[l].numpy() - p.lam[:nev]))) for l, p in enumerate(evalseq.problems))
            out[form] = {"eigenpairs_per_s": float(torch.isfinite(ev).sum()) / (ms / 1e3), "ms": ms,
                         "filter_matvecs": int(sum(x["filter_matvecs"] for x in st)),
                         "filter_products": int(sum(x["filter_products"] for x in st)),
                         "loops": int(sum(x["loops"] for x in st)),
                         "t_filter_ms": sum(x["t_filter_ms"] for x in st),
                         "phase_ms": {k: round(sum(x[k] for x in st), 1) for k in
                                      ("t_reduce_ms", "t_lanczos_ms", "t_filter_ms", "t_filter_gemm_ms", "t_qr_ms",
                                       "t_small_ms", "t_rr_ms", "t_eig_ms", "t_resid_ms", "t_total_ms")},
                         "loops_per_problem": [x["loops"] for x in st],
                         "max_resid": max(x["max_resid"] for x in st), "max_eig_err": err / scale}
        cb.chfsi_set_degree_model(s.ctx, None)
    L, C, F = out["learned"], out["closed_form"], out["fixed_degree_25"]
    print(json.dumps({
        "metric": "learned vs closed-form vs fixed filter degree (wall time, filter matvecs) @res<=1e-10",
        "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
        "fixed_degree_25": F, "closed_form": C, "learned": L,
        "speedup_learned_vs_fixed": F["ms"] / L["ms"], "speedup_learned_vs_closed_form": C["ms"] / L["ms"],
        "matvec_ratio_learned_over_fixed": L["filter_matvecs"] / F["filter_matvecs"],
        "matvec_ratio_learned_over_closed_form": L["filter_matvecs"] / C["filter_matvecs"],
        "training": {"records": int(log.shape[0]), "samples": int(len(z)), "epochs": args.epochs,
                     "final_loss": loss, "target_variance": float(np.var(z)) if len(z) else None,
                     "seconds": t_train, "log_seconds": t_logs,
                     "data": "degree logs of the n=512 and n=2600 sequences (seed offset 3, 6 problems each), "
                             "closed-form degrees in [4, 40]"},
        "config": {"workload": f"{name}: n={n} nev={nev} blk={blk} N={N}, degree range [4, 40], "
                               "first problem cold, rest warm"},
    }), flush=True)


def run_kernel_case(args):
    """One Chebyshev filter call (deg launches of the filter GEMM) through the C ABI on a
    seeded n x n Hermitian matrix and n x m block: the small case used for kernel profiles."""
    from paper_1206_3768_gb300 import binding as cb

    dev = torch.device("cuda:0")
    g = torch.Generator(device="cpu").manual_seed(1206)
    n, m = args.case_n, args.case_m
    M = torch.randn(n, n, dtype=torch.complex128, generator=g)
    H = (0.5 * (M + M.mH) / math.sqrt(n)).to(dev)
    Y = torch.randn(n, m, dtype=torch.complex128, generator=g).to(dev)
    degs = [args.case_deg] * m

    def call():
        if args.case_slices > 0:
            return cb.chfsi_filter_split(s.ctx, H, Y, degs, -2.0, -1.0, 2.5, args.case_slices)
        return cb.chfsi_filter(s.ctx, H, Y, degs, -2.0, -1.0, 2.5)

    with cb.Solver(n, m, precision=1 if args.case_slices > 0 else 0) as s:
        for _ in range(args.case_reps):
            out = call()
        torch.cuda.synchronize()
        times = []
        for _ in range(max(1, args.case_timed)):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            out = call()
            ev1.record()
            torch.cuda.synchronize()
            times.append(ev0.elapsed_time(ev1))
        ref = (cb.chfsi_filter(s.ctx, H, Y, degs, -2.0, -1.0, 2.5) if args.case_slices > 0 and args.case_check
               else out)
    ms = min(times)
    flops = 8.0 * n * n * m * args.case_deg
    err = float(((out - ref).abs().max() / ref.abs().max()).item())
    print(json.dumps({"case": "filter", "n": n, "m": m, "deg": args.case_deg,
                      "slices": args.case_slices, "ms": ms, "fp64_equiv_tflops": flops / ms / 1e9,
                      "rel_err_vs_fp64": err, "finite": bool(torch.isfinite(out).all())}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-budget", type=float, default=150.0,
                    help="seconds of oracle work for the cpu_baseline sample (one warm problem)")
    ap.add_argument("--ref-problems", type=int, default=6,
                    help="problems generated for the reference arm (its loops run through them)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-angles", action="store_true")
    ap.add_argument("--degree-model", action="store_true",
                    help="train the learned degree on logs of training sequences and compare it with "
                         "the closed form on the workload (a separate line, not the headline)")
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--kpoints", type=int, default=32)
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--workload", choices=["c2", "c3", "c4", "c5"], default=WORKLOAD,
                    help="c3: n=9300, nev=256, blk=320, deg 20 (the headline); c2: n=2600 adaptive "
                         "degree; c5: n=13400, blk=1200, degrees in [4, 40]; c4: --kpoints "
                         "sequences of uneven size solved by a batch of --workers contexts against "
                         "one context (a separate line, not the headline)")
    ap.add_argument("--no-direct", action="store_true")
    ap.add_argument("--problems", type=int, default=None,
                    help="solve only the first N problems of the sequence (profiling runs)")
    ap.add_argument("--kernel-case", choices=["filter", "heev"], default=None)
    ap.add_argument("--case-n", type=int, default=4096)
    ap.add_argument("--case-m", type=int, default=128)
    ap.add_argument("--case-deg", type=int, default=3)
    ap.add_argument("--case-reps", type=int, default=1)
    ap.add_argument("--case-slices", type=int, default=0)
    ap.add_argument("--case-timed", type=int, default=1, help="timed calls (the minimum is reported)")
    ap.add_argument("--case-check", type=int, default=1, help="compare with the FP64 filter")
    args = ap.parse_args()
    if args.degree_model and args.impl == "ours":
        run_degree_model(args)
    elif args.workload == "c4" and args.impl == "ours" and not args.kernel_case:
        run_batch(args)
    elif args.kernel_case == "heev":
        run_heev_case(args)
    elif args.kernel_case:
        run_kernel_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
