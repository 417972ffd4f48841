"""Benchmark: converged eigenpairs per second of warm-started ChFSI sequences on GB300.

One step = one full sequence solve (the whole hot path: reduction, Lanczos bound,
Chebyshev filter, Cholesky QR, Rayleigh-Ritz, locking, back-transform) of the FLAPW-shaped
workload: n = 2600, nev = 100, blk = 130, adaptive degree in [8, 25], 20 correlated
problems (first cold, the rest warm-started), cond(B) = 1e4, planted spectrum.  Inputs are
seeded synthetic matrices resident in HBM (4.3 GB per step, larger than L2).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own independent sequence (different seed): the units
(eigenpairs) of all ranks are summed and divided by the slowest rank's time ("weak").
``--impl reference`` times the CPU oracle (NumPy/SciPy FP64) on a bounded sample of the
same workload; only rank 0 runs it.
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
WORKLOAD = "c2"


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


def load_workload(device, rank: int, name: str = WORKLOAD, N=None):
    from paper_1206_3768_gb300 import inputs

    return inputs.planted_sequence(name, device=device, keep_vectors=False, seed_offset=rank, N=N)


def cpu_oracle_sample(seq, problems: int):
    """Time the oracle on the first `problems` problems of the sequence (host cores)."""
    import oracle.chfsi_oracle as O

    As = [np.tril(p.A.cpu().numpy()) for p in seq.problems[:problems]]
    Bs = [np.tril(p.B.cpu().numpy()) for p in seq.problems[:problems]]
    t0 = time.perf_counter()
    out = O.chfsi_solve_sequence(As, Bs, seq.nev, seq.blk, seq.tol, deg=seq.deg,
                                 deg_min=seq.deg_min, deg_max=seq.deg_max)
    dt = time.perf_counter() - t0
    pairs = sum(int(np.isfinite(lam).sum()) for lam, _, _ in out)
    return pairs, dt


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    seq = load_workload("cpu", 0, N=args.cpu_problems)
    k = max(1, args.steps)
    w = max(0, args.warmup)
    # Warm-up steps on a one-problem sample, timed steps on the sample of --cpu-problems.
    for _ in range(w):
        cpu_oracle_sample(seq, 1)
    times, pairs_tot = [], 0
    for _ in range(k):
        pairs, dt = cpu_oracle_sample(seq, args.cpu_problems)
        times.append(dt)
        pairs_tot += pairs
    total = sum(times)
    value = pairs_tot / total
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": k, "warmup": w, "ms_per_step": 1e3 * total / k, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: n=2600 nev=100 blk=130 deg adaptive 8-25 cond(B)=1e4",
                   "sample_problems": args.cpu_problems},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"first {args.cpu_problems} problems (1 cold + "
                                   f"{args.cpu_problems - 1} warm) of the n=2600 sequence"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    from paper_1206_3768_gb300 import binding as cb

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    seq = load_workload(dev, rank, name=args.workload, N=args.problems)
    n, nev, blk, N = seq.n, seq.nev, seq.blk, len(seq.problems)
    As = [cb.fortran(torch.tril(p.A)) for p in seq.problems]
    Bs = [cb.fortran(torch.tril(p.B)) for p in seq.problems]
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    solver = cb.Solver(n, blk, stream=stream, deg_min=seq.deg_min, deg_max=seq.deg_max)
    ctx = solver.ctx

    def step(A_list, B_list, want_vectors=True):
        cb.chfsi_reset_warm_state(ctx)
        return cb.chfsi_solve_sequence(ctx, A_list, B_list, nev, blk, seq.deg, seq.tol,
                                       want_vectors=want_vectors)

    for _ in range(args.warmup):
        step(As, Bs)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            import torch.distributed as dist

            dist.barrier()

    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    all_stats = []
    converged = 0
    e0.record(stream)
    for _ in range(args.steps):
        evals, evecs, stats = step(As, Bs)
        all_stats.extend(stats)
        converged += int(torch.isfinite(evals).sum())
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
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
                ratio = float(json.load(f)["dram_bytes_over_slice_bytes"])
            traffic = ratio * sum(s["filter_slice_bytes"] for s in all_stats) / products
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
                                 "slice-pair products (2 x pairs x 2n x m x 2n flops each, "
                                 "unpadded) over the product kernel's CUDA-event time"}
    else:
        fp64_peak = peaks["bf16_tflops_sustained"] * 1.25 / 2250.0
        achieved = fp64_equiv / (g_ms / 1e3) / 1e12 if g_ms > 0 else None
        roofline = {"bound": "tensor", "kernel": "zgemm3m_kernel (FP64 filter step)",
                    "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": (achieved / fp64_peak) if achieved else None, "traffic": traffic,
                    "peak_note": f"FP64 = {peak_kind} bf16 sustained x 1.25/2250 (nominal FP64/bf16 "
                                 "ratio); achieved counts 8 flops per complex FMA"}
    phase = {k: sum(s[k] for s in all_stats) / args.steps for k in
             ("t_reduce_ms", "t_lanczos_ms", "t_filter_ms", "t_filter_gemm_ms", "t_qr_ms", "t_small_ms",
              "t_rr_ms", "t_eig_ms", "t_resid_ms", "t_total_ms")}

    # ---- deviation angles between eigenvectors of adjacent problems (Section 2.2, Fig. 1),
    # from the last timed step's eigenvectors (outside the timed region)
    dev_angles = None
    if not args.no_angles and evecs is not None and N > 1:
        medians, maxs = [], []
        for ell in range(1, N):
            th, _ = cb.chfsi_deviation_angles(ctx, evecs[ell - 1], evecs[ell], Bs[ell])
            medians.append(float(th.median()))
            maxs.append(float(th.max()))
        dev_angles = {"median": medians, "max": maxs,
                      "note": "angle between x_i of problem l-1 and its associated x of problem l "
                              "(B-inner product), l = 1..N-1; a max near pi/2 marks an "
                              "eigenvalue crossing the nev boundary (its partner is not computed)"}

    # ---- a direct solver on the same problem for context (library code, not this path):
    # torch.linalg Cholesky, triangular solves and the dense Hermitian eigensolver (all
    # eigenpairs, from which the nev lowest are kept), one cold problem
    direct = None
    if not args.no_direct:
        A0 = seq.problems[0].A
        B0 = seq.problems[0].B
        torch.linalg.eigh(torch.eye(64, dtype=torch.complex128, device=dev))  # library warm-up
        torch.cuda.synchronize()
        d0 = torch.cuda.Event(enable_timing=True)
        d1 = torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        Lc = torch.linalg.cholesky(B0)
        T1 = torch.linalg.solve_triangular(Lc, A0, upper=False)
        Hd = torch.linalg.solve_triangular(Lc, T1.mH, upper=False).mH
        wd, _ = torch.linalg.eigh(0.5 * (Hd + Hd.mH))
        d1.record(stream)
        torch.cuda.synchronize()
        dms = d0.elapsed_time(d1)
        err = float((wd[:nev].cpu().numpy() - seq.problems[0].lam[:nev]).__abs__().max())
        direct = {"value": nev / (dms / 1e3), "unit": UNIT, "ms_per_problem": dms,
                  "kind": "torch.linalg cholesky + solve_triangular + eigh (cuSOLVER), one cold problem",
                  "max_abs_eig_err": err}

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the region
    e2e = None
    if not args.no_e2e:
        Ah = [a.mT.contiguous().cpu().pin_memory().mT for a in As]
        Bh = [b.mT.contiguous().cpu().pin_memory().mT for b in Bs]
        evecs_h = None
        steps_e2e = max(1, min(args.steps, 2))
        step_host = lambda: (cb.chfsi_reset_warm_state(ctx),
                             cb.chfsi_solve_sequence(ctx, Ah, Bh, nev, blk, seq.deg, seq.tol))
        step_host()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        conv_e2e = 0
        for _ in range(steps_e2e):
            _, (ev, evecs_h, _) = step_host()
            conv_e2e += int(torch.isfinite(ev).sum())
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        t_e, c_e = combine_ranks(dt, conv_e2e, dev)
        e2e = {"value": c_e / t_e, "unit": UNIT,
               "h2d_bytes_per_step": N * 2 * n * n * 16,
               "d2h_bytes_per_step": N * (nev * 8 + n * nev * 16), "steps": steps_e2e}

    # ---- the plain FP64 form on the same workload (one timed step), for the speed-up
    plain = None
    if not args.no_plain:
        with cb.Solver(n, blk, stream=stream, deg_min=seq.deg_min, deg_max=seq.deg_max,
                       precision=0) as s64:
            cb.chfsi_reset_warm_state(s64.ctx)
            torch.cuda.synchronize()
            p0 = torch.cuda.Event(enable_timing=True)
            p1 = torch.cuda.Event(enable_timing=True)
            p0.record(stream)
            ev64, _, st64 = cb.chfsi_solve_sequence(s64.ctx, As, Bs, nev, blk, seq.deg, seq.tol,
                                                    want_vectors=False)
            p1.record(stream)
            torch.cuda.synchronize()
            pms = p0.elapsed_time(p1)
        # per-eigenpair difference between the mixed-precision and the FP64 eigenvalues, and
        # both against the planted spectrum, relative to max |lambda|
        lam_ref = np.stack([p.lam[:nev] for p in seq.problems])
        scale = float(np.max(np.abs(np.stack([p.lam for p in seq.problems]))))
        e_mixed, e_fp64 = evals.cpu().numpy(), ev64.cpu().numpy()
        plain = {"value": float(torch.isfinite(ev64).sum()) / (pms / 1e3), "ms_per_step": pms,
                 "steps": 1, "max_resid": max(s["max_resid"] for s in st64),
                 "max_eig_diff_mixed_vs_fp64": float(np.max(np.abs(e_mixed - e_fp64))) / scale,
                 "max_eig_err_mixed_vs_planted": float(np.max(np.abs(e_mixed - lam_ref))) / scale,
                 "max_eig_err_fp64_vs_planted": float(np.max(np.abs(e_fp64 - lam_ref))) / scale}

    # ---- CPU baseline (oracle, host cores, bounded sample), rank 0 at N = 1 only
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        pairs, dt = cpu_oracle_sample(seq, args.cpu_problems)
        cpu = {"value": pairs / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"first {args.cpu_problems} problems (1 cold + {args.cpu_problems - 1} "
                         f"warm) of the same n={n} sequence, NumPy/SciPy FP64, {dt:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 (bf16 digit-slice tensor products)",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: n={n} nev={nev} blk={blk} "
                                   + (f"deg={seq.deg} fixed" if seq.deg > 0 else
                                      f"deg adaptive {seq.deg_min}-{seq.deg_max}")
                                   + f" N={N} "
                                   + ("cond(B)=1e4" if args.workload == "c2" else "B=I+0.1G^HG/n")
                                   + ", planted spectrum, first problem cold, rest warm",
                       "l2": f"inputs larger than L2 (A,B of {N} problems = "
                             f"{N * 2 * n * n * 16 / 1e9:.1f} GB per step)",
                       "filter_arithmetic": "FP64 results from bf16 digit-slice tensor-core "
                                            "products (exact fp32 chunks, double-float sums): "
                                            "filter 2-7 slices chosen per loop, Rayleigh-Ritz, "
                                            "reduction and other large products 7 slices; FP32 "
                                            "Cholesky QR + FP64 Loewdin steps; FP64 Jacobi "
                                            "eigensolver, residuals and small products",
                       "tol": seq.tol, "max_resid": max_resid,
                       "loops_per_problem": [s["loops"] for s in all_stats[:N]],
                       "filtered_vectors_per_problem": [s["filtered_vectors"] for s in all_stats[:N]],
                       "phase_ms_per_step": phase},
            "roofline": roofline,
            "plain_fp64": plain,
            "speedup_vs_plain_fp64": (value / plain["value"]) if plain else None,
            "cpu_baseline": cpu,
            "direct_solver": direct,
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
    with cb.Solver(max(args.case_n, m), m) as s:
        for _ in range(args.case_reps):
            cb.chfsi_heev(s.ctx, G)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        w, V = cb.chfsi_heev(s.ctx, G)
        ev1.record()
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    resid = float(((G @ V - V * w.to(V.dtype).unsqueeze(0)).abs().max() / G.abs().max()).item())
    print(json.dumps({"case": "heev", "m": m, "ms": ms, "rel_resid": resid}))


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
    seqs = inputs.kpoint_sequences(K=K, N=N, device=dev)
    data = [([cb.fortran(torch.tril(p.A)) for p in q.problems],
             [cb.fortran(torch.tril(p.B)) for p in q.problems]) for q in seqs]
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
    print(json.dumps({
        "metric": "batched k-point sequences, converged eigenpairs/s", "value": conv_b / t_batch,
        "unit": UNIT, "higher_is_better": True, "n_gpus": 1,
        "sequential": {"value": conv_s / t_seq, "seconds": t_seq},
        "speedup_vs_sequential": (conv_b / t_batch) / (conv_s / t_seq), "seconds": t_batch,
        "pairs": pairs, "max_resid": max_resid,
        "config": {"workload": f"c4: K={K} k-point sequences, N={N} problems each, n_k in "
                               f"[3000, 6000] ({min(q.n for q in seqs)}..{n_max}), nev_k = "
                               f"ceil(0.04 n_k), blk_k = ceil(1.3 nev_k), deg 20, first problem "
                               f"cold, rest warm", "workers": args.workers},
    }), flush=True)


def run_degree_model(args):
    """The learned per-vector degree against the closed-form rule (degree range [4, 40]):
    the model is trained on degree logs of independent training sequences of the same shape
    (seed offsets 1 and 2, not timed), then the evaluation sequence is solved with each
    rule; both solves are timed with CUDA events over the whole sequence."""
    from paper_1206_3768_gb300 import binding as cb
    from paper_1206_3768_gb300 import degree_model as dm
    from paper_1206_3768_gb300 import inputs

    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    N = args.problems or 20
    stream = torch.cuda.current_stream(dev)
    evalseq = inputs.planted_sequence(args.workload, N=N, device=dev, keep_vectors=False)
    n, nev, blk = evalseq.n, evalseq.nev, evalseq.blk
    with cb.Solver(n, blk, stream=stream, deg_min=4, deg_max=40) as s:
        cb.chfsi_degree_log_start(s.ctx, 10_000_000)
        for off in (1, 2):
            tr = inputs.planted_sequence(args.workload, N=min(N, 8), device=dev, keep_vectors=False,
                                         seed_offset=off)
            cb.chfsi_reset_warm_state(s.ctx)
            cb.chfsi_solve_sequence(s.ctx, [p.A for p in tr.problems], [p.B for p in tr.problems], nev, blk, 0,
                                    evalseq.tol, want_vectors=False)
            del tr
        log = cb.chfsi_degree_log_read(s.ctx)
        cb.chfsi_degree_log_start(s.ctx, 0)
        X, z = dm.training_pairs(log)
        model = cb.chfsi_mlp_init(12063768)
        t0 = time.perf_counter()
        loss = cb.chfsi_mlp_train(s.ctx, model, X, z, epochs=args.epochs, batch=256, lr=2e-3, seed=1)
        t_train = time.perf_counter() - t0
        z_var = float(np.var(z)) if len(z) else float("nan")
        As = [p.A for p in evalseq.problems]
        Bs = [p.B for p in evalseq.problems]
        out = {}
        for name, mdl in (("closed_form", None), ("learned", model)):
            cb.chfsi_set_degree_model(s.ctx, mdl)
            for _ in range(max(1, args.warmup)):
                cb.chfsi_reset_warm_state(s.ctx)
                cb.chfsi_solve_sequence(s.ctx, As, Bs, nev, blk, 0, evalseq.tol, want_vectors=False)
            cb.chfsi_reset_warm_state(s.ctx)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ev, _, st = cb.chfsi_solve_sequence(s.ctx, As, Bs, nev, blk, 0, evalseq.tol, want_vectors=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            scale = max(float(np.max(np.abs(p.lam))) for p in evalseq.problems)
            err = max(float(np.max(np.abs(ev[l].numpy() - p.lam[:nev]))) for l, p in enumerate(evalseq.problems))
            out[name] = {"eigenpairs_per_s": float(torch.isfinite(ev).sum()) / (ms / 1e3), "ms": ms,
                         "filter_matvecs": int(sum(x["filter_matvecs"] for x in st)),
                         "loops": int(sum(x["loops"] for x in st)),
                         "max_resid": max(x["max_resid"] for x in st), "max_eig_err": err / scale}
        cb.chfsi_set_degree_model(s.ctx, None)
    print(json.dumps({
        "metric": "learned vs closed-form filter degree (converged eigenpairs/s, filter matvecs)",
        "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
        "closed_form": out["closed_form"], "learned": out["learned"],
        "matvec_ratio_learned_over_closed": out["learned"]["filter_matvecs"] / out["closed_form"]["filter_matvecs"],
        "speedup_learned": out["learned"]["eigenpairs_per_s"] / out["closed_form"]["eigenpairs_per_s"],
        "training": {"samples": int(len(z)), "epochs": args.epochs, "final_loss": loss,
                     "target_variance": z_var, "seconds": t_train,
                     "data": "degree logs of 2 training sequences (seed offsets 1, 2) of the same shape"},
        "config": {"workload": f"{args.workload}: n={n} nev={nev} blk={blk} N={N}, degree range [4, 40], "
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
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        out = call()
        ev1.record()
        torch.cuda.synchronize()
        ref = cb.chfsi_filter(s.ctx, H, Y, degs, -2.0, -1.0, 2.5) if args.case_slices > 0 else out
    ms = ev0.elapsed_time(ev1)
    flops = 8.0 * n * n * m * args.case_deg
    err = float(((out - ref).abs().max() / ref.abs().max()).item())
    print(json.dumps({"case": "filter", "n": n, "m": m, "deg": args.case_deg,
                      "slices": args.case_slices, "ms": ms, "fp64_equiv_tflops": flops / ms / 1e9,
                      "rel_err_vs_fp64": err, "finite": bool(torch.isfinite(out).all())}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-problems", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-angles", action="store_true")
    ap.add_argument("--degree-model", action="store_true",
                    help="train the learned degree on logs of training sequences and compare it with "
                         "the closed form on the workload (a separate line, not the headline)")
    ap.add_argument("--epochs", type=int, default=150)
    ap.add_argument("--kpoints", type=int, default=32)
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--workload", choices=["c2", "c3", "c4"], default=WORKLOAD,
                    help="c2: n=2600 adaptive degree (the headline); c3: n=9300, nev=256, blk=320, "
                         "deg 20 (the mixed-precision workload; use --problems to bound it); c4: "
                         "--kpoints sequences of uneven size solved by a batch of --workers "
                         "contexts against one context (a separate line, not the headline)")
    ap.add_argument("--no-direct", action="store_true")
    ap.add_argument("--problems", type=int, default=None,
                    help="solve only the first N problems of the sequence (profiling runs)")
    ap.add_argument("--kernel-case", choices=["filter", "heev"], default=None)
    ap.add_argument("--case-n", type=int, default=4096)
    ap.add_argument("--case-m", type=int, default=128)
    ap.add_argument("--case-deg", type=int, default=3)
    ap.add_argument("--case-reps", type=int, default=1)
    ap.add_argument("--case-slices", type=int, default=0)
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
