"""Benchmark: MG-preconditioned SQMR (Tao & Sifakis, Alg. 4) on the 256^3 MAC Stokes workload.

One step = one full solve of a 256^3 box problem (Gaussian-bump forcing, 16 bumps, seed = step mod 5,
eta = 1, gamma = 1e-3, no-slip walls) from x0 = 0 to true relative residual 1e-8, with inputs resident in
HBM.  The headline runs the FP32 V-cycle with FP64 SQMR recurrences; the plain FP64 V-cycle solve of the
same problems is timed beside it.  Under torchrun every rank solves its own problems (weak scaling, no
collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference] [--n 256]

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a bounded sample of the same
workload (see cpu_sample()).
"""
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

METRIC = "solved unknowns/sec to rel. residual 1e-8 at 256^3; V-cycle HBM GB/s vs peak"
UNIT = "unknowns/s"


def unknowns(n):
    return 3 * n * n * (n - 1) + n ** 3


def packed_len(n):
    return 3 * (n + 1) * n * n + n ** 3


def workload_name(n):
    return (f"{n}^3 MAC Stokes box, 16 Gaussian bumps (seeds 0-4), eta=1, gamma=1e-3, no-slip walls, "
            f"MG(V-cycle, Alg. 3 smoother)-preconditioned SQMR from x0=0 to rel. residual 1e-8")


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def oracle_iterations(n, seed=0, tol=1e-8):
    p = os.path.join(ROOT, "tests", "golden", "oracle_iterations.txt")
    if not os.path.exists(p):
        return None
    for line in open(p):
        if line.startswith("#") or not line.strip():
            continue
        f = [v.strip() for v in line.split(",")]
        if int(f[0]) == n and int(f[1]) == seed and float(f[2]) == tol:
            return int(f[3])
    return None


# ------------------------------------------------------------------------------------------ CPU oracle

ARM_PARTS = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1", "0xd49": "Arm Neoverse N2"}


def host_info():
    """nproc and the CPU model of this host (for the CPU-baseline records); Arm hosts report the CPU part."""
    model, part = None, None
    try:
        for line in open("/proc/cpuinfo"):
            if ":" not in line:
                continue
            k, v = (t.strip() for t in line.split(":", 1))
            if k.lower() == "model name" and model is None:
                model = v
            if k.lower() == "cpu part" and part is None:
                part = v
    except OSError:
        pass
    if model is None and part is not None:
        model = f"{ARM_PARTS.get(part, 'Arm')} (CPU part {part})"
    return {"nproc": os.cpu_count(), "cpu_model": model}


def cpu_sample(n, steps=1, warmup=0, iters=None, threads=None):
    """Time the oracle (FP64 C, as it stands) on bounded samples of the n^3 workload.

    Sample = one Alg. 3 smoothing application on the finest level of the n^3 problem (the solve's
    single largest piece of work), run `threads` OpenMP threads wide (the oracle's order-free loops;
    its results are bit-identical for any thread count).  The whole solve's time is extrapolated
    from it: a full MG-SQMR solve of the 64^3 problem to 1e-8 is timed with the same threads, which
    gives the cost of one SQMR iteration in units of one 64^3 smoothing; times the oracle's iteration
    count for the n^3 workload (tests/golden/oracle_iterations.txt, written by the oracle alone) plus
    the initial V-cycle.  Returns the timed samples and the extrapolated solve time.
    """
    import oracle
    import synthetic
    threads = threads or os.cpu_count() or 1
    used = oracle.set_threads(threads)
    try:
        o64 = oracle.Oracle(64, coarsest_max=8)
        b64 = o64.rhs(synthetic.bumps(64, seed=0)["f"].numpy(), None)
        z = np.zeros(o64.n())
        o64.smooth(z, b64, level=0)  # warm
        t0 = time.perf_counter()
        o64.smooth(z, b64, level=0)
        t_s64 = time.perf_counter() - t0
        t0 = time.perf_counter()
        x64, rc64, it64, rr64, _ = o64.sqmr(b64, tol=1e-8, maxit=200)
        t_solve64 = time.perf_counter() - t0
        ratio = t_solve64 / (it64 + 1) / t_s64  # one SQMR iteration (or the first V-cycle) in 64^3 smoothings
        o = oracle.Oracle(n, coarsest_max=8)
        b = o.rhs(synthetic.bumps(n, seed=0)["f"].numpy(), None)
        x0 = np.zeros(o.n())
        times = []
        for st in range(warmup + steps):
            t0 = time.perf_counter()
            o.smooth(x0, b, level=0)
            dt = time.perf_counter() - t0
            if st >= warmup:
                times.append(dt)
    finally:
        oracle.set_threads(1)
    if iters is None:
        iters = oracle_iterations(n) or 14
    t_smooth = float(np.mean(times))
    t_solve = t_smooth * ratio * (iters + 1)
    return {
        "value": unknowns(n) / t_solve, "unit": UNIT, "cores": used, "kind": "oracle",
        "sample": (f"one finest-level Alg. 3 smoothing of the {n}^3 problem (FP64 C oracle, {used} threads, "
                   f"{t_smooth:.2f} s per sample, {len(times)} timed); the solve's time is extrapolated as "
                   f"sample x {ratio:.2f} (one SQMR iteration in smoothings, from a timed full 64^3 solve) x "
                   f"{iters}+1 (the oracle's iterations for this workload)"),
        "seconds_per_sample": t_smooth, "est_solve_seconds": t_solve, "times": times, "x64": x64, "b64": b64,
        "full_solve_64": {"value": unknowns(64) / t_solve64, "unit": UNIT, "seconds": t_solve64, "iterations": it64,
                          "rel_residual": rr64, "status": rc64,
                          "meaning": "a complete oracle MG-SQMR solve of the 64^3 bump problem to 1e-8, timed"},
    }


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle timed on the host cores, on the native arm's workload.  Each
    timed step is one bounded sample (a finest-level smoothing of the 256^3 problem, all host threads);
    ms_per_step is that sample's measured time; value is the solve throughput extrapolated from it (see
    cpu_sample), and the line says so."""
    if rank != 0:
        return
    n = args.n
    cb = cpu_sample(n, steps=args.steps, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": cb["seconds_per_sample"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(n, world),
        "step": "one timed sample: a finest-level Alg. 3 smoothing of the %d^3 problem by the FP64 oracle" % n,
        "value_basis": "extrapolated: unknowns / (sample seconds x SQMR-iteration/smoothing ratio x (iterations+1))",
        "est_solve_seconds": cb["est_solve_seconds"],
        "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "full_solve_64": cb["full_solve_64"], "host": host_info(),
        "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def bench_config(n, world):
    """The workload description both arms print (precisions are in dtype, not here)."""
    return {"workload": workload_name(n), "n": n, "unknowns": unknowns(n), "levels": auto_levels(n), "tol": 1e-8,
            "l2": "inputs larger than L2 (each FP64 vector %d MB)" % (packed_len(n) * 8 // 2 ** 20),
            "parallelism": f"replicas x{world}"}


def auto_levels(n, coarsest_max=8):
    lev = 1
    while n % 2 == 0 and n > coarsest_max and n >= 4:
        n //= 2
        lev += 1
    return lev


# ------------------------------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in self.rows if len(r) > 8 for j in range(4) if r[5 + j] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------------------------------------ roofline

def alg_bytes(kind, n, e, launches_per_level0=1):
    """Algorithmic bytes of ONE level-0 launch of a kernel kind on the n^3 grid.

    Counted as compulsory traffic: every array the launch must read is read once, every array it
    writes is written once (e = element size of the V-cycle, FP64 = 8 for SQMR vectors).
    nf = face entries, np = cells, npk = nf + np (packed length)."""
    np_ = n ** 3
    npk = packed_len(n)
    nf = npk - np_
    v1 = n ** 3 - (n - 2) ** 3
    table = {
        "dgs_u": (3 * nf + np_) * e,              # read x faces, p, b faces; write x faces
        "dgs_p_bwd": (nf / 2 + 3 * np_ / 2) * e,  # g on the colour's face rows, p and h at radius 1, write p
        "dgs_p_bwd_prep": 3 * npk * e,            # read x, b; write g (faces) and h (cells)
        "dgs_p_fwd": (2 * nf / 4 + 3 * np_ / 4) * e,  # a colour touches 1/4 of the rows of faces and cells
        "dgs_p_gather": 3 * np_ * e,              # read delta, read+write p
        "residual": 3 * npk * e,                  # read x, b; write r
        "restrict": (npk + npk / 8) * e,
        "prolong": (2 * npk + npk / 8) * e,
        "memset": npk * e,
        "vanka_compute": v1 / 8 * 21 * e,         # b and x of the patch, 7 corrections written
        "vanka_apply": v1 / 8 * 21 * e,
        "apply_dot": 2 * npk * 8,
        "update_s": 3 * npk * 8 + (npk * e if e == 4 else 0),
        "dot2": npk * e + npk * 8,
        "update_x": 9 * npk * 8 + npk * e,
    }
    return table.get(kind)


# FP64 roof of the CUDA cores, derived from the nominal dense FP64 rate of this part (1.25 TFLOP/s: 2
# FP64 FMA per SM per cycle, 152 SMs, 2.07 GHz); an FMA is one DP instruction and 2 flops
FP64_NOMINAL_TFLOPS = 1.25
DP_INSTR_PEAK_G = FP64_NOMINAL_TFLOPS * 1e3 / 2


def roofline(prof, n, e, peak, traffic_db, precision, total_ms=None, fp64_measured_tflops=None):
    """Roofline entry of the kernel kind with the largest total time in prof.  share_of_iteration is
    that kind's share of the whole iteration's kernel time (total_ms; default: the sum over prof)."""
    kind = max(prof, key=lambda k: prof[k][0])
    ms_all, cnt_all, ms0, cnt0 = prof[kind]
    if cnt0 == 0:
        return None
    total = total_ms if total_ms else sum(v[0] for v in prof.values())
    avg_ms = ms0 / cnt0
    tr = traffic_db.get(f"{precision}:{kind}:{n}")
    if kind in ("apply_dot", "update_x"):
        # FP64 kernels of SQMR: bound by the DP pipe; count DP instructions (per packed entry: apply
        # ~9.25 = 3/4 face rows x 9 + 1/4 cell rows x 6 + the dot's DFMA; update_x 8)
        # (update_x: the critical r/q kernel and the deferred d/x kernel together, 5 + 3 per entry; the
        # kind's total time per iteration is the denominator)
        per = 9.25 if kind == "apply_dot" else 8.0
        npk = packed_len(n)
        achieved = per * npk / (ms0 * 1e-3) / 1e9
        out = {"kernel": kind, "bound": "alu", "achieved": achieved, "peak": DP_INSTR_PEAK_G,
               "peak_source": "nominal FP64 rate 1.25 TFLOP/s = 625 G DP instructions/s (2 DFMA/SM/cycle, 152 SMs, "
                              "2.07 GHz)",
               "unit": "G DP-instr/s", "frac": achieved / DP_INSTR_PEAK_G, "traffic": tr,
               "dp_instr_per_launch": per * npk, "avg_launch_ms": avg_ms, "launches_level0_per_iteration": cnt0,
               "share_of_iteration": ms_all / total}
        if fp64_measured_tflops:
            out["measured_fp64_tflops"] = fp64_measured_tflops
            out["frac_of_measured"] = achieved / (fp64_measured_tflops * 1e3 / 2)
        return out
    b = alg_bytes(kind, n, e)
    achieved = b / (avg_ms * 1e-3) / 1e9 if b else None
    return {"kernel": kind, "bound": "hbm", "achieved": achieved, "peak": peak[0],
            "peak_source": f"{peak[1]} hbm_gbs (MEASURED_PEAKS.json)" if peak[1] == "measured" else "fallback 6.8 TB/s",
            "unit": "GB/s", "frac": achieved / peak[0] if achieved else None, "traffic": tr,
            "traffic_over_algorithmic": (tr / b) if (tr and b) else None,
            "algorithmic_bytes_per_launch": b, "avg_launch_ms": avg_ms, "launches_level0_per_iteration": cnt0,
            "share_of_iteration": ms_all / total}


# ------------------------------------------------------------------------------------------ native arm

def apply_schedule(smg, S, sched):
    """Set every level's Vanka schedule, transfer tiles and DGS velocity form from a recorded choice."""
    for l in range(S.levels - 1):
        if l < len(sched.get("vanka", [])):
            mode, blocks = sched["vanka"][l]
            smg.stokes_set_level_schedule(S.h, l, mode, blocks)
        if l < len(sched.get("tiles", [])):
            rt, pt = sched["tiles"][l]
            smg.stokes_set_level_tiles(S.h, l, rt, pt)
        if l < len(sched.get("dgs_fused", [])):
            smg.stokes_set_level_dgs(S.h, l, sched["dgs_fused"][l])


def max_over_ranks(ms, dist, device):
    """The slowest rank's time in ms (the whole job ends with it); ms itself on one process."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def batch_problems(rank, count):
    """One rank's independent problems: cube sizes uniform over BATCH_SIZES (PCG64 seed 4000 + rank) and
    bump seeds rank * 100000 + i, disjoint across ranks (replicas: no data is exchanged)."""
    import numpy as np
    rng = np.random.default_rng(4000 + rank)
    return [int(v) for v in rng.choice(BATCH_SIZES, size=count)], [rank * 100000 + i for i in range(count)]


def whole_job_value(units_per_rank, world, ms):
    """Units per second of all ranks together, each rank having processed units_per_rank in ms."""
    return units_per_rank * world / (ms * 1e-3)


def run_e2e(smg, S, rhs_dev, npk, args, barrier, stream, world, n):
    """sqmr_solve through the C ABI with pinned HOST rhs / x0 / x: the H2D copies of the inputs and the
    D2H copy of the solution happen inside the call, inside the timed region."""
    import torch
    bh = torch.empty(npk, dtype=torch.float64, pin_memory=True)
    bh.copy_(rhs_dev.cpu())
    xh = torch.zeros(npk, dtype=torch.float64, pin_memory=True)
    for _ in range(max(1, args.warmup)):
        xh.zero_()
        smg.sqmr_solve(S.h, bh, xh, args.tol, 200)
    barrier()
    ms_e2e = 0.0
    for _ in range(args.steps):
        xh.zero_()  # the step's x0, prepared on the host outside the timed call
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        ev0.record(stream)
        smg.sqmr_solve(S.h, bh, xh, args.tol, 200)  # H2D of rhs and x0, solve, D2H of x, synchronised
        ev1.record(stream)
        barrier()
        ms_e2e += max(ev0.elapsed_time(ev1), (time.perf_counter() - t0) * 1e3)
    if world > 1:
        import torch.distributed as dist
        ms_e2e = max_over_ranks(ms_e2e, dist, "cuda")
    return {"value": whole_job_value(unknowns(n) * args.steps, world, ms_e2e), "unit": UNIT,
            "h2d_bytes_per_step": 2 * npk * 8, "d2h_bytes_per_step": npk * 8,
            "note": "sqmr_solve with pinned host rhs/x0/x, each call timed (its copies inside); the host "
                    "zeroing of x0 before each call is not timed"}


BATCH_SIZES = (32, 48, 64, 96, 128)


def run_batch(args, smg, synthetic, torch, dev, rank, world, dist):
    """Independent problems with cube sizes drawn uniformly from BATCH_SIZES (seeded per rank), Gaussian-bump
    forcing per problem, FP32 V-cycle + FP64 SQMR to args.tol.  Headline: the batched form -- the problems of
    each size in one batched handle (stokes_create_batch: one launch per V-cycle and SQMR step for all of
    them, the iteration one captured graph), the size classes concurrently on their own streams.  Beside
    it: sqmr_solve_batch (one handle per problem, args.streams concurrent streams), and the problems solved
    one after another (FP32 V-cycle, and the plain FP64 V-cycle).  A step returns once every problem has
    converged, so it is timed on the host with the device synchronised on both sides."""
    sizes, bump_seeds = batch_problems(rank, args.batch)
    S32, rhs, xs = [], [], []
    for i, n in enumerate(sizes):
        S = smg.Stokes(n, precision=smg.PREC_FP32)
        S32.append(S)
        rhs.append(S.rhs(synthetic.bumps(n, seed=bump_seeds[i], device=dev)["f"], None))
        xs.append(torch.zeros(S.n, dtype=torch.float64, device=dev))
    total_unknowns = sum(unknowns(n) for n in sizes)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def maxrank(ms):
        return max_over_ranks(ms, dist, dev)

    def batch_step():
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        return smg.sqmr_solve_batch([S.h for S in S32], rhs, xs, args.tol, 200, nstreams=args.streams)

    # the batched form: one handle per size class holding all problems of that size
    classes = sorted(set(sizes))
    members = {n: [i for i, m in enumerate(sizes) if m == n] for n in classes}
    BH = {n: smg.Stokes(n, precision=smg.PREC_FP32, batch=len(members[n])) if len(members[n]) > 1
          else smg.Stokes(n, precision=smg.PREC_FP32) for n in classes}
    cstreams = {n: torch.cuda.Stream(device=dev) for n in classes}

    def batched_step():
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos, done, errs = [None] * len(sizes), [0.0] * len(sizes), []

        def run(n):
            try:
                ii = members[n]
                if len(ii) > 1:
                    inf = smg.sqmr_solve_batched(BH[n].h, [rhs[i] for i in ii], [xs[i] for i in ii], args.tol, 200,
                                                 stream=cstreams[n])
                else:
                    inf = [smg.sqmr_solve(BH[n].h, rhs[ii[0]], xs[ii[0]], args.tol, 200, stream=cstreams[n])]
                t = (time.perf_counter() - t0) * 1e3
                for i, f in zip(ii, inf):
                    infos[i], done[i] = f, t
            except Exception as e:  # noqa: BLE001 -- re-raised below on the main thread
                errs.append(e)

        threads = [threading.Thread(target=run, args=(n,)) for n in classes]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        if errs:
            raise errs[0]
        return infos, done

    def timed(step):
        for _ in range(args.warmup):
            step()
        barrier()
        lat, its, res = [], [], []
        with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
            t0 = time.perf_counter()
            for _ in range(args.steps):
                infos, done = step()
                lat += done
                its.append([inf.iterations for inf in infos])
                res += [inf.rel_residual for inf in infos]
            barrier()
            ms = maxrank((time.perf_counter() - t0) * 1e3)
        assert all(r < args.tol for r in res), max(res)
        return ms, lat, its, clk

    ms, lat, its, clk = timed(batched_step)
    value = total_unknowns * args.steps * world / (ms * 1e-3)
    ms_st, lat_st, its_st, _ = timed(batch_step)
    value_st = total_unknowns * args.steps * world / (ms_st * 1e-3)

    def sequential(handles, k):
        durations = []
        barrier()
        t0 = time.perf_counter()
        for _ in range(k):
            for S, b, x in zip(handles, rhs, xs):
                t1 = time.perf_counter()
                x.zero_()
                smg.sqmr_solve(S.h, b, x, args.tol, 200)
                durations.append((time.perf_counter() - t1) * 1e3)
        barrier()
        return maxrank((time.perf_counter() - t0) * 1e3), durations

    sequential(S32, 1)  # warm
    ms_seq32, dur32 = sequential(S32, 1)
    S64 = [smg.Stokes(n, precision=smg.PREC_FP64) for n in sizes]
    sequential(S64, 1)
    ms_seq64, dur64 = sequential(S64, 1)
    for S in S64:
        S.close()
    # launches of the batched form: per class, its longest-running problem's iterations times the launches of
    # one iteration of the fixed batched schedule (profiled on a one-problem handle with the same schedule),
    # plus the per-problem setup and finish launches
    gpu_launches = 0
    for n in classes:
        P = smg.Stokes(n, precision=smg.PREC_FP32, autotune=False)
        prof = smg.stokes_profile_iteration(P.h)
        per_iter = sum(v[1] for v in prof.values())
        P.close()
        k = max(its[-1][i] for i in members[n])
        gpu_launches += k * per_iter + per_iter + 16 * len(members[n])
    for S in BH.values():
        S.close()
    if rank == 0:
        q = lambda a, p: float(np.percentile(np.asarray(a), p))
        line = {
            "metric": "batched solved unknowns/sec to rel. residual %g" % args.tol, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 SQMR + f32 V-cycle",
            "data": "synthetic",
            "config": {"workload": "batch of %d problems, n^3 cells with n drawn from %s, 16 Gaussian bumps each"
                                   % (args.batch, list(BATCH_SIZES)),
                       "sizes": sizes, "unknowns_per_batch": total_unknowns, "streams": args.streams, "tol": args.tol,
                       "timer": "host clock, device synchronised on both sides (the batch call blocks until done)",
                       "parallelism": f"replicas x{world}"},
            "form": "batched handles: one per size class (%s problems), one launch per V-cycle and SQMR step for "
                    "all problems of the class, the iteration one CUDA graph; the classes concurrently on %d streams"
                    % ({n: len(members[n]) for n in classes}, len(classes)),
            "iterations": its[-1],
            "latency_ms": {"p50": q(lat, 50), "p99": q(lat, 99), "max": max(lat),
                           "meaning": "time from the step's start to the problem's solution (its size class's end)"},
            "streams_path": {"value": value_st, "unit": UNIT, "ms_per_step": ms_st / args.steps,
                             "latency_ms": {"p50": q(lat_st, 50), "p99": q(lat_st, 99), "max": max(lat_st)},
                             "form": "sqmr_solve_batch: one handle per problem, %d host threads with a stream each"
                                     % args.streams},
            "sequential_fp32_vcycle": {"value": total_unknowns * world / (ms_seq32 * 1e-3), "unit": UNIT,
                                       "ms_per_batch": ms_seq32, "solve_ms_p50": q(dur32, 50), "solve_ms_p99": q(dur32, 99)},
            "sequential_fp64_vcycle": {"value": total_unknowns * world / (ms_seq64 * 1e-3), "unit": UNIT,
                                       "ms_per_batch": ms_seq64, "solve_ms_p50": q(dur64, 50), "solve_ms_p99": q(dur64, 99)},
            "gpu_launches": gpu_launches * args.steps, "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    for S in S32:
        S.close()


def labelled_unknowns(lab):
    """Unknowns of a label array (nz+2, ny+2, nx+2) (Sec. 5): interior cells, and faces with no Dirichlet
    cell beside them and an interior cell on at least one side (Neumann faces next to exterior cells
    included)."""
    it, dr = lab == 0, lab == 1
    cnt = int(it[1:-1, 1:-1, 1:-1].sum())
    for a, b in (((slice(1, -1), slice(1, -1), slice(1, -2)), (slice(1, -1), slice(1, -1), slice(2, -1))),
                 ((slice(1, -1), slice(1, -2), slice(1, -1)), (slice(1, -1), slice(2, -1), slice(1, -1))),
                 ((slice(1, -2), slice(1, -1), slice(1, -1)), (slice(2, -1), slice(1, -1), slice(1, -1)))):
        cnt += int(((it[a] | it[b]) & ~dr[a] & ~dr[b]).sum())
    return cnt


def run_cavity(args, smg, synthetic, torch, dev, rank, world, dist):
    """3D lid-driven cavity (Sec. 7): n^3 cells, lid u = 1 on the top, no slip elsewhere, or (porous) a
    box of random spherical Dirichlet obstacles with a flux-balanced plug inflow/outflow along x and
    Gaussian-bump forcing; eta = gamma = 1e-3, from x0 = 0 to args.tol; FP32 V-cycle + FP64 SQMR beside
    the plain FP64 V-cycle."""
    n = args.n
    labels = None
    if args.mode == "porous":
        labels = synthetic.porous_labels(n, seed=0)
        prob = {"f": synthetic.bumps(n, seed=0, device=dev)["f"],
                "g": synthetic.plug_flow(n, labels=labels, device=dev)}
        nunk = labelled_unknowns(labels)
        workload = "3D porous medium %d^3 (12 random spherical obstacles, %.1f%% of the cells), plug flow " \
                   "along x + bump forcing, eta = gamma = 1e-3" % (n, 100.0 * (labels[1:-1, 1:-1, 1:-1] == 1).mean())
        metric = "solved unknowns/sec to rel. residual %g, 3D porous medium" % args.tol
    else:
        prob = synthetic.lid(n, device=dev)
        nunk = unknowns(n)
        workload = "3D lid-driven cavity %d^3, eta = gamma = 1e-3" % n
        metric = "solved unknowns/sec to rel. residual %g, 3D lid-driven cavity" % args.tol
    res = {}
    for name, prec in (("fp32_vcycle", smg.PREC_FP32), ("fp64_vcycle", smg.PREC_FP64)):
        S = smg.Stokes(n, viscosity=1e-3, gamma=1e-3, precision=prec, labels=labels)
        b = S.rhs(prob["f"], prob["g"])
        x = torch.zeros_like(b)
        for _ in range(args.warmup):
            x.zero_()
            smg.sqmr_solve(S.h, b, x, args.tol, 400)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        its = []
        e0.record(stream)
        for _ in range(args.steps):
            x.zero_()
            info = smg.sqmr_solve(S.h, b, x, args.tol, 400)
            its.append((info.iterations, info.rel_residual))
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
        res[name] = {"value": whole_job_value(nunk * args.steps, world, ms), "ms_per_step": ms / args.steps,
                     "iterations": [i for i, _ in its], "rel_residual": [r for _, r in its], "levels": S.levels}
        S.close()
    if rank == 0:
        h = res["fp32_vcycle"]
        line = {"metric": metric,
                "value": h["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": h["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64 SQMR + f32 V-cycle", "data": "synthetic",
                "config": {"workload": workload, "n": n,
                           "unknowns": nunk, "tol": args.tol, "parallelism": f"replicas x{world}"},
                "fp32_vcycle": h, "fp64_vcycle": res["fp64_vcycle"]}
        print(json.dumps(line), flush=True)


def run_warmstart(args, smg, synthetic, torch, dev, rank, world):
    """Learned initial guess: args.train + args.test problems (n^3, 8 Gaussian bumps each, seeds
    20000 + i); every problem is solved by the method (FP32 V-cycle, FP64 SQMR, tol 1e-8) to give the
    training targets; the network (BF16 activations, FP32 accumulation) is trained with Adam for
    args.epochs passes (loss chosen by --ws-loss); on the held-out seeds the solve from the network's guess is timed against the
    solve from x0 = 0 (same handle, same tolerance)."""
    import numpy as np
    n = args.n
    S = smg.Stokes(n, precision=smg.PREC_FP32)
    npk = S.n
    seeds = [20000 + rank * 1000000 + i for i in range(args.train + args.test)]

    def rhs(sd):
        return S.rhs(synthetic.bumps(n, seed=sd, nbumps=8, device=dev)["f"], None)

    t0 = time.perf_counter()
    xs_store = torch.empty((len(seeds), npk), dtype=torch.float32, device=dev)
    its0 = []
    ratio = []
    for i, sd in enumerate(seeds):
        b = rhs(sd)
        x = torch.zeros_like(b)
        info = smg.sqmr_solve(S.h, b, x, 1e-8, 200)
        its0.append(info.iterations)
        xs_store[i] = x.float()
        if i < 64:
            ratio.append(float(x.norm() / b.norm()))
    gen_s = time.perf_counter() - t0
    scale = float(np.median(ratio))  # ||x*|| / ||b||: the network's output is scale * ||b|| * O(1)
    ws = smg.WarmStart(n, smg.STORE_BF16, scale=scale)
    w_init = synthetic.net_weights(7).astype(np.float32)
    w_init[-16 * 4:] = 0.0  # zero output layer: training starts from x0 = 0 (loss 1) and only improves on it
    ws.set_weights(w_init)
    steps = args.epochs * args.train
    rng = np.random.default_rng(5)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    losses = []
    for st in range(steps):
        i = int(rng.integers(args.train))
        lr = 1e-3 * 0.5 * (1 + np.cos(np.pi * st / steps))  # cosine decay
        b = rhs(seeds[i])
        want = st % 200 == 0 or st == steps - 1
        loss = ws.train_step(b, xs_store[i].double(), lr, S=S if args.ws_loss == "residual" else None, want_loss=want)
        if want:
            losses.append((st, loss))
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    # the network's forward pass on each engine (CUDA events, 20 passes after 3 warm-up passes)
    stream = torch.cuda.current_stream()
    b_probe = rhs(seeds[0])
    x_probe = torch.empty_like(b_probe)
    predict_ms = {}
    for name, eng in (("tensor_cores", 1), ("cuda_cores", 0)):
        ws.set_engine(eng)
        for _ in range(3):
            ws.predict(b_probe, x_probe)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(20):
            ws.predict(b_probe, x_probe)
        ev1.record(stream)
        torch.cuda.synchronize()
        predict_ms[name] = ev0.elapsed_time(ev1) / 20
    ws.set_engine(1)
    conv_flop = 2 * 27 * 16 * (4 * n ** 3 + 16 * (2 * n ** 3 + 3 * (n // 2) ** 3 + 3 * (n // 4) ** 3 + 2 * (n // 8) ** 3))
    # held-out evaluation
    rows = []
    for k in range(args.test):
        i = args.train + k
        b = rhs(seeds[i])
        xstar = xs_store[i].double()
        x = torch.zeros_like(b)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize()
        e0.record(stream)
        info0 = smg.sqmr_solve(S.h, b, x, 1e-8, 200)
        e1.record(stream)
        xw, infow, used = ws.solve(S, b, tol=1e-8, check=False)
        e2.record(stream)
        torch.cuda.synchronize()
        x0 = ws.predict(b)
        err = float((x0 - xstar).norm() / xstar.norm())
        rows.append((info0.iterations, e0.elapsed_time(e1), infow.iterations, e1.elapsed_time(e2), used, err,
                     infow.rel_residual if infow.status == 0 else float("inf")))
    r = np.array([[a, b_, c, d, float(e), f, g] for a, b_, c, d, e, f, g in rows])
    if rank == 0:
        line = {
            "metric": "solved unknowns/sec to rel. residual 1e-8, learned initial guess vs x0 = 0",
            "value": unknowns(n) * world / (r[:, 3].mean() * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.test, "warmup": 1, "ms_per_step": float(r[:, 3].mean()), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 net (f32 acc) + f32 V-cycle + f64 SQMR",
            "data": "synthetic",
            "config": {"workload": "%d^3 box, 8 Gaussian bumps per seed; %d training solves, %d held-out seeds"
                                   % (n, args.train, args.test), "n": n, "epochs": args.epochs,
                       "network": "4 levels, 16 channels, 3x3x3 convolutions, leaky ReLU 0.1, no bias",
                       "loss": ("||L (x0 - x*)||^2 / ||b||^2" if args.ws_loss == "residual" else
                                "||x0 - x*||^2 / ||x*||^2") + ", Adam, cosine-decayed lr from 1e-3, output layer "
                               "initialised to 0",
                       "parallelism": f"replicas x{world}"},
            "x0_zero": {"iterations_mean": float(r[:, 0].mean()), "ms_mean": float(r[:, 1].mean()),
                        "value": unknowns(n) / (r[:, 1].mean() * 1e-3)},
            "learned_x0": {"iterations_mean": float(r[:, 2].mean()), "ms_mean": float(r[:, 3].mean()),
                           "value": unknowns(n) / (r[:, 3].mean() * 1e-3), "guess_used": float(r[:, 4].mean()),
                           "x0_rel_error_mean": float(r[:, 5].mean()), "max_rel_residual": float(r[:, 6].max())},
            "network_forward": {"ms_tensor_cores": predict_ms["tensor_cores"], "ms_cuda_cores": predict_ms["cuda_cores"],
                                "conv_gflop": conv_flop * 1e-9,
                                "conv_tflops_tensor_cores": conv_flop / (predict_ms["tensor_cores"] * 1e-3) * 1e-12,
                                "engine": "BF16 tensor cores (tcgen05 convolution, mma.sync weight gradient)"},
            "training": {"solves_s": gen_s, "train_s": train_s, "steps": steps, "ms_per_step": train_s * 1e3 / steps,
                         "loss_trace": losses[:: max(1, len(losses) // 12)] + losses[-1:],
                         "data_iterations_mean": float(np.mean(its0))},
        }
        print(json.dumps(line), flush=True)
    ws.close()
    S.close()


def run_variants(args, smg, synthetic, torch, dev, rank, world, dist):
    """The method's variants on the headline workload (n^3 bumps, FP32 V-cycle, FP64 SQMR, tol): k_b = 1, 2, 3
    symmetric Vanka sweeps (Alg. 3), the W-cycle (Sec. 8.2), the damped additive Vanka (Eq. av) and the
    symmetric distributive weighted Jacobi (Sec. 3.1)."""
    n = args.n
    rows = []
    for name, kw in [("V, k_b=1 (default)", {}), ("V, k_b=2", {"kb_vanka": 2}), ("V, k_b=3", {"kb_vanka": 3}),
                     ("W, k_b=1", {"cycle": 2}), ("V, additive Vanka, k_b=1", {"additive": True}),
                     ("V, additive Vanka, k_b=3", {"additive": True, "kb_vanka": 3}),
                     ("V, distributive weighted Jacobi", {"dwj": True})]:
        S = smg.Stokes(n, precision=smg.PREC_FP32, **kw)
        b = S.rhs(synthetic.bumps(n, seed=0, device=dev)["f"], None)
        x = torch.zeros_like(b)
        for _ in range(args.warmup):
            x.zero_()
            smg.sqmr_solve(S.h, b, x, args.tol, 200, check=False)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        its = []
        e0.record(stream)
        for _ in range(args.steps):
            x.zero_()
            info = smg.sqmr_solve(S.h, b, x, args.tol, 200, check=False)
            its.append((info.iterations, info.rel_residual, info.status))
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        rows.append({"variant": name, "value": unknowns(n) / (ms * 1e-3), "ms_per_solve": ms,
                     "iterations": its[-1][0], "rel_residual": its[-1][1], "status": its[-1][2]})
        S.close()
    if rank == 0:
        base = rows[0]
        line = {"metric": "solved unknowns/sec to rel. residual %g, smoother and cycle variants" % args.tol,
                "value": base["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": base["ms_per_solve"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64 SQMR + f32 V-cycle", "data": "synthetic",
                "config": {"workload": workload_name(n), "n": n, "tol": args.tol, "parallelism": f"replicas x{world}"},
                "variants": rows}
        print(json.dumps(line), flush=True)


def run_comparators(args, smg, synthetic, torch, dev, rank, world, dist):
    """The paper's comparison (Sec. 6, Sec. 7): MG-preconditioned SQMR beside Alg. 1 iterated outright on L~
    (pure multigrid, FP32 cycle, FP64 residual) and SQMR without preconditioner (FP64), on the n^3 bump box
    and on the porous domain (eta = gamma = 1e-3).  One timed solve each after one warm-up solve; the plain
    SQMR is capped at --plain-iters iterations."""
    n = args.n
    lab = synthetic.porous_labels(n, seed=0)
    cases = [("box bumps, eta = 1", None, 1.0, synthetic.bumps(n, seed=0, device=dev)["f"], None, unknowns(n)),
             ("porous, plug flow + bumps, eta = 1e-3", lab, 1e-3, synthetic.bumps(n, seed=0, device=dev)["f"],
              synthetic.plug_flow(n, labels=lab, device=dev), labelled_unknowns(lab))]
    rows = []
    stream = torch.cuda.current_stream()
    for cname, labels, eta, f, g, nunk in cases:
        for solver, prec, cap in (("MG-preconditioned SQMR", smg.PREC_FP32, 400),
                                  ("pure multigrid on L~", smg.PREC_FP32, 400),
                                  ("SQMR, no preconditioner", smg.PREC_FP64, args.plain_iters)):
            S = smg.Stokes(n, viscosity=eta, gamma=1e-3, precision=prec, labels=labels)
            b = S.rhs(f, g)
            x = torch.zeros_like(b)
            fn = {"MG-preconditioned SQMR": smg.sqmr_solve, "pure multigrid on L~": smg.mg_solve,
                  "SQMR, no preconditioner": smg.sqmr_solve_unpreconditioned}[solver]
            fn(S.h, b, x, args.tol, cap if solver != "SQMR, no preconditioner" else 20, check=False)
            x.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = fn(S.h, b, x, args.tol, cap, check=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            rows.append({"case": cname, "solver": solver, "precision": "fp32 cycle" if prec == smg.PREC_FP32 else "fp64",
                         "iterations": info.iterations, "status": smg.stokes_strerror(info.status) if info.status else "ok",
                         "rel_residual": info.rel_residual, "ms": ms,
                         "value": nunk / (ms * 1e-3) if info.status == 0 else None})
            S.close()
    if rank == 0:
        base = rows[0]
        line = {"metric": "solved unknowns/sec to rel. residual %g, MG-SQMR against pure multigrid and plain SQMR"
                          % args.tol,
                "value": base["value"], "unit": UNIT, "n_gpus": world, "steps": 1, "warmup": 1,
                "ms_per_step": base["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64 SQMR + f32 V-cycle", "data": "synthetic",
                "config": {"workload": "%d^3 box (16 bumps, eta = 1) and %d^3 porous medium (eta = gamma = 1e-3)"
                                       % (n, n), "n": n, "tol": args.tol, "plain_sqmr_cap": args.plain_iters,
                           "parallelism": f"replicas x{world}"},
                "solvers": rows}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n", "--cells", dest="n", type=int, default=None,
                    help="cells per axis (default 256; 128 for --mode cavity, warmstart, comparators); --cells is the "
                         "spelling to use under torchrun, whose own options start with --n")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 V-cycle solve beside the headline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffer) measurement")
    ap.add_argument("--no-bf16", action="store_true", help="skip the BF16-storage V-cycle solve beside the headline")
    ap.add_argument("--no-autotune", action="store_true",
                    help="per-colour Vanka launches on every level (profiler runs: timings under a profiler would "
                         "steer the autotuner)")
    ap.add_argument("--train", type=int, default=2000, help="training solves (--mode warmstart)")
    ap.add_argument("--test", type=int, default=200, help="held-out seeds (--mode warmstart)")
    ap.add_argument("--epochs", type=int, default=2, help="passes over the training solves (--mode warmstart)")
    ap.add_argument("--ws-loss", default="residual", choices=["error", "residual"],
                    help="training loss of --mode warmstart: ||x0 - x*||^2/||x*||^2 or ||L (x0 - x*)||^2/||b||^2")
    ap.add_argument("--mode", default="solve", choices=["solve", "vcycle", "batch", "cavity", "porous", "warmstart", "variants",
                                                     "comparators"],
                    help="vcycle: only time mg_precondition (one V-cycle per step) -- for profiler captures; "
                         "batch: independent problems of uneven sizes solved concurrently; "
                         "cavity: the 3D lid-driven cavity (eta = gamma = 1e-3); "
                         "porous: spherical Dirichlet obstacles given by cell labels, plug flow along x; "
                         "comparators: MG-SQMR against pure multigrid and plain SQMR (Sec. 6); "
                         "warmstart: train the initial-guess network on solves, then solve held-out seeds; "
                         "variants: k_b sweeps, W-cycle and additive Vanka on the headline workload")
    ap.add_argument("--plain-iters", type=int, default=3000, help="iteration cap of plain SQMR (--mode comparators)")
    ap.add_argument("--batch", type=int, default=64, help="problems per batch (--mode batch)")
    ap.add_argument("--streams", type=int, default=8, help="concurrent streams / host threads (--mode batch)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"], help="V-cycle precision of --mode vcycle")
    ap.add_argument("--schedule", default=None,
                    help="JSON of per-level schedule choices (vanka, tiles, dgs_fused) to apply instead of the "
                         "autotuner's, e.g. profiles/schedule_solve256_fp32.json -- for profiler runs, whose "
                         "timings would steer the autotuner")
    ap.add_argument("--host-loop", action="store_true",
                    help="drive the SQMR loop from the host, one iteration graph at a time, instead of the device-side "
                         "loop graph -- for profiler runs, which list the kernels of every iteration this way")
    args = ap.parse_args()
    if args.n is None:
        args.n = 128 if args.mode in ("cavity", "warmstart", "comparators") else 256

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import paper_2312_10615_gb300 as smg
    import synthetic

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    n = args.n
    npk = packed_len(n)
    if args.mode == "vcycle":
        S = smg.Stokes(n, precision=smg.PREC_FP32 if args.precision == "fp32" else smg.PREC_FP64,
                       autotune=not args.no_autotune)
        sv = S.rhs(synthetic.bumps(n, seed=0, device=dev)["f"], None)
        tv = torch.empty_like(sv)
        for _ in range(args.warmup):
            smg.mg_precondition(S.h, sv, tv)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            smg.mg_precondition(S.h, sv, tv)
        e1.record()
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"mode": "vcycle", "n": n, "precision": args.precision, "steps": args.steps,
                              "ms_per_vcycle": e0.elapsed_time(e1) / args.steps}), flush=True)
        S.close()
        return
    if args.mode == "batch":
        run_batch(args, smg, synthetic, torch, dev, rank, world, dist)
        return
    if args.mode in ("cavity", "porous"):
        run_cavity(args, smg, synthetic, torch, dev, rank, world, dist)
        return
    if args.mode == "warmstart":
        run_warmstart(args, smg, synthetic, torch, dev, rank, world)
        return
    if args.mode == "variants":
        run_variants(args, smg, synthetic, torch, dev, rank, world, dist)
        return
    if args.mode == "comparators":
        run_comparators(args, smg, synthetic, torch, dev, rank, world, dist)
        return
    seeds = [(rank * 1000 + s) % 5 for s in range(5)]
    rhs = {}
    S32 = smg.Stokes(n, precision=smg.PREC_FP32, autotune=not (args.no_autotune or args.schedule))
    if args.schedule:
        apply_schedule(smg, S32, json.load(open(args.schedule)))
    if args.host_loop:
        smg.stokes_set_device_loop(S32.h, False)
    for sd in sorted(set(seeds)):
        rhs[sd] = S32.rhs(synthetic.bumps(n, seed=sd, device=dev)["f"], None)
    x = torch.zeros(npk, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(S, k, w, collect):
        for s in range(w):
            x.zero_()
            smg.sqmr_solve(S.h, rhs[seeds[s % len(seeds)]], x, args.tol, 200)
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for s in range(k):
            x.zero_()
            info = smg.sqmr_solve(S.h, rhs[seeds[s % len(seeds)]], x, args.tol, 200)
            collect.append((info.iterations, info.rel_residual))
        ev1.record(stream)
        barrier()
        return max_over_ranks(ev0.elapsed_time(ev1), dist, dev)

    # headline: FP32 V-cycle, FP64 SQMR
    its32 = []
    with ClockSampler(local) as clk:
        ms32 = timed(S32, args.steps, args.warmup, its32)
    assert all(r < args.tol for _, r in its32), its32
    value = whole_job_value(unknowns(n) * args.steps, world, ms32)

    prof32 = smg.stokes_profile_iteration(S32.h)
    launches_iter = sum(v[1] for v in prof32.values())
    launches_vc = launches_iter - sum(prof32[k][1] for k in ("apply_dot", "update_s", "dot2", "update_x", "scalars"))
    fixed = 16  # masks, norms, initial residual, first V-cycle bookkeeping, final mean removal and check
    gpu_launches = sum(it * launches_iter + launches_vc + fixed for it, _ in its32)

    peak = read_peaks()
    traffic_db = {}
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tp):
        traffic_db = json.load(open(tp))
    fp64_tflops = smg.stokes_measure_fma_peak(True) / 1e12
    iter_ms = sum(v[0] for v in prof32.values())
    roof = roofline(prof32, n, 4, peak, traffic_db, "fp32", iter_ms, fp64_tflops)
    # the streaming kernel with the largest share, for context beside the dominant one
    stream_kinds = {k: v for k, v in prof32.items() if k in ("dgs_u", "dgs_p_bwd_prep", "residual", "prolong")}
    roof_stream = roofline(stream_kinds, n, 4, peak, traffic_db, "fp32", iter_ms) if stream_kinds else None
    # every kind of the iteration against its own roof (algorithmic bytes or DP instructions), for the record
    roof_all = {k: roofline({k: v}, n, 4, peak, traffic_db, "fp32", iter_ms, fp64_tflops)
                for k, v in prof32.items() if v[3] > 0 and (alg_bytes(k, n, 4) or k in ("apply_dot", "update_x"))}

    # symmetry of the preconditioner as applied (SQMR assumes a symmetric one): |x.My - y.Mx| / (|x| |My|) on
    # two seeded vectors that vanish off the unknowns (themselves V-cycle outputs)
    def asymmetry(S):
        g = torch.Generator(device=dev).manual_seed(123)
        r1 = torch.randn(npk, dtype=torch.float64, device=dev, generator=g)
        r2 = torch.randn(npk, dtype=torch.float64, device=dev, generator=g)
        xv, yv = S.precondition(r1), S.precondition(r2)
        mx, my = S.precondition(xv), S.precondition(yv)
        return float(abs(torch.dot(xv, my) - torch.dot(yv, mx)) / (torch.linalg.norm(xv) * torch.linalg.norm(my)))
    asym = {"fp32_vcycle": asymmetry(S32)}

    # e2e through the C ABI with pinned host buffers: H2D of rhs and x0, D2H of x inside the timed region
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(smg, S32, rhs[seeds[0]], npk, args, barrier, stream, world, n)

    # the plain FP64 V-cycle beside it
    fp64 = None
    if not args.no_fp64:
        S64 = smg.Stokes(n, precision=smg.PREC_FP64)
        its64 = []
        ms64 = timed(S64, max(1, args.steps // 2), 1, its64)
        prof64 = smg.stokes_profile_iteration(S64.h)
        asym["fp64_vcycle"] = asymmetry(S64)
        k64 = max(prof64, key=lambda k: prof64[k][0])
        # error of the mixed-precision solution against the plain FP64 GPU run on the same right-hand side
        xa, xb = torch.zeros_like(x), torch.zeros_like(x)
        smg.sqmr_solve(S32.h, rhs[seeds[0]], xa, args.tol, 200)
        smg.sqmr_solve(S64.h, rhs[seeds[0]], xb, args.tol, 200)
        diff_max = float(torch.max(torch.abs(xa - xb)) / torch.max(torch.abs(xb)))
        diff_l2 = float(torch.linalg.norm(xa - xb) / torch.linalg.norm(xb))
        del xa, xb
        fp64 = {"value": unknowns(n) * len(its64) * world / (ms64 * 1e-3), "unit": UNIT,
                "ms_per_step": ms64 / len(its64), "iterations": [it for it, _ in its64],
                "rel_residual": [r for _, r in its64], "dominant_kernel": k64,
                "fp32_vcycle_solution_rel_diff": {"max": diff_max, "l2": diff_l2,
                                                  "meaning": "FP32-V-cycle solve vs this FP64-V-cycle solve, "
                                                             "same right-hand side, both to the tolerance"},
                "kernel_ms_per_iteration": {k: round(v[0], 4) for k, v in prof64.items()}}
        S64.close()

    # BF16 storage of the level operands on the two finest levels, FP32 arithmetic
    bf = None
    if not args.no_bf16:
        Sb = smg.Stokes(n, precision=smg.PREC_MIXED_BF16)
        itsb = []
        msb = timed(Sb, args.steps, 1, itsb)
        asym["bf16_storage_vcycle"] = asymmetry(Sb)
        xa, xb = torch.zeros_like(x), torch.zeros_like(x)
        smg.sqmr_solve(Sb.h, rhs[seeds[0]], xa, args.tol, 200)
        smg.sqmr_solve(S32.h, rhs[seeds[0]], xb, args.tol, 200)
        bf = {"value": unknowns(n) * len(itsb) * world / (msb * 1e-3), "unit": UNIT, "ms_per_step": msb / len(itsb),
              "iterations": [it for it, _ in itsb], "rel_residual": [r for _, r in itsb],
              "solution_rel_diff_vs_fp32_vcycle": {"max": float(torch.max(torch.abs(xa - xb)) / torch.max(torch.abs(xb))),
                                                   "l2": float(torch.linalg.norm(xa - xb) / torch.linalg.norm(xb))}}
        del xa, xb
        Sb.close()

    cpu = None
    acc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # all host threads, and one thread (the oracle's results are the same for both)
        cb = cpu_sample(n)
        cb1 = cpu_sample(n, threads=1)
        cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        cpu["single_thread"] = {k: cb1[k] for k in ("value", "unit", "cores", "sample")}
        cpu["full_solve_64"] = {"all_threads": cb["full_solve_64"], "single_thread": cb1["full_solve_64"]}
        cpu["host"] = host_info()
        # accuracy of the mixed-precision V-cycles against the oracle's 1e-8 solve of the 64^3 bump problem
        acc = {}
        bt = torch.from_numpy(cb["b64"]).to(dev)
        for pname, prec in (("fp32_vcycle", smg.PREC_FP32), ("bf16_storage_vcycle", smg.PREC_MIXED_BF16)):
            Sa = smg.Stokes(64, precision=prec)
            xa, ia = Sa.solve(bt, tol=1e-8, max_iter=200)
            xa = xa.cpu().numpy()
            acc[pname] = {"max_rel_error_vs_oracle": float(np.max(np.abs(xa - cb["x64"])) / np.max(np.abs(cb["x64"]))),
                          "iterations": ia.iterations, "oracle_iterations": cb["full_solve_64"]["iterations"]}
            Sa.close()
        acc.update({"tol": 1e-8, "target": 1e-7, "tolerance_needed_for_target": 1e-8 if all(
            v["max_rel_error_vs_oracle"] <= 1e-7 for v in acc.values() if isinstance(v, dict)) else None,
            "workload": "64^3 bump problem, both solved to relative residual 1e-8"})

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms32 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 SQMR + f32 V-cycle", "data": "synthetic",
            "config": bench_config(n, world), "vcycle_precision": "fp32", "sqmr_precision": "fp64",
            "vanka_schedule_per_level": [dict(zip(("mode", "blocks", "ms_per_sweep"), smg.stokes_level_schedule(S32.h, l)))
                                         for l in range(S32.levels - 1)],
            "transfer_tiles_per_level": [dict(zip(("restrict", "prolong", "ms"), smg.stokes_level_tiles(S32.h, l)))
                                         for l in range(S32.levels - 1)],
            "dgs_velocity_per_level": [dict(zip(("fused", "ms_in_place_vs_fused"), smg.stokes_level_dgs(S32.h, l)))
                                       for l in range(S32.levels - 1)],
            "iterations": [it for it, _ in its32], "rel_residual": [r for _, r in its32],
            "kernel_ms_per_iteration": {k: round(v[0], 4) for k, v in prof32.items()},
            "kernel_ms_per_iteration_level0": {k: round(v[2], 4) for k, v in prof32.items()},
            "fp64_vcycle": fp64, "bf16_storage_vcycle": bf, "roofline": roof, "roofline_streaming_kernel": roof_stream,
            "roofline_per_kernel": {k: {kk: v[kk] for kk in ("bound", "achieved", "unit", "frac", "traffic",
                                                              "share_of_iteration") if kk in v}
                                    for k, v in roof_all.items() if v},
            "fp64_fma_measured_tflops": fp64_tflops,
            "preconditioner_asymmetry": dict(asym, meaning="|x.My - y.Mx| / (|x| |My|), M the V-cycle as applied"),
            "cpu_baseline": cpu, "accuracy_64": acc, "e2e": e2e,
            "gpu_launches": gpu_launches, "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    S32.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
