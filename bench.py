"""Benchmark of the GB300 CR-Solver hot path: beam-search IK (Algorithm 1) on the 3-segment,
9-tendon robot, 4096 full-pose targets per GPU, 256 seeds -> 64 projected-gradient steps (FP32,
adjoint) -> top 8 -> 30 LM iterations (FP64 Cholesky) -> FP64 acceptance at <= 1 mm / <= 1 deg.

Prints ONE JSON line (rank 0). `value` = IK solves/s over all GPUs with inputs resident in HBM;
`e2e` = the same through the host-buffer API (pinned H2D of the targets, D2H of the results inside
the timed region). `roofline` reports the stage-one kernel (the dominant kernel) against the FP32
ALU peak. `--impl reference` times the FP64 CPU oracle on host cores on the same workload.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun, one rank per GPU, each solving its own 4096 targets (weak scaling).
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

from paper_2607_11340_gb300 import synth  # noqa: E402

METRIC = "IK solves/s at <=1mm/<=1deg (batched FP32+adjoint two-stage beam search)"
UNIT = "solves/s"
WORKLOAD = "ik_3seg_9tendon_4096targets_256seeds_pg64_top8_lm30"
SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128
MUFU_PER_SM = 16
# DRAM bytes (read + write) of one stage-one call per target (k_ik_stage1 + k_ik_select, the pair the
# bench times), from an ncu capture of both kernels at 608 targets (dram__bytes_read.sum +
# dram__bytes_write.sum: 77,312 B + 6,872,320 B; ncu flushes the caches between kernels, so
# SelectTop's read of the seeds' end states comes from DRAM there, from L2 in a live step); traffic
# grows in proportion to the targets (each target reads its pose and its 256 end states).
STAGE1_DRAM_BYTES_PER_TARGET = (77312 + 6872320) / 608


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-baseline", action="store_true",
                    help="skip the CPU oracle sample (and, for the ragged batch, the per-problem comparison)")
    ap.add_argument("--targets", type=int, default=synth.P_3SEG, help="targets per GPU (default 4096)")
    ap.add_argument("--items", type=int, default=synth.N_RAGGED,
                    help="items of the ragged batch (default 16384; smaller for profiling cases)")
    ap.add_argument("--paths", type=int, default=synth.P_PATH,
                    help="path workload: paths (default 512; smaller for profiling cases)")
    ap.add_argument("--breakdown", action="store_true",
                    help="ragged workload: also time the batch's IK items and its path items (n <= 3, n >= 4) as "
                         "batches of their own")
    ap.add_argument("--workload", default="ik3",
                    choices=["ik3", "ik1", "path", "traj", "shelf", "prm", "calib", "ragged", "e1", "e2", "self"],
                    help="ik3: the headline two-stage IK; the others time the other workloads")
    return ap.parse_args()


def load_counts(key="ik_3seg_pose"):
    with open(os.path.join(ROOT, "tests", "golden", "opcounts.json")) as f:
        return json.load(f)[key]


def method_ops(c, n_seed, k_init, accepted):
    """The method's own work in stage one (oracle op counts): every seed's first value and gradient
    with all rows; at each of the k_init steps the step rule's arithmetic and a value at the
    projected trial point, without the rows that vanish there; a gradient only where the trial is
    accepted. Returns (flops, special-function calls)."""
    flop = (n_seed * (c["fwd_flop"] + c["tan_flop"]) + n_seed * k_init * (c["trial_fwd_flop"] + c["pg_step_flop"])
            + accepted * c["trial_tan_flop"])
    sfu = (n_seed * (c["fwd_sfu"] + c["tan_sfu"]) + n_seed * k_init * (c["trial_fwd_sfu"] + c["pg_step_sfu"])
           + accepted * c["trial_tan_sfu"])
    return flop, sfu


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_targets(torch, api, lib, spec, P, seed, device):
    """Full-pose targets [7][P] (FP64, device) from FK of hexagon-uniform states, via the CUDA FK."""
    rng = np.random.default_rng(seed)
    u_true = synth.hexagon_states(rng, P, spec.n, spec.umax)
    ug = torch.as_tensor(u_true.T.copy(), dtype=torch.float64, device=device)
    T, _ = api.fk(api.robot_struct(spec), ug)
    tg = synth.pose_targets(T.cpu().numpy().T, "pose")
    return tg


def cpu_oracle_rate(tg, spec, ik, budget_s=12.0, p0=0, threads=None, spheres=None, weights=synth.WEIGHTS, kind=None):
    """Oracle solves/s on host cores over a bounded contiguous sample of the targets."""
    import oracle as O

    O.build()
    rb = O.make_robot(list(spec.L), spec.rc, spec.umax, thmax=spec.thmax, nb=spec.nb, rbody=spec.body_radius,
                      lmin=spec.lmin, lmax=spec.lmax)
    W = O.make_weights(**weights.as_dict())
    threads = threads or os.cpu_count()
    cfg = O.IkConfig(S=ik.S, n_final=ik.n_final, k_init=ik.k_init, k_final=ik.k_final, lambda0=ik.lambda0,
                     alpha0=ik.alpha0, dedup_eps=ik.dedup_eps, lim_tol=ik.lim_tol, pos_tol=ik.pos_tol,
                     rot_tol=ik.rot_tol, seed=ik.seed, p0=p0)
    kind = O.IK6 if kind is None else kind
    n = max(threads, 16)
    t0 = time.perf_counter()
    r = O.solve_ik(rb, W, spheres, kind, tg[:n], cfg, threads=threads)
    dt = time.perf_counter() - t0
    done = n
    res = [r]
    while dt < budget_s and done < len(tg):
        m = min(len(tg) - done, max(threads, int(done / dt * (budget_s - dt))))
        cfg.p0 = p0 + done
        t1 = time.perf_counter()
        res.append(O.solve_ik(rb, W, spheres, kind, tg[done:done + m], cfg, threads=threads))
        dt += time.perf_counter() - t1
        done += m
    succ = np.concatenate([x["success"] for x in res])
    u = np.concatenate([x["u"] for x in res])
    return done / dt, done, threads, dt, succ, u


def oracle_sample(run, n_total, unit, what, budget_s=12.0, threads=None):
    """The oracle on host cores over a bounded contiguous sample: run(lo, hi, threads) solves problems
    [lo, hi) (seed counters from lo) and returns their success flags; chunks of at least one problem
    per thread until budget_s of wall time is spent. Returns the cpu_baseline object."""
    threads = threads or os.cpu_count()
    done, dt, succ = 0, 0.0, []
    while done < n_total and (done == 0 or dt < budget_s):
        m = min(n_total - done, threads if done == 0 else max(threads, int(done / dt * (budget_s - dt))))
        t0 = time.perf_counter()
        succ.append(np.asarray(run(done, done + m, threads), dtype=bool))
        dt += time.perf_counter() - t0
        done += m
    succ = np.concatenate(succ)
    return {"value": done / dt, "unit": unit, "cores": threads, "kind": "oracle",
            "sample": f"first {done} {what} ({dt:.1f} s on {threads} threads)", "success_rate": float(succ.mean()),
            "_success": succ}


def gpu_form(torch, run, n, unit, what):
    """One timed pass of run() (CUDA events on the current stream) over n problems, after one untimed
    pass."""
    run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    r = run()
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b)
    return {"value": n / (ms / 1e3), "unit": unit, "problems": n, "ms": ms, "what": what}, r


def agreement(gpu_success, cpu):
    """Success flags of the GPU form against the oracle's on the oracle's sample."""
    o = cpu.pop("_success")
    g = np.asarray(gpu_success, dtype=bool)[: len(o)]
    return {"problems": len(o), "success_rate_oracle": float(o.mean()), "success_rate_gpu": float(g.mean()),
            "success_flag_mismatches": int((g != o).sum())}


def cpu_oracle_traj_prm(us, goal, sph, ps, budget_s=15.0, threads=None):
    """Oracle trajectories/s with the PRM initialiser (goal IK, roadmap build, query, refinement) on
    host cores over the first problems: one problem per thread at a time, until the budget is spent.
    Returns (rate, problems, threads, seconds, success flags)."""
    import concurrent.futures as cf

    import oracle as O

    O.build()
    spec, ik = synth.ROBOT_3SEG, synth.IK_GOAL
    rb = O.make_robot(list(spec.L), spec.rc, spec.umax, thmax=spec.thmax, nb=spec.nb, rbody=spec.body_radius)
    W = O.make_weights(**synth.WEIGHTS.as_dict())
    threads = threads or os.cpu_count()
    Tn = synth.T_TRAJ

    def one(p):
        cfg = O.IkConfig(S=ik.S, n_final=ik.n_final, k_init=ik.k_init, k_final=ik.k_final, lambda0=ik.lambda0,
                         alpha0=ik.alpha0, dedup_eps=ik.dedup_eps, seed=ik.seed, p0=p)
        ug = O.solve_ik(rb, W, sph[p], O.IK6, goal[p:p + 1], cfg, threads=1)["u"][0]
        rm = O.prm_build(rb, synth.WEIGHTS.delta, sph[p], ps.seed, p, ps.N, ps.k, ps.n_check, ps.attempts)
        X0 = O.prm_query(rb, synth.WEIGHTS.delta, sph[p], rm, ps.k, ps.n_check, us[p], ug, Tn)[0]
        r = O.traj_refine(rb, W, sph[p:p + 1], us[p:p + 1], goal[p:p + 1], X0[None], synth.K_TRAJ, synth.ALPHA_TRAJ,
                          threads=1)
        return bool(r["col_ok"][0] and r["lim_ok"][0] and r["goal_pos"][0] <= 1e-3
                    and r["goal_rot"][0] <= np.deg2rad(1.0))

    done, dt, succ = 0, 0.0, []
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        while dt < budget_s and done < len(us):
            m = min(threads, len(us) - done)
            t0 = time.perf_counter()
            succ += list(ex.map(one, range(done, done + m)))
            dt += time.perf_counter() - t0
            done += m
    return done / dt, done, threads, dt, np.array(succ)


def reference_arm(args):
    """Times the FP64 CPU oracle (as it stands) on the benchmark workload, rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O

    O.build()
    spec, ik = synth.ROBOT_3SEG, synth.IK_3SEG
    rb = O.make_robot(list(spec.L), spec.rc, spec.umax, thmax=spec.thmax, nb=spec.nb, rbody=spec.body_radius,
                      lmin=spec.lmin, lmax=spec.lmax)
    W = O.make_weights(**synth.WEIGHTS.as_dict())
    tg, _ = synth.ik_workload(spec, synth.P_3SEG, "pose", lambda u: O.fk(rb, u)[0], seed=0)
    threads = os.cpu_count()
    per_step = max(threads, 16)
    cfg = O.IkConfig(S=ik.S, n_final=ik.n_final, k_init=ik.k_init, k_final=ik.k_final, lambda0=ik.lambda0,
                     alpha0=ik.alpha0, dedup_eps=ik.dedup_eps, lim_tol=ik.lim_tol, pos_tol=ik.pos_tol,
                     rot_tol=ik.rot_tol, seed=ik.seed)
    times, succ = [], []
    for k in range(args.warmup + args.steps):
        lo = (k * per_step) % (len(tg) - per_step)
        cfg.p0 = lo
        t0 = time.perf_counter()
        r = O.solve_ik(rb, W, None, O.IK6, tg[lo:lo + per_step], cfg, threads=threads)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            succ.append(r["success"].mean())
    ms = 1e3 * float(np.mean(times))
    value = per_step / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_targets_per_step": per_step},
            "success_rate": float(np.mean(succ)),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} contiguous targets per step of the 4096-target workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def shard_p0(rank: int, P: int) -> int:
    """Seed-counter offset of a rank's problems: rank r solves problems r P .. (r + 1) P - 1 of the
    job, so the counter-based seeds of every problem are those of one process solving them all."""
    return rank * P


def max_over_ranks(torch, dist, world, total_ms, device):
    """The job's time: the largest of the ranks' summed step times (all_reduce MAX)."""
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, P, ms_per_step):
    """Whole-job throughput: all ranks' problems over the slowest rank's step time."""
    return world * P / (ms_per_step / 1e3)


def time_steps(torch, fn, steps, flush, stream):
    """Median and mean of CUDA-event times of fn() over `steps` steps, L2 flushed before each."""
    ts = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts)), float(np.mean(ts))


def other_workload(args):
    """Times one of the other workloads and prints its JSON line: one GPU, except the ragged batch,
    which a torchrun launch splits over the processes by estimated cost (cr_batch_partition; the
    items are independent, so no collective touches the data path)."""
    import torch
    import torch.distributed as dist

    from paper_2607_11340_gb300 import api, build_lib, lib

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.workload != "ragged":
        raise SystemExit(f"--workload {args.workload} runs on one GPU; only the ragged batch is split over processes")
    if world > 1:
        dist.init_process_group("nccl")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if rank == 0:
        build_lib.build()
    if world > 1:
        dist.barrier()
    lib.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    rng = np.random.default_rng(0)
    line = {"n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic"}
    if args.workload == "ik1":
        spec, ik, P = synth.ROBOT_1SEG, synth.IK_1SEG, synth.P_1SEG
        u = synth.hexagon_states(rng, P, spec.n, spec.umax)
        T, _ = api.fk(api.robot_struct(spec), torch.as_tensor(u.T.copy(), dtype=torch.float64, device=dev))
        tg = torch.as_tensor(synth.pose_targets(T.cpu().numpy().T, "axis").T.copy(), dtype=torch.float64, device=dev)
        s = api.IkSolver(spec, ik, synth.WEIGHTS, lib.CR_TASK_IK5, P, precision=lib.CR_F64, device=dev)
        fn = lambda: s.solve(tg)
        units, unit, metric = P, "solves/s", "IK solves/s, 1-segment 5-DoF, FP64, single stage (32 seeds, 50 LM)"
        wl = "ik_1seg_256targets_32seeds_lm50_fp64"

        def extra():
            out = {"success_rate": float(s.out.success.float().mean())}
            forms = {}
            sp = api.IkSolver(spec, ik, synth.WEIGHTS, lib.CR_TASK_IK5, P, plain=True, device=dev)
            forms["plain_gpu"], _ = gpu_form(torch, lambda: sp.solve(tg), P, "solves/s",
                                             "one launch per target, FP64, iterates through global memory")
            forms["plain_gpu"]["success_rate"] = float(sp.out.success.float().mean())
            n1 = 32
            s1 = api.IkSolver(spec, ik, synth.WEIGHTS, lib.CR_TASK_IK5, 1, precision=lib.CR_F64, device=dev)
            tg1 = [tg[:, i:i + 1].contiguous() for i in range(n1)]
            forms["per_problem_optimised"], _ = gpu_form(
                torch, lambda: [s1.solve(tg1[i], i) for i in range(n1)], n1, "solves/s",
                "the optimised kernels launched once per target (P = 1), FP64, first 32 targets")
            if not args.no_baseline:
                import oracle as O

                tgh = tg.cpu().numpy().T
                rate, n, cores, dt, osucc, _ = cpu_oracle_rate(tgh, spec, ik, kind=O.IK5)
                out["cpu_baseline"] = {"value": rate, "unit": "solves/s", "cores": cores, "kind": "oracle",
                                       "sample": f"first {n} targets ({dt:.1f} s on {cores} threads)"}
                gs = s.out.success[:n].cpu().numpy().astype(bool)
                out["oracle_agreement"] = {"targets": n, "success_rate_oracle": float(osucc.mean()),
                                           "success_rate_gpu": float(gs.mean()),
                                           "success_flag_mismatches": int((gs != osucc).sum())}
            out["forms"] = forms
            return out

        dtype = "f64"
    elif args.workload == "path":
        spec, ik, P, H = synth.ROBOT_4SEG, synth.IK_PATH0, args.paths, synth.H_PATH

        def fkb(uu):
            T, bb = api.fk(api.robot_struct(spec), torch.as_tensor(uu.T.copy(), dtype=torch.float64, device=dev), True)
            return T.cpu().numpy().T, bb.cpu().numpy().transpose(2, 0, 1)

        wp, _, sph = synth.path_workload(spec, P, H, synth.NO_PATH, fkb, seed=0)
        s = api.PathSolver(spec, ik, synth.WEIGHTS, P, H, api.Scene(sph, per_problem=True), device=dev)
        wps = api.waypoints_soa(wp, device=dev)
        fn = lambda: s.solve(wps)
        units, unit, metric = P, "paths/s", "path following paths/s (64 waypoints, 32 spheres, FP32 + FP64 block Cholesky)"
        wl = f"path_4seg_{P}paths_64wp_32spheres_warm30_joint20"
        def path_success(sol, n):
            pos = sol.pos.reshape(n, H).max(1).values.cpu().numpy()
            rot = sol.rot.reshape(n, H).max(1).values.cpu().numpy()
            return (pos <= 1e-3) & (rot <= np.deg2rad(1.0)) & (sol.lim_ok.cpu().numpy() > 0) & \
                (sol.col_ok.cpu().numpy() > 0)

        def extra():
            out = {"tracked_rate_1mm": float((s.pos.reshape(P, H).max(1).values <= 1e-3).float().mean()),
                   "success_rate": float(path_success(s, P).mean()),
                   "waypoint_solves_per_s": P * H / (line["ms_per_step"] / 1e3),
                   "pos_err_median_m": float(s.pos.median()), "rot_err_median_rad": float(s.rot.median())}
            n1 = 8
            per = [(api.PathSolver(spec, ik, synth.WEIGHTS, 1, H, api.Scene(sph[i:i + 1], per_problem=True),
                                   device=dev), api.waypoints_soa(wp[i:i + 1], device=dev)) for i in range(n1)]
            forms = {"plain_gpu": {"unavailable": "no separate plain path kernels: the plain comparator of this "
                                                  "config is the per-problem launch below"}}
            forms["per_problem_optimised"], _ = gpu_form(
                torch, lambda: [p_.solve(w_, i) for i, (p_, w_) in enumerate(per)], n1, "paths/s",
                "the optimised kernels launched once per path (P = 1), first 8 paths")
            if not args.no_baseline:
                import oracle as O

                O.build()
                rb = O.make_robot(list(spec.L), spec.rc, spec.umax, thmax=spec.thmax, nb=spec.nb,
                                  rbody=spec.body_radius)
                W = O.make_weights(**synth.WEIGHTS.as_dict())

                def run(lo, hi, threads):
                    cfg = O.IkConfig(S=ik.S, n_final=ik.n_final, k_init=ik.k_init, k_final=ik.k_final,
                                     lambda0=ik.lambda0, alpha0=ik.alpha0, dedup_eps=ik.dedup_eps,
                                     lim_tol=ik.lim_tol, seed=ik.seed, p0=lo)
                    o = O.solve_path(rb, W, sph[lo:hi], wp[lo:hi], cfg, synth.K_WARM, synth.K_JOINT, threads=threads)
                    return (o["pos"].max(1) <= 1e-3) & (o["rot"].max(1) <= np.deg2rad(1.0)) & o["lim_ok"] & o["col_ok"]

                cpu = oracle_sample(run, P, "paths/s", "paths of 64 waypoints")
                out["oracle_agreement"] = agreement(path_success(s, P), cpu)
                out["cpu_baseline"] = cpu
            out["forms"] = forms
            return out

        dtype = "f32"
    elif args.workload == "traj":
        spec, ik, P, Tn = synth.ROBOT_3SEG, synth.IK_GOAL, synth.P_TRAJ, synth.T_TRAJ

        def fkb(uu):
            T, bb = api.fk(api.robot_struct(spec), torch.as_tensor(uu.T.copy(), dtype=torch.float64, device=dev), True)
            return T.cpu().numpy().T, bb.cpu().numpy().transpose(2, 0, 1)

        us, goal, sph, _ = synth.traj_workload(spec, P, synth.NO_TRAJ, fkb, seed=0)
        s = api.TrajSolver(spec, ik, synth.WEIGHTS, P, Tn, api.Scene(sph, per_problem=True), device=dev)
        usd = torch.as_tensor(us.T.copy(), dtype=torch.float64, device=dev)
        gd = torch.as_tensor(goal.T.copy(), dtype=torch.float64, device=dev)
        fn = lambda: s.solve(usd, gd)
        units, unit, metric = P, "trajectories/s", "trajectory planning trajectories/s (32 states, 64 spheres, 100 PG steps)"
        wl = "traj_3seg_256problems_32states_64spheres_pg100"
        def traj_success(t):
            return ((t.goal_pos <= 1e-3) & (t.goal_rot <= np.deg2rad(1.0)) & (t.col_ok > 0) &
                    (t.lim_ok > 0)).cpu().numpy()

        def extra():
            out = {"goal_reached_rate": float((s.goal_pos <= 1e-3).float().mean()),
                   "success_rate": float(traj_success(s).mean()),
                   "collision_free_rate": float(s.col_ok.float().mean()),
                   "speed_ratio_max": float(s.speed.max()), "accel_ratio_max": float(s.accel.max())}
            n1 = 8
            per = [(api.TrajSolver(spec, ik, synth.WEIGHTS, 1, Tn, api.Scene(sph[i:i + 1], per_problem=True),
                                   device=dev), usd[:, i:i + 1].contiguous(), gd[:, i:i + 1].contiguous())
                   for i in range(n1)]
            forms = {"plain_gpu": {"unavailable": "no separate plain trajectory kernels: the plain comparator of "
                                                  "this config is the per-problem launch below"}}
            forms["per_problem_optimised"], _ = gpu_form(
                torch, lambda: [t_.solve(u_, g_, i) for i, (t_, u_, g_) in enumerate(per)], n1, "trajectories/s",
                "the optimised kernels launched once per problem (P = 1), first 8 problems")
            if not args.no_baseline:
                import oracle as O

                O.build()
                rb = O.make_robot(list(spec.L), spec.rc, spec.umax, thmax=spec.thmax, nb=spec.nb,
                                  rbody=spec.body_radius)
                W = O.make_weights(**synth.WEIGHTS.as_dict())

                def run(lo, hi, threads):
                    cfg = O.IkConfig(S=ik.S, n_final=ik.n_final, k_init=ik.k_init, k_final=ik.k_final,
                                     lambda0=ik.lambda0, alpha0=ik.alpha0, dedup_eps=ik.dedup_eps,
                                     lim_tol=ik.lim_tol, seed=ik.seed, p0=lo)
                    r = O.solve_traj(rb, W, sph[lo:hi], us[lo:hi], goal[lo:hi], Tn, cfg, synth.K_TRAJ,
                                     synth.ALPHA_TRAJ, threads=threads)
                    return ((r["goal_pos"] <= 1e-3) & (r["goal_rot"] <= np.deg2rad(1.0)) & r["lim_ok"]
                            & r["col_ok"])

                cpu = oracle_sample(run, P, "trajectories/s", "problems of 32 states, 64 spheres", budget_s=20.0)
                out["oracle_agreement"] = agreement(traj_success(s), cpu)
                out["cpu_baseline"] = cpu
            out["forms"] = forms
            return out

        dtype = "f32"
    elif args.workload == "shelf":
        # trajectory planning among shelves (boxes) and capsules, each problem its own scene
        spec, ik, P, Tn = synth.ROBOT_3SEG, synth.IK_GOAL, synth.P_TRAJ, synth.T_TRAJ
        rbs = api.robot_struct(spec)

        def clearance(cand, prims):
            ug = torch.as_tensor(cand.T.copy(), dtype=torch.float64, device=dev)
            tgt = torch.zeros((7, 1), dtype=torch.float64, device=dev)
            tgt[3] = 1.0
            task = api.task_struct(lib.CR_TASK_IK6, tgt, cand.shape[0], synth.WEIGHTS)
            _, cl, _, _ = api.cost_grad(rbs, api.Scene(None, prims=prims, device=dev), task, ug, grad=False,
                                        coll=True)
            return cl.cpu().numpy()

        us, ugoal, prims = synth.shelf_traj_workload(spec, P, clearance, seed=0)
        Tg, _ = api.fk(rbs, torch.as_tensor(ugoal.T.copy(), dtype=torch.float64, device=dev))
        goal = synth.pose_targets(Tg.cpu().numpy().T, "pose")
        s = api.TrajSolver(spec, ik, synth.WEIGHTS, P, Tn, api.Scene(None, per_problem=True, prims=prims, device=dev),
                           device=dev)
        usd = torch.as_tensor(us.T.copy(), dtype=torch.float64, device=dev)
        gd = torch.as_tensor(goal.T.copy(), dtype=torch.float64, device=dev)
        fn = lambda: s.solve(usd, gd)
        units, unit = P, "trajectories/s"
        metric = (f"trajectory planning among shelves trajectories/s (32 states, 6 boxes + {synth.N_SHELF_CAPS} "
                  "capsules per problem, 100 PG steps)")
        wl = f"shelf_traj_3seg_256problems_32states_6boxes_{synth.N_SHELF_CAPS}capsules_pg100"

        def traj_success(t):
            return ((t.goal_pos <= 1e-3) & (t.goal_rot <= np.deg2rad(1.0)) & (t.col_ok > 0) &
                    (t.lim_ok > 0)).cpu().numpy()

        def extra():
            out = {"goal_reached_rate": float((s.goal_pos <= 1e-3).float().mean()),
                   "success_rate": float(traj_success(s).mean()),
                   "collision_free_rate": float(s.col_ok.float().mean())}
            if not args.no_baseline:
                import oracle as O

                O.build()
                rb = O.make_robot(list(spec.L), spec.rc, spec.umax, thmax=spec.thmax, nb=spec.nb,
                                  rbody=spec.body_radius)
                W = O.make_weights(**synth.WEIGHTS.as_dict())

                def run(lo, hi, threads):
                    cfg = O.IkConfig(S=ik.S, n_final=ik.n_final, k_init=ik.k_init, k_final=ik.k_final,
                                     lambda0=ik.lambda0, alpha0=ik.alpha0, dedup_eps=ik.dedup_eps,
                                     lim_tol=ik.lim_tol, seed=ik.seed, p0=lo)
                    r = O.solve_traj(rb, W, (None, prims[lo:hi]), us[lo:hi], goal[lo:hi], Tn, cfg, synth.K_TRAJ,
                                     synth.ALPHA_TRAJ, threads=threads)
                    return ((r["goal_pos"] <= 1e-3) & (r["goal_rot"] <= np.deg2rad(1.0)) & r["lim_ok"]
                            & r["col_ok"])

                cpu = oracle_sample(run, P, "trajectories/s", "problems of 32 states among a shelf and capsules",
                                    budget_s=20.0)
                out["oracle_agreement"] = agreement(traj_success(s), cpu)
                out["cpu_baseline"] = cpu
            return out

        dtype = "f32"
    elif args.workload == "prm":
        # Algorithm 2: roadmaps built once per scene (offline, timed apart), then per query the goal IK,
        # the roadmap query (attachment, shortest path, resampling) and the 100 PG steps
        spec, ik, P, Tn, ps = synth.ROBOT_3SEG, synth.IK_GOAL, synth.P_TRAJ, synth.T_TRAJ, synth.PRM_TRAJ

        def fkb(uu):
            T, bb = api.fk(api.robot_struct(spec), torch.as_tensor(uu.T.copy(), dtype=torch.float64, device=dev), True)
            return T.cpu().numpy().T, bb.cpu().numpy().transpose(2, 0, 1)

        us, goal, sph, _ = synth.traj_workload(spec, P, synth.NO_TRAJ, fkb, seed=0)
        scene = api.Scene(sph, per_problem=True)
        rm = api.Roadmap(spec, ps, P, device=dev)
        s = api.TrajSolver(spec, ik, synth.WEIGHTS, P, Tn, scene, device=dev, roadmap=rm)
        lin = api.TrajSolver(spec, ik, synth.WEIGHTS, P, Tn, scene, device=dev)
        usd = torch.as_tensor(us.T.copy(), dtype=torch.float64, device=dev)
        gd = torch.as_tensor(goal.T.copy(), dtype=torch.float64, device=dev)
        rm.build(scene, synth.WEIGHTS)
        build_ms = time_steps(torch, lambda: rm.build(scene, synth.WEIGHTS), max(3, args.steps), flush, stream)[1]
        ugd = torch.empty_like(usd)
        ugd.copy_(usd.flip(1))  # query timing only: any states in bounds
        query_ms = time_steps(torch, lambda: rm.query(scene, synth.WEIGHTS, usd, ugd, Tn), max(3, args.steps), flush,
                              stream)[1]
        fn = lambda: s.solve(usd, gd)
        units, unit = P, "trajectories/s"
        metric = "trajectory planning trajectories/s with the PRM initialiser (goal IK, roadmap query, 100 PG steps)"
        wl = f"traj_prm_3seg_256problems_32states_64spheres_roadmap{ps.N}x{ps.k}_check{ps.n_check}_pg100"

        def success(t):
            return ((t.goal_pos <= 1e-3) & (t.goal_rot <= np.deg2rad(1.0)) & (t.col_ok > 0) & (t.lim_ok > 0)).float()

        def extra():
            s.solve(usd, gd)
            lin.solve(usd, gd)
            torch.cuda.synchronize()
            h = s.hops.cpu().numpy()
            base = {}
            if not args.no_baseline:
                rate, n, cores, dt, osucc = cpu_oracle_traj_prm(us, goal, sph, ps)
                gs = success(s)[:n].cpu().numpy().astype(bool)
                base = {"cpu_baseline": {"value": rate, "unit": "trajectories/s", "cores": cores, "kind": "oracle",
                                         "sample": f"first {n} problems: goal IK, roadmap build, query and "
                                                   f"refinement per problem ({dt:.1f} s on {cores} threads)"},
                        "oracle_agreement": {"problems": n, "success_rate_oracle": float(osucc.mean()),
                                             "success_rate_gpu": float(gs.mean()),
                                             "success_flag_mismatches": int((gs != osucc).sum())}}
            return {**base, "roadmap_build_ms": build_ms, "roadmap_query_ms": query_ms, "roadmaps": P, "nodes_per_roadmap": ps.N,
                    "valid_node_rate": float(rm.node_ok.float().mean()),
                    "edges_per_roadmap": float(rm.row[:, -1].double().mean() / 2),
                    "path_found_rate": float((h > 0).mean()), "hops_mean": float(h[h > 0].mean()) if (h > 0).any() else 0.0,
                    "success_rate_prm": float(success(s).mean()), "success_rate_linear": float(success(lin).mean()),
                    "collision_free_rate_prm": float(s.col_ok.float().mean()),
                    "collision_free_rate_linear": float(lin.col_ok.float().mean()),
                    "trajectory_cost_median_prm": float(s.cost.median()),
                    "trajectory_cost_median_linear": float(lin.cost.median())}

        dtype = "f32"
    elif args.workload == "self":
        # IK with the self-contact rows (Eq. ik_coll over the robot itself), half the targets posed by
        # self-intersecting curled states
        spec, ik, P = synth.ROBOT_SELF, synth.IK_SELF, synth.P_SELF

        def fk_np(uu):
            T, _ = api.fk(api.robot_struct(spec), torch.as_tensor(uu.T.copy(), dtype=torch.float64, device=dev))
            return T.cpu().numpy().T

        tg_np, _ = synth.self_contact_workload(spec, P, fk_np, seed=0)
        tgd = torch.as_tensor(tg_np.T.copy(), dtype=torch.float64, device=dev)
        s = api.IkSolver(spec, ik, synth.WEIGHTS_SELF, lib.CR_TASK_IK6, P, device=dev)
        s_off = api.IkSolver(spec, ik, synth.WEIGHTS, lib.CR_TASK_IK6, P, device=dev)
        fn = lambda: s.solve(tgd)
        units, unit = P, "solves/s"
        metric = "IK solves/s with self-contact rows, 4-segment robot (128 seeds -> top 8, FP32 + FP64 Cholesky)"
        wl = "ik_self_4seg_1024targets_half_self_intersecting_128seeds_top8_pg32_lm30"

        def extra():
            s_off.solve(tgd)
            off_ms = time_steps(torch, lambda: s_off.solve(tgd), args.steps, flush, stream)[1]
            out = {"success_rate": float(s.out.success.float().mean()),
                   "success_rate_first_half_self_intersecting_targets": float(s.out.success[:P // 2].float().mean()),
                   "ms_per_step_without_self_rows": off_ms, "device_status": s.status()}
            if not args.no_baseline:
                rate, n, cores, dt, osucc, _ = cpu_oracle_rate(tg_np, spec, ik, budget_s=12.0,
                                                               weights=synth.WEIGHTS_SELF)
                gs = s.out.success[:n].cpu().numpy().astype(bool)
                out["cpu_baseline"] = {"value": rate, "unit": "solves/s", "cores": cores, "kind": "oracle",
                                       "sample": f"first {n} targets ({dt:.1f} s on {cores} threads)"}
                out["oracle_agreement"] = {"targets": n, "success_rate_oracle": float(osucc.mean()),
                                           "success_rate_gpu": float(gs.mean()),
                                           "success_flag_mismatches": int((gs != osucc).sum())}
            return out

        dtype = "f32"
    elif args.workload in ("e1", "e2"):
        # the paper's own IK benchmarks in its (theta, phi, L) parameterisation (Sec. V-B)
        ik = synth.IK_E1
        rbs = {}

        def fkb_of(spec):
            def fkb(q):
                T, bb = api.fk(api.robot_struct(spec), torch.as_tensor(q.T.copy(), dtype=torch.float64, device=dev), True)
                return T.cpu().numpy().T, bb.cpu().numpy().transpose(2, 0, 1)
            return fkb

        cases = []
        if args.workload == "e1":
            spec, P = synth.ROBOT_E1, synth.P_E1
            tg, _ = synth.e1_workload(spec, P, lambda q: fkb_of(spec)(q)[0], seed=0)
            cases.append(("3seg_ext", spec, tg, None))
            metric = "IK solves/s, paper's arc model, 3 extendable 1 m segments, no obstacles (128 seeds -> top 8, 200 its)"
            wl = "e1_arc_3seg_ext_1000targets_128seeds_top8_pg150_lm50"
        else:
            for name, spec in (("4seg_ext", synth.ROBOT_E2_EXT), ("3seg_fixed", synth.ROBOT_E2_FIXED)):
                tg, _, sph = synth.e2_workload(spec, synth.P_E2, fkb_of(spec), seed=0)
                cases.append((name, spec, tg, sph))
            metric = "IK solves/s, paper's arc model, 4 extendable 1 m segments, 27-sphere lattice (128 seeds -> top 8, 200 its)"
            wl = "e2_arc_4seg_ext_lattice27_100targets_128seeds_top8_pg150_lm50"
        for name, spec, tg, sph in cases:
            s_ = api.IkSolver(spec, ik, synth.WEIGHTS, lib.CR_TASK_IK6, len(tg), api.Scene(sph), precision=lib.CR_F32,
                              device=dev)
            rbs[name] = (s_, torch.as_tensor(tg.T.copy(), dtype=torch.float64, device=dev), spec, tg, sph)
        first = cases[0][0]
        s, tgd = rbs[first][0], rbs[first][1]
        fn = lambda: s.solve(tgd)
        units, unit = len(cases[0][2]), "solves/s"

        def extra():
            out = {"success_rate": float(s.out.success.float().mean()), "pos_err_median_m": float(s.out.pos_err.median()),
                   "rot_err_median_rad": float(s.out.rot_err.median()), "device_status": s.status()}
            if args.workload == "e1":
                # stage one alone (seeds, PG steps, SelectTop) against the FP32 peak, as for the headline
                s.stage1(tgd)
                s1_med, s1_ms = time_steps(torch, lambda: s.stage1(tgd), args.steps, flush, stream)
                c = load_counts("ik_arc_3seg_pose")
                acc = s.pg_accepted()
                n_seed = units * ik.S
                n_eval = n_seed * (ik.k_init + 1)
                fl, _ = method_ops(c, n_seed, ik.k_init, acc)  # the method's work, as for the headline
                ach = fl / (s1_ms / 1e3) / 1e12
                sm_max = measured_peaks().get("sm_max_mhz", 2070.0)
                peak = torch.cuda.get_device_properties(dev).multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
                out["roofline"] = {"bound": "alu", "kernel": "k_ik_stage1 (arc model)", "achieved": ach, "peak": peak,
                                   "unit": "TFLOP/s", "frac": ach / peak, "traffic": None, "kernel_ms": s1_ms,
                                   "count": "method (oracle op counts; gradients at accepted trials only)",
                                   "evals_per_launch": n_eval, "flop_per_launch": fl, "pg_accepted_per_launch": acc}
            for name, (s2, tg2, spec2, tgh, sph) in rbs.items():
                if name == first:
                    continue
                for _ in range(3):
                    s2.solve(tg2)
                med2, mean2 = time_steps(torch, lambda: s2.solve(tg2), args.steps, flush, stream)
                out[name] = {"value": len(tgh) / (mean2 / 1e3), "unit": "solves/s", "ms_per_step": mean2,
                             "success_rate": float(s2.out.success.float().mean())}
            if not args.no_baseline:
                spec1, tgh1, sph1 = rbs[first][2], rbs[first][3], rbs[first][4]
                rate, n, cores, dt, osucc, _ = cpu_oracle_rate(tgh1, spec1, ik, budget_s=10.0, spheres=sph1)
                gs = s.out.success[:n].cpu().numpy().astype(bool)
                out["cpu_baseline"] = {"value": rate, "unit": "solves/s", "cores": cores, "kind": "oracle",
                                       "sample": f"first {n} targets ({dt:.1f} s on {cores} threads)"}
                out["oracle_agreement"] = {"targets": n, "success_rate_oracle": float(osucc.mean()),
                                           "success_rate_gpu": float(gs.mean()),
                                           "success_flag_mismatches": int((gs != osucc).sum())}
            return out

        dtype = "f32"
    elif args.workload == "ragged":
        fam = synth.ROBOT_FAMILY
        # args.items items per process (weak scaling); the job's batch is split by estimated cost
        n_all = args.items * world
        items_all, targets_all, spheres_all, _ = synth.ragged_workload(n_all, api.family_fk_backbone(fam, dev), seed=0)
        bounds = lib.cr_batch_partition(lib._batch_items(items_all), api.BatchSolver.params(synth.IK_RAGGED), world)
        lo, hi = bounds[rank], bounds[rank + 1]
        w0 = np.concatenate([[0], np.cumsum(items_all[:, 2])])
        o0 = np.concatenate([[0], np.cumsum(items_all[:, 4])])
        items = items_all[lo:hi]
        targets, spheres = targets_all[w0[lo]:w0[hi]], spheres_all[o0[lo]:o0[hi]]
        s = api.BatchSolver(fam, items, synth.IK_RAGGED, synth.WEIGHTS, seeds_per_unit=0, device=dev, p0=lo)
        s.set_inputs(targets, spheres)
        spu, n_units, workers = s.plan()
        fn = lambda: s.run()
        units, unit = n_all, "problems/s"
        line["partition"] = {"bounds": bounds, "rule": "contiguous, by the planner's cost estimate"}
        metric = f"ragged batch problems/s ({args.items} mixed IK / path items, one graph launch)"
        wl = f"ragged_{args.items}_items_n1-6_H1-128_S16-256_no0-64"
        W = int(items[:, 2].sum())

        def lat(t_ns):
            t = np.asarray(t_ns, dtype=np.float64) / 1e6
            return {"p50_ms": float(np.percentile(t, 50)), "p99_ms": float(np.percentile(t, 99)),
                    "max_ms": float(t.max())}

        def subset(nsub=256):
            """The plain per-problem form against the batch on the first nsub items, same order."""
            sub = api.BatchSolver(fam, items[:nsub], synth.IK_RAGGED, synth.WEIGHTS, seeds_per_unit=spu, device=dev,
                                   seed_regs=s.seed_regs)
            sub.set_inputs(targets[: int(items[:nsub, 2].sum())], spheres[: int(items[:nsub, 4].sum())])
            sub.plan()
            sub.run()
            torch.cuda.synchronize()
            out = {}
            for name, run in (("batch", lambda: sub.run()), ("plain", lambda: sub.solve_plain())):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                r = run()
                b.record()
                b.synchronize()
                ms = a.elapsed_time(b)
                t_ns = (sub.t_done if name == "batch" else r["t_done"]).cpu().numpy()
                fl = (sub.flags if name == "batch" else r["flags"]).cpu().numpy()
                out[name] = {"items": nsub, "problems_per_s": nsub / (ms / 1e3), "ms": ms,
                             "success_rate": float((fl & 1).mean()), **lat(t_ns)}
            return out

        def oracle_items(lo, hi, threads):
            """The oracle's solve of items [lo, hi), one item per thread (item i: seed counter i)."""
            import concurrent.futures as cf

            import oracle as O

            O.build()
            W_ = O.make_weights(**synth.WEIGHTS.as_dict())
            w0 = np.concatenate([[0], np.cumsum(items[:, 2])])
            o0 = np.concatenate([[0], np.cumsum(items[:, 4])])
            ik_ = synth.IK_RAGGED

            def one(i):
                kind, n, H, S, no = (int(v) for v in items[i])
                rb = O.make_robot(list(fam.L[:n]), fam.rc, fam.umax, thmax=fam.thmax, nb=fam.nb,
                                  rbody=fam.body_radius)
                tg = targets[w0[i]:w0[i] + H]
                sp = spheres[o0[i]:o0[i] + no] if no else None
                cfg = O.IkConfig(S=S, n_final=min(ik_.n_final, S), k_init=ik_.k_init, k_final=ik_.k_final,
                                 lambda0=ik_.lambda0, alpha0=ik_.alpha0, dedup_eps=ik_.dedup_eps,
                                 lim_tol=ik_.lim_tol, seed=ik_.seed, p0=i)
                if kind == 1 and H > 1:
                    o = O.solve_path(rb, W_, None if sp is None else sp[None], tg[None], cfg, synth.K_WARM,
                                     synth.K_JOINT, threads=1)
                    return bool((o["pos"][0] <= 1e-3).all() and (o["rot"][0] <= np.deg2rad(1.0)).all()
                                and o["lim_ok"][0] and o["col_ok"][0])
                return bool(O.solve_ik(rb, W_, sp, 0, tg, cfg, threads=1)["success"][0])

            with cf.ThreadPoolExecutor(max_workers=threads) as ex:
                return list(ex.map(one, range(lo, hi)))

        def extra():
            t_ns = s.t_done.cpu().numpy()
            fl = s.flags.cpu().numpy()
            out = {"waypoint_solves_per_s": W / (line["ms_per_step"] / 1e3), "latency": lat(t_ns),
                   "success_rate": float((fl & 1).mean()), "seeds_per_unit": spu,
                   "seed_phase_registers": {1: "wide", 2: "tight"}.get(s.seed_regs), "work_units": n_units,
                   "worker_warps": workers, "items_ik": int((items[:, 0] == 0).sum()),
                   "items_path": int((items[:, 0] == 1).sum()), "waypoints": W,
                   "vs_plain_subset": None if args.no_baseline else subset()}
            if not args.no_baseline:
                cpu = oracle_sample(oracle_items, len(items), "problems/s", "items of the batch")
                out["oracle_agreement"] = agreement(fl & 1, cpu)
                out["cpu_baseline"] = cpu
            if args.breakdown:
                w0 = np.concatenate([[0], np.cumsum(items[:, 2])])
                o0 = np.concatenate([[0], np.cumsum(items[:, 4])])
                bd = {}
                for name, sel in (("ik_items", items[:, 0] == 0), ("path_items", items[:, 0] == 1),
                                  ("path_items_n_le_3", (items[:, 0] == 1) & (items[:, 1] <= 3)),
                                  ("path_items_n_ge_4", (items[:, 0] == 1) & (items[:, 1] >= 4))):
                    idx = np.nonzero(sel)[0]
                    sub = api.BatchSolver(fam, items[idx], synth.IK_RAGGED, synth.WEIGHTS, seeds_per_unit=spu,
                                          device=dev, seed_regs=s.seed_regs)
                    sub.set_inputs(np.concatenate([targets[w0[i]:w0[i + 1]] for i in idx]),
                                   np.concatenate([spheres[o0[i]:o0[i + 1]] for i in idx] + [np.zeros((0, 4))]))
                    sub.plan()
                    r, _ = gpu_form(torch, lambda: sub.run(), len(idx), "problems/s", "the subset as a batch of its own")
                    bd[name] = {"items": len(idx), "ms": r["ms"]}
                out["breakdown"] = bd
            return out

        dtype = "f32"
    else:
        spec = synth.ROBOT_3SEG

        def fkp(U, L, rc):
            r = api.robot_struct(spec)
            for i in range(spec.n):
                r.L[i], r.r_c[i] = L[i], rc[i]
            T, _ = api.fk(r, torch.as_tensor(U.T.copy(), dtype=torch.float64, device=dev))
            return T.cpu().numpy().T

        U, Pm, true, nom = synth.calib_workload(spec, synth.K_CALIB, fkp, seed=0)
        Ud = torch.as_tensor(U.T.copy(), dtype=torch.float32, device=dev)
        Pd = torch.as_tensor(Pm.T.copy(), dtype=torch.float64, device=dev)
        res = {}

        def fn():
            res["th"] = api.calibrate(spec, Ud, Pd, nom)[0]

        units, unit, metric = 1, "calibrations/s", "calibration of 6 parameters from 1024 noisy poses (20 LM iterations)"
        wl = "calib_3seg_1024poses"

        def extra():
            out = {"param_rel_err_max": float(np.abs(res["th"].cpu().numpy() / true - 1).max())}
            Ud64 = Ud.double()
            forms = {"plain_gpu": {"unavailable": "one problem: the optimised form is already one launch pair per "
                                                  "LM iteration"}}
            forms["fp64_bulk"], _ = gpu_form(torch, lambda: api.calibrate(spec, Ud64, Pd, nom), 1, "calibrations/s",
                                             "the same kernels with FP64 kinematics")
            if not args.no_baseline:
                import oracle as O

                O.build()
                rb = O.make_robot(list(spec.L), spec.rc, spec.umax, nb=spec.nb)
                t0 = time.perf_counter()
                ref = O.calibrate(rb, U, Pm, nom, synth.ITERS_CALIB)
                dt = time.perf_counter() - t0
                out["cpu_baseline"] = {"value": 1.0 / dt, "unit": unit, "cores": 1, "kind": "oracle",
                                       "sample": f"the whole calibration ({dt:.2f} s, one thread)"}
                out["oracle_agreement"] = {"param_rel_diff_max": float(np.abs(res["th"].cpu().numpy() / ref["theta"]
                                                                               - 1).max())}
            out["forms"] = forms
            return out

        dtype = "f32"
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    med, mean = time_steps(torch, fn, args.steps, flush, stream)
    mean = max_over_ranks(torch, dist, world, mean * args.steps, dev) / args.steps
    line.update({"metric": metric, "value": units / (mean / 1e3), "unit": unit, "ms_per_step": mean,
                 "ms_per_step_median": med, "dtype": dtype,
                 "config": {"workload": wl, "l2": "flushed between timed steps (512 MiB write)"}})
    if rank == 0:
        line.update(extra())
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.workload != "ik3":
        other_workload(args)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2607_11340_gb300 import api, build_lib, lib

    if rank == 0:
        build_lib.build()
    if world > 1:
        dist.barrier()
    lib.load()

    spec, ik, P = synth.ROBOT_3SEG, synth.IK_3SEG, args.targets
    counts = load_counts()
    tg = make_targets(torch, api, lib, spec, P, seed=rank, device=dev)
    tg_dev = torch.as_tensor(tg.T.copy(), dtype=torch.float64, device=dev)
    solver = api.IkSolver(spec, ik, synth.WEIGHTS, lib.CR_TASK_IK6, P, precision=lib.CR_F32, device=dev)
    p0 = shard_p0(rank, P)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # 512 MiB > 129 MB L2
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        solver.solve(tg_dev, p0)
        solver.stage1(tg_dev, p0)
    torch.cuda.synchronize()

    # ---- timed region: K full solves, inputs resident, L2 flushed between steps ----
    clk = ClockSampler(local)
    clk.start()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        solver.solve(tg_dev, p0)
        ev[k][1].record(stream)
    barrier()
    clocks = clk.stop()
    step_ms = np.array([a.elapsed_time(b) for a, b in ev])
    ms_per_step = max_over_ranks(torch, dist, world, step_ms.sum(), dev) / args.steps
    value = job_rate(world, P, ms_per_step)
    res = solver.out
    succ = float(res.success.float().mean().item())
    pos_med = float(res.pos_err.median().item())
    rot_med = float(res.rot_err.median().item())
    status = solver.status()

    # ---- the dominant kernel alone (stage one: seeds, 64 PG steps, SelectTop), same launch config ----
    ev1 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        ev1[k][0].record(stream)
        solver.stage1(tg_dev, p0)
        ev1[k][1].record(stream)
    torch.cuda.synchronize()
    s1_ms = float(np.mean([a.elapsed_time(b) for a, b in ev1]))
    accepted = solver.pg_accepted()  # accepted PG steps of the last stage-one launch (device counter)
    # ---- stage two alone (refine + argmin) on the candidates the last stage one left ----
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        ev2[k][0].record(stream)
        solver.stage2()
        ev2[k][1].record(stream)
    torch.cuda.synchronize()
    s2_ms = float(np.mean([a.elapsed_time(b) for a, b in ev2]))
    n_eval = P * ik.S * (ik.k_init + 1)  # value evaluations per stage-one launch
    # The method's own work (method_ops). The kernel computes the gradient at every trial (fused, one
    # pass; a warp's lanes accept independently), which is reported beside it.
    n_seed = P * ik.S
    flop_method, sfu_method = method_ops(counts, n_seed, ik.k_init, accepted)
    flop_fused = (n_seed * (counts["fwd_flop"] + counts["tan_flop"]) + n_seed * ik.k_init
                  * (counts["trial_fwd_flop"] + counts["pg_step_flop"] + counts["trial_tan_flop"]))
    achieved_tflops = flop_method / (s1_ms / 1e3) / 1e12
    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_fp32 = sm_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12

    # ---- live calibration: FFMA / MUFU / DFMA / copy peaks on this GPU in the same run ----
    cal = {}
    pbuf = torch.empty(1 << 30, dtype=torch.uint8, device=dev)
    for kind, name, it in ((0, "ffma_tflops", 4000), (1, "mufu_tops", 4000), (2, "dfma_tflops", 200), (3, "copy_gbs", 1),
                           (4, "dfma_one_lane_tflops", 200), (5, "ffma2_tflops", 4000)):
        lib.cr_peak_launch(kind, pbuf, it)
        best = 0.0
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ops = lib.cr_peak_launch(kind, pbuf, it)
            b.record(stream)
            b.synchronize()
            rate = ops / (a.elapsed_time(b) / 1e3)
            best = max(best, rate / (1e9 if kind == 3 else 1e12))
        cal[name] = best
    del pbuf

    # ---- end to end through the host-buffer API ----
    tg_host = torch.as_tensor(tg.T.copy(), dtype=torch.float64).pin_memory()
    out_host = solver.solve_host(tg_host, p0=p0)
    e2e_ms = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        solver.solve_host(tg_host, out_host, p0=p0)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_value = job_rate(world, P, max_over_ranks(torch, dist, world, np.sum(e2e_ms), dev) / args.steps)
    h2d = tg_host.numel() * 8
    d2h = sum(v.numel() * v.element_size() for v in out_host.values())

    # ---- plain one-launch-per-target FP64 comparator on a subset ----
    Pp = 16
    plain = api.IkSolver(spec, ik, synth.WEIGHTS, lib.CR_TASK_IK6, Pp, plain=True, device=dev)
    plain.solve(tg_dev[:, :Pp].contiguous(), p0)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    plain.solve(tg_dev[:, :Pp].contiguous(), p0)
    b.record(stream)
    b.synchronize()
    plain_rate = Pp / (a.elapsed_time(b) / 1e3)
    plain_succ = float(plain.out.success.float().mean().item())
    opt_succ_sub = float(res.success[:Pp].float().mean().item())

    if world > 1:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "targets_per_gpu": P, "seeds": ik.S, "k_init": ik.k_init,
                   "n_final": ik.n_final, "k_final": ik.k_final, "segments": spec.n,
                   "l2": "flushed between timed steps (512 MiB write)", "lm_cholesky": "f64"},
        "success_rate": succ, "pos_err_median_m": pos_med, "rot_err_median_rad": rot_med, "device_status": status,
        "evals_per_s": world * (n_eval + P * ik.n_final * (2 * ik.k_final + 1)) / (ms_per_step / 1e3),
        "roofline": {"bound": "alu", "kernel": "k_ik_stage1 + k_ik_select", "achieved": achieved_tflops, "peak": peak_fp32,
                     "unit": "TFLOP/s", "frac": achieved_tflops / peak_fp32,
                     "traffic": STAGE1_DRAM_BYTES_PER_TARGET * P,
                     "peak_source": f"{sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz",
                     "kernel_ms": s1_ms, "count": "method (oracle op counts; gradients at accepted trials only)",
                     "flop_per_launch": flop_method, "evals_per_launch": n_eval,
                     "pg_accepted_per_launch": accepted, "pg_accept_rate": accepted / (n_seed * ik.k_init),
                     "frac_of_live_ffma": achieved_tflops / cal["ffma_tflops"],
                     "frac_fused_form": flop_fused / (s1_ms / 1e3) / 1e12 / peak_fp32,
                     "sfu_results_per_s": sfu_method / (s1_ms / 1e3),
                     "sfu_frac_of_live_mufu": sfu_method / (s1_ms / 1e3) / (cal["mufu_tops"] * 1e12)},
        "refine": {"kernel": "k_ik_refine + k_ik_argmin", "kernel_ms": s2_ms, "bound": "fp64",
                   "fp64_flop_per_launch": P * ik.n_final * ik.k_final * counts["lm_update_flop"],
                   "achieved_tflops": P * ik.n_final * ik.k_final * counts["lm_update_flop"] / (s2_ms / 1e3) / 1e12,
                   "peak_live_dfma_tflops": cal["dfma_tflops"],
                   "frac": P * ik.n_final * ik.k_final * counts["lm_update_flop"] / (s2_ms / 1e3) / 1e12
                   / cal["dfma_tflops"],
                   "count": "oracle op count of one LM update (damping, Cholesky, solves, gain ratio) per "
                            "candidate and iteration; the FP32 evaluations and the FP64 acceptance are not "
                            "in it"},
        "calibration": cal,
        "plain_form": {"value": plain_rate, "unit": UNIT, "targets": Pp, "success_rate": plain_succ,
                       "optimised_success_rate_same_targets": opt_succ_sub, "speedup": value / world / plain_rate},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": 4 * args.steps,  # stage one, SelectTop, refine, argmin
        "clocks": clocks,
    }
    if world == 1 and not args.no_baseline:
        rate, n, cores, dt, osucc, ou = cpu_oracle_rate(tg, spec, ik, p0=p0)
        gsucc = res.success[:n].cpu().numpy().astype(bool)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"first {n} of the 4096 targets ({dt:.1f} s on {cores} threads)"}
        line["oracle_agreement"] = {"targets": n, "success_rate_oracle": float(osucc.mean()),
                                    "success_rate_gpu": float(gsucc.mean()),
                                    "success_flag_mismatches": int((gsucc != osucc).sum())}
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
