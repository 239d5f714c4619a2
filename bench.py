#!/usr/bin/env python3
"""Throughput of the constrained forward-dynamics step: world-steps/s on 4096 closed-loop bipeds.

Workload (one "step" = one kamino_step over the whole batch, the full hot path in one launch):
4096 synthetic bipeds (31 bodies, 36 revolute joints, 6 loops, 16 foot-corner contact candidates
on the plane), dt = 2 ms, Gaussian actuation sigma = 5 N m from the counter-based generator,
Proximal-ADMM to tol 1e-5 with N_max = 1000 and rho = 0.1.  Five variants are timed: plain FP32
from a cold start, the mixed mode (TF32 tensor-core sweep, FP32 iteration; the FP64 refinement
stays off at tol 1e-5) from a cold start, from the impulse cache and from the learned warm start,
and the sparse formulation of Sec. 5.1 (matrix-free Delassus operator, --cr warm-started Conjugate
Residual iterations per x-step, FP32, cold start); the headline is the learned warm start.  The simulation really advances: K timed steps follow W warm-up steps from the standing pose.

Reported: ``value`` = world-steps/s with the state resident in HBM (CUDA events on the launching
stream, L2 flushed between timed steps); ``e2e`` = the same through the C ABI with the actuation
uploaded from pinned host memory and the body state downloaded every step; ``roofline`` of the
step kernel; ``cpu_baseline`` = the FP64 CPU oracle on a bounded sample.  ``--impl reference``
times the oracle alone (the reference arm of this comparison).
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "world-steps/s @4096 closed-loop bipeds, NCP residual<=1e-5; warm vs plain"
UNIT = "world-steps/s"
FP32_LANES = 128                      # FP32 FMA lanes per SM (sm_100 / sm_103)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--worlds", type=int, default=4096)
    p.add_argument("--iters", type=int, default=1000)
    p.add_argument("--tol", type=float, default=1e-5)
    p.add_argument("--dt", type=float, default=2e-3)
    p.add_argument("--rho", type=float, default=0.1)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--cpu-sample", type=int, default=4096, help="worlds in the CPU-oracle sample (one step each)")
    p.add_argument("--ref-sample", type=int, default=64, help="worlds per timed step of --impl reference")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--workload", default="biped", choices=["biped", "heightfield", "hetero", "fourbar", "team"])
    p.add_argument("--team", type=int, default=2, help="bipeds per world of the 'team' workload (sparse formulation)")
    p.add_argument("--learned", type=int, default=1, help="train and time the learned warm start")
    p.add_argument("--gen-steps", type=int, default=40, help="solver steps generating training pairs")
    p.add_argument("--train-steps", type=int, default=600, help="Adam steps of the warm-start network")
    p.add_argument("--graph", type=int, default=0, help="replay a captured CUDA graph per step")
    p.add_argument("--ncp-stop", type=int, default=1, help="a world converges only once its natural-map NCP "
                                                           "residual is below tol too (the metric's condition)")
    p.add_argument("--stall-window", type=int, default=64,
                   help="with --ncp-stop: the stall exit of worlds whose dual residual sits on its floor (0: off)")
    p.add_argument("--cr", type=int, default=9, help="CR iterations per x-step of the timed sparse-formulation "
                                                     "variant (Sec. 5.1); 0: not timed")
    return p.parse_args()


# ----------------------------------------------------------------------------- CPU oracle (baseline)
_ORACLE_WORLDS = {}


def _oracle_chunk(job):
    """Solve one step of the given worlds with the oracle; returns the solve time (the world set is
    generated once per process and kept)."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import worldgen as wg
    from oracle import timestep as T
    n, seed, worlds, dt, iters, tol, rho = job
    if (n, seed) not in _ORACLE_WORLDS:
        _ORACLE_WORLDS[(n, seed)] = wg.make_biped(num_worlds=n, seed=seed)
    ws = _ORACLE_WORLDS[(n, seed)]
    tau = wg.actuation(ws, seed, 0)
    params = T.SolverParams(rho=rho, eps=tol, n_max=iters)
    t0 = time.perf_counter()
    T.step(ws, T.initial_state(ws), tau, dt, params, worlds=worlds)
    return time.perf_counter() - t0


def oracle_rate(pool, cores, n_worlds, sample, seed, dt, iters, tol, rho, offset=0):
    """World-steps/s of the oracle over `sample` worlds starting at `offset` (first step from the
    standing pose), split over the pool's processes: the sample over the slowest process's solve
    time (world generation excluded)."""
    worlds = [(offset + i) % n_worlds for i in range(sample)]
    chunks = [worlds[i::cores] for i in range(cores)]
    jobs = [(n_worlds, seed, c, dt, iters, tol, rho) for c in chunks if c]
    times = pool.map(_oracle_chunk, jobs)
    wall = max(times)
    return sample / wall, wall


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go to $KAMINO_CLOCKS_DIR (default: the system's temporary directory)
        import tempfile
        out_dir = os.environ.get("KAMINO_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"kamino_clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    cores = host_cores()
    ctx = mp.get_context("spawn")
    sample = max(cores, min(args.ref_sample, args.worlds))
    with ctx.Pool(cores) as pool:
        for k in range(args.warmup):
            oracle_rate(pool, cores, args.worlds, cores, args.seed, args.dt, args.iters, args.tol, args.rho,
                        offset=k * cores)
        total, n = 0.0, 0
        for k in range(args.steps):
            _, wall = oracle_rate(pool, cores, args.worlds, sample, args.seed, args.dt, args.iters, args.tol,
                                  args.rho, offset=k * sample)
            total += wall
            n += sample
    value = n / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.worlds} closed-loop bipeds (31 bodies, 36 revolute, 6 loops), dt={args.dt}, "
                                   f"tol={args.tol}, N_max={args.iters}", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{sample} of {args.worlds} bipeds x 1 step (standing pose) per timed step, "
                                       f"successive worlds each step; solve time of the slowest process"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- ranks (weak scaling)
# Every rank steps its own worlds (seed + rank): no data-path collective.  The only exchange is the
# timing: the job's time is the slowest rank's, and the job's work is the sum over the ranks.
def rank_seed(seed, rank):
    return seed + rank


def job_units(worlds_per_rank, steps, world):
    return worlds_per_rank * steps * world


def max_over_ranks(v, world, device):
    """The largest of the ranks' values (every rank gets it); the identity on one rank."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- GPU arm
def algorithmic_flops(rows, iters):
    """Flops of the method per world-step: dense Cholesky m^3/3, per PADMM iteration a forward and
    a backward substitution 2 m^2 plus ~20 m elementwise (De Saxce, projection, dual update,
    Nesterov, residuals), block-sparse Delassus assembly ~ 2 * 12 * m * k (k ~ 8 rows sharing a
    body)."""
    m = rows.astype("float64")
    it = iters.astype("float64")
    return m ** 3 / 3.0 + it * (2.0 * m * m + 20.0 * m) + 2.0 * 12.0 * m * 8.0


def algorithmic_flops_sparse(rows, iters, k):
    """Flops of the sparse formulation per world-step: per PADMM iteration k + 1 applications of the
    matrix-free operator (per row: the two 6-blocks of J against the gathered body vectors, and the
    gather of J^T P v, ~96 flops), k CR iterations of vector updates and dot products (~10 m) and
    ~20 m elementwise; no factorisation."""
    m = rows.astype("float64")
    it = iters.astype("float64")
    return it * ((k + 1) * 96.0 * m + k * 10.0 * m + 20.0 * m)


def ncp_report(ncp, status, its, tol, n_max, rate):
    """The metric's qualifying condition over every world-step of a variant: the device's
    natural-map NCP residual of the returned (lambda, u+) (kamino_residual.r_ncp) against the
    tolerance; the world-steps that meet it per second; and, for the world-steps that ran to N_max
    without meeting the ADMM test, their residuals and their share of the PADMM iterations (of the
    step's SM time, since one iteration costs the same in every world of the batch)."""
    import numpy as np
    ok = ncp <= tol
    capped = (status & 1) != 0
    out = {"ncp_le_tol_fraction": float(ok.mean()), "ncp_qualified_value": float(rate * ok.mean()),
           "ncp_median": float(np.median(ncp)), "ncp_p99": float(np.quantile(ncp, 0.99)),
           "capped_fraction": float(capped.mean()), "stalled_fraction": float(np.mean((status & 8) != 0)),
           "capped_iteration_share": float(its[capped].sum() / max(its.sum(), 1))}
    if capped.any():
        c = ncp[capped]
        out["capped_ncp"] = {"median": float(np.median(c)), "p90": float(np.quantile(c, 0.9)), "max": float(c.max()),
                             "le_tol_fraction": float(np.mean(c <= tol))}
    return out


def kernel_source_hash():
    """SHA-256 of the step kernel's sources: DRAM counters taken from another version are stale."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2603_16536_gb300", "csrc")
    for f in ("kamino_step.cu", "kamino_device.cuh", "kamino_internal.h"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def step_kernel_traffic(workload, worlds):
    """dram__bytes_read.sum + dram__bytes_write.sum of one step-kernel launch, from the ncu capture
    recorded in profiles/traffic.json, scaled from the captured world count to `worlds` (the
    kernel's traffic is per world); None when absent or taken on other kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        entry = json.load(open(path)).get(workload)
    except (OSError, ValueError):
        return None
    if not entry or entry.get("source_sha256") != kernel_source_hash():
        return None
    return entry["dram_bytes"] * worlds / entry["worlds"]


def hbm_roofline(traffic, launch_ms, peaks):
    """The step kernel against the HBM roofline: its DRAM bytes per launch (ncu, scaled to the
    launch's worlds) over the CUDA-event launch time, as a fraction of the measured copy bandwidth.
    None when either the bytes or the peak is unknown."""
    peak = peaks.get("hbm_gbs")
    if traffic is None or not peak or not launch_ms:
        return None
    gbs = traffic / (launch_ms / 1e3) / 1e9
    return {"achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "bytes_per_launch": traffic, "peak_note": "measured copy bandwidth (MEASURED_PEAKS hbm_gbs)"}


def build_workload(args, seed):
    import worldgen as wg
    if args.workload == "biped":
        return wg.make_biped(num_worlds=args.worlds, seed=seed), \
            f"{args.worlds} closed-loop bipeds (31 bodies, 36 revolute joints, 6 loops, 16 foot contact candidates, plane)"
    if args.workload == "heightfield":
        return wg.make_biped_heightfield(num_worlds=args.worlds, seed=seed), \
            f"{args.worlds} bipeds on a 64x64 heightfield (heights U[0,0.05] m, 32 candidates, up to 276 rows)"
    if args.workload == "hetero":
        q = args.worlds // 4
        return wg.concat([wg.make_fourbar(q, seed=seed), wg.make_stewart(q, seed=seed), wg.make_excavator(q, seed=seed),
                          wg.make_biped(q, seed=seed)]), \
            f"{4 * q} heterogeneous worlds ({q} each: four-bar 20 rows, 6-UPS Stewart 72, excavator 60, biped <=228)"
    if args.workload == "team":
        return wg.make_biped_team(num_worlds=args.worlds, seed=seed, per_world=args.team), \
            f"{args.worlds} worlds of {args.team} closed-loop bipeds each ({31 * args.team} bodies, " \
            f"{180 * args.team} joint rows + up to {48 * args.team} contact rows; beyond the dense formulation)"
    if args.workload == "fourbar":
        return wg.make_fourbar(num_worlds=args.worlds, seed=seed), f"{args.worlds} planar four-bars (20 rows)"
    raise ValueError(args.workload)


def run_gpu(args, rank, world):
    import numpy as np

    # CPU baseline first (spawned pool, before any CUDA call)
    cpu = None
    if rank == 0 and not args.no_cpu and args.workload == "biped":
        cores = host_cores()
        with mp.get_context("spawn").Pool(cores) as pool:
            rate, wall = oracle_rate(pool, cores, args.worlds, min(args.cpu_sample, args.worlds), args.seed,
                                     args.dt, args.iters, args.tol, args.rho)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{min(args.cpu_sample, args.worlds)} of {args.worlds} bipeds x 1 step (standing pose), "
                         f"tol {args.tol}, N_max {args.iters}; {wall:.1f} s solve time of the slowest of {cores} processes"}

    import ctypes as C
    import torch
    import torch.distributed as dist
    import worldgen as wg
    from paper_2603_16536_gb300 import kamino as K

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    seed = rank_seed(args.seed, rank)
    ws, desc = build_workload(args, seed)
    W = ws.num_worlds
    stream = torch.cuda.current_stream()
    n_act = max(ws.n_act_max, 1)
    total_steps = args.warmup + args.steps
    tau_host = np.stack([wg.actuation(ws, seed, 10_000 + k) for k in range(total_steps)]).astype(np.float32)
    tau_dev = torch.tensor(tau_host, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > L2 (129 MB)
    lib = K.load_library()
    sptr = C.c_void_p(stream.cuda_stream)
    def dense_model(precision):
        """The dense formulation's model, or None where its matrix does not fit (larger worlds)."""
        try:
            return K.Model(ws, precision, K.make_params(rho=args.rho))
        except K.KaminoError as e:
            if e.status != 7:
                raise
            return None

    model_plain = dense_model("fp32")
    model = dense_model("mixed")
    if model is None:
        args.learned = 0              # the learned warm start is timed with the dense formulation
    model_sparse = K.Model(ws, "fp32", K.make_params(rho=args.rho, cr_iters=args.cr)) if args.cr > 0 else None
    tune_report = None
    if args.workload == "hetero":
        # per-bucket (group size, panel) chosen by the autotuner on a scratch state (not timed)
        for mdl in (model_plain, model):
            st_tune = K.State(mdl, dev)
            st_tune.autotune(args.dt, args.iters, args.tol, tau_dev[0], stream)
            torch.cuda.synchronize()
            del st_tune
        tune_report = model.plan()[1]

    # ---- learned warm start: train the per-type network on solver-generated pairs (not timed)
    nets = []
    train_report = None
    if args.learned:
        # one network per world type (its worlds share body, joint, candidate and actuator
        # counts), all trained on pairs the solver generates from the same trajectory
        t0 = time.perf_counter()
        st_gen = K.State(model, dev)
        types = [np.nonzero(ws.world_type == t)[0] for t in np.unique(ws.world_type)]
        steps_gen = args.gen_steps
        bufs = []
        for ti, worlds in enumerate(types):
            net = K.Mlp(model, worlds, hidden=256, max_batch=max(4096, len(worlds)), seed=seed + ti)
            X = torch.empty((steps_gen * len(worlds), net.info.d_in), device=dev)
            Y = torch.empty((steps_gen * len(worlds), net.info.d_out), device=dev)
            nets.append(net)
            bufs.append((X, Y, len(worlds)))
        for k in range(steps_gen):
            tk = torch.tensor(wg.actuation(ws, seed, k), dtype=torch.float32, device=dev)
            for net, (X, Y, n) in zip(nets, bufs):
                net.features(st_gen, tk, out=X[k * n:(k + 1) * n])
            st_gen.step(args.dt, 4 * args.iters, args.tol / 10, tk)
            for net, (X, Y, n) in zip(nets, bufs):
                net.targets(st_gen, out=Y[k * n:(k + 1) * n])
        gen = torch.Generator(device=dev).manual_seed(seed)
        loss = torch.zeros(1, device=dev)
        firsts, lasts = [], []
        for net, (X, Y, n) in zip(nets, bufs):
            net.fit_normalization(X, Y)
            first = None
            for it in range(args.train_steps):
                rows = torch.randint(0, steps_gen * n, (4096,), device=dev, generator=gen, dtype=torch.int32)
                if it == 0 or it == args.train_steps - 1:
                    loss.zero_()
                net.train_step(X, Y, rows, lr=1e-3 if it < 0.7 * args.train_steps else 2e-4,
                               loss=loss if it in (0, args.train_steps - 1) else None)
                if it == 0:
                    first = loss.item()
            firsts.append(first)
            lasts.append(loss.item())
        torch.cuda.synchronize()
        train_report = {"networks": len(nets), "pairs": steps_gen * W, "adam_steps": args.train_steps,
                        "batch": 4096, "loss_first": firsts if len(nets) > 1 else firsts[0],
                        "loss_last": lasts if len(nets) > 1 else lasts[0], "seconds": time.perf_counter() - t0}
        del bufs, st_gen

    def learned_vs_cold():
        """The learned warm start against the cold start on identical states (not timed): the bipeds
        after the warm-up steps, one step each way to the benchmark's tolerance; iterations to tol and
        the relative velocity difference |u_learned - u_cold|inf / max(|u_cold|inf, g dt) per world."""
        model.set_params(K.make_params(rho=args.rho, ncp_stop=args.ncp_stop, stall_window=args.stall_window))
        st0 = K.State(model, dev)
        for k in range(args.warmup):
            st0.step(args.dt, args.iters, args.tol, tau_dev[k], stream)
        q0, u0, c0 = st0.body_q.clone(), st0.body_u.clone(), st0.cache.clone()
        out = {}
        for name, mode in (("cold", K.WARM_COLD), ("learned", K.WARM_EXTERNAL)):
            model.set_params(K.make_params(rho=args.rho, warm_mode=mode, ncp_stop=args.ncp_stop,
                                           stall_window=args.stall_window))
            st1 = K.State(model, dev)
            st1.body_q.copy_(q0); st1.body_u.copy_(u0); st1.cache.copy_(c0)
            if mode == K.WARM_EXTERNAL:
                for net in nets:
                    net.warm_start(st1, tau_dev[args.warmup], stream)
            st1.step(args.dt, args.iters, args.tol, tau_dev[args.warmup], stream)
            torch.cuda.synchronize()
            rep = st1.residuals()
            out[name] = (st1.body_u.double().cpu().numpy(), rep)
        uc, ul = out["cold"][0], out["learned"][0]
        err = []
        for w in range(W):
            b = slice(int(ws.world_body_offset[w]), int(ws.world_body_offset[w + 1]))
            err.append(np.abs(ul[b] - uc[b]).max() / max(np.abs(uc[b]).max(), 9.81 * args.dt))
        err = np.array(err)
        both = (out["cold"][1]["status"] == 0) & (out["learned"][1]["status"] == 0)
        return {"state": f"the {W} worlds after {args.warmup} warm-up steps, one step each way, tol {args.tol}",
                "mean_iterations": {k: float(v[1]["iterations"].mean()) for k, v in out.items()},
                "converged_fraction": {k: float(np.mean(v[1]["status"] == 0)) for k, v in out.items()},
                "err_u_learned_vs_cold": {"median": float(np.median(err)), "p99": float(np.quantile(err, 0.99)),
                                          "max_where_both_converged": float(err[both].max()) if both.any() else None}}

    learned_report = learned_vs_cold() if nets and args.workload == "biped" else None

    def run_variant(name, warm_mode, learned=False, mdl=None, refine64=True, cr=0):
        mdl = mdl or model
        mdl.set_params(K.make_params(rho=args.rho, warm_mode=warm_mode, refine64=refine64, cr_iters=cr,
                                     ncp_stop=args.ncp_stop, stall_window=args.stall_window))
        st = K.State(mdl, dev)
        graph = None
        if args.graph:
            gstream = torch.cuda.Stream(device=dev)
            with torch.cuda.stream(gstream):
                graph = st.graph(args.dt, args.iters, args.tol, st.tau, gstream)
            torch.cuda.synchronize()

        def one(k, ev=None):
            if learned:
                for net in nets:
                    net.warm_start(st, tau_dev[k], stream)
            if ev is not None:
                ev[0].record(stream)
            if graph is not None:
                st.tau.copy_(tau_dev[k].reshape(-1)[:st.tau.numel()])
                graph.launch(stream)
            else:
                st.step(args.dt, args.iters, args.tol, tau_dev[k], stream)
            if ev is not None:
                ev[1].record(stream)

        for k in range(args.warmup):
            one(k)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        ms, ms_step, rows, its, conv, ncp, status = [], [], [], [], [], [], []
        torch.cuda.nvtx.range_push(f"timed_{name}")
        for k in range(args.warmup, total_steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one(k, (s0, s1))
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            ms_step.append(s0.elapsed_time(s1))
            rep = st.residuals()
            rows.append(rep["num_rows"].copy())
            its.append(rep["iterations"].copy())
            conv.append(float(np.mean((rep["status"] & ~8) == 0)))    # converged, or stopped by the stall exit
            ncp.append(rep["r_ncp"].copy())
            status.append(rep["status"].copy())
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        barrier()
        return st, ms, np.concatenate(rows), np.concatenate(its), conv, ms_step, np.concatenate(ncp), \
            np.concatenate(status)

    def reduce_max(v):
        return max_over_ranks(v, world, dev)

    sampler = ClockSampler(local)
    sampler.start()
    results = {}
    if model_plain is not None:
        results["plain_fp32_cold"] = run_variant("plain_fp32_cold", K.WARM_COLD, mdl=model_plain, refine64=False)
    if model is not None:
        results["mixed_cold"] = run_variant("mixed_cold", K.WARM_COLD)
        results["mixed_cached_warm"] = run_variant("mixed_cached_warm", K.WARM_CACHED)
    if nets:
        results["mixed_learned_warm"] = run_variant("mixed_learned_warm", K.WARM_EXTERNAL, learned=True)
    if model_sparse is not None:
        results[f"sparse_cr{args.cr}_fp32_cold"] = run_variant(f"sparse_cr{args.cr}_fp32_cold", K.WARM_COLD,
                                                               mdl=model_sparse, refine64=False, cr=args.cr)
    clocks = sampler.stop()
    units = job_units(W, args.steps, world)
    variants = {}
    for name, (_, ms, rows, its, conv, _, ncp, status) in results.items():
        t = reduce_max(sum(ms) / 1e3)
        variants[name] = {"value": units / t, "ms_per_step": 1e3 * t / args.steps,
                          "mean_iterations": float(its.mean()), "converged_fraction": float(np.mean(conv)),
                          **ncp_report(ncp, status, its, args.tol, args.iters, units / t)}
    sparse_name = f"sparse_cr{args.cr}_fp32_cold"
    head = "mixed_learned_warm" if nets else "mixed_cached_warm" if model is not None else sparse_name
    head_sparse = head == sparse_name
    st_h, ms_h, rows_h, its_h, _, ms_step_h, _, _ = results[head]
    v_head = variants[head]["value"]
    t_head = units / v_head

    # ---- end to end through the C ABI: pinned host actuation in, body state out, every step
    learned = head == "mixed_learned_warm"
    if head_sparse:
        model = model_sparse
    model.set_params(K.make_params(rho=args.rho, warm_mode=K.WARM_EXTERNAL if learned else K.WARM_COLD if head_sparse
                                   else K.WARM_CACHED, cr_iters=args.cr if head_sparse else 0,
                                   ncp_stop=args.ncp_stop, stall_window=args.stall_window))
    B = int(ws.world_body_offset[-1])
    tau_pin = torch.tensor(tau_host).pin_memory()
    q_out = torch.empty((B, 7), dtype=torch.float32).pin_memory()
    u_out = torch.empty((B, 6), dtype=torch.float32).pin_memory()
    # a fresh state, so that the end-to-end run follows the same trajectory as the timed variant
    st_h = K.State(model, dev)
    tau_dev_ptr = C.c_void_p(st_h.tau.data_ptr())

    def e2e_step(k):
        K._check(lib.kamino_state_upload(st_h.handle, K.BUF_TAU, C.c_void_p(tau_pin[k].data_ptr()), W * ws.n_act_max, sptr))
        if learned:
            for net in nets:
                K._check(lib.kamino_mlp_warm_start(net.handle, st_h.handle, tau_dev_ptr, sptr))
        K._check(lib.kamino_step(st_h.handle, args.dt, args.iters, args.tol, tau_dev_ptr, sptr))
        K._check(lib.kamino_state_download(st_h.handle, K.BUF_BODY_Q, C.c_void_p(q_out.data_ptr()), B * 7, sptr))
        K._check(lib.kamino_state_download(st_h.handle, K.BUF_BODY_U, C.c_void_p(u_out.data_ptr()), B * 6, sptr))

    for k in range(args.warmup):
        e2e_step(k)
    torch.cuda.synchronize()
    barrier()
    e_ms = []
    for k in range(args.warmup, total_steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_step(k)
        e1.record(stream)
        e1.synchronize()
        e_ms.append(e0.elapsed_time(e1))
    barrier()
    v_e2e = units / reduce_max(sum(e_ms) / 1e3)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # ---- roofline of the step kernel (one launch = the whole batch) for the headline variant:
    # algorithmic flops of the launch over its own duration (CUDA events around kamino_step on the
    # launching stream, so the warm-start network's launches are not counted).
    peaks = measured_peaks()
    smax = clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = sm_count * FP32_LANES * 2 * smax * 1e6 / 1e12       # FP32 FMA lanes x clock, TFLOP/s
    flops = float((algorithmic_flops_sparse(rows_h, its_h, args.cr) if head_sparse
                   else algorithmic_flops(rows_h, its_h)).sum()) / 1e12
    achieved = flops / (sum(ms_step_h) / 1e3)
    traffic = step_kernel_traffic(args.workload, W)
    plan_mode, plan_buckets = model.plan()
    # one launch per bucket (persistent plan), else the step kernel and the longest-first order kernel
    step_launches = len(plan_buckets) if plan_mode == K.LAUNCH_PERSISTENT else 2
    launches_per_step = step_launches + (7 * len(nets) if learned else 0)
    line = {
        "metric": METRIC, "value": v_head, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_head / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if head_sparse else "f32+tf32+bf16", "data": "synthetic",
        "config": {"workload": f"{desc} per GPU, dt={args.dt}, Gaussian actuation sigma=5, PADMM tol={args.tol}, "
                               f"N_max={args.iters}, rho={args.rho}"
                               f"{', converged = ADMM residuals and NCP residual below tol' if args.ncp_stop else ''}"
                               f"{f', stall exit every {args.stall_window} iterations' if args.ncp_stop and args.stall_window else ''}"
                               f"; headline: {head}",
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}"},
        "variants": variants,
        "warm_over_plain": v_head / variants["plain_fp32_cold"]["value"] if "plain_fp32_cold" in variants else None,
        "mean_rows": float(rows_h.mean()),
        "gpu_launches": args.steps * launches_per_step,
        "e2e": {"value": v_e2e, "unit": UNIT, "h2d_bytes_per_step": W * ws.n_act_max * 4,
                "d2h_bytes_per_step": B * 13 * 4},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": achieved / alu_peak, "traffic": traffic,
                     "kernel": "kamino step kernel, sparse formulation" if head_sparse
                     else "kamino step kernel (one launch per step)",
                     "launch_ms": sum(ms_step_h) / len(ms_step_h),
                     "peak_note": f"derived FP32 FMA peak: {sm_count} SMs x {FP32_LANES} lanes x 2 x {smax:.0f} MHz",
                     "hbm": hbm_roofline(traffic, sum(ms_step_h) / len(ms_step_h), peaks)},
        "clocks": clocks,
    }
    if train_report:
        line["learned_warm_start_training"] = train_report
    if learned_report:
        line["learned_vs_cold_start"] = learned_report
    if tune_report:
        line["autotuned_plan"] = tune_report
    if args.graph:
        line["config"]["cuda_graph"] = "each timed step replays a captured graph of kamino_step"
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_gpu(args, rank, world)


if __name__ == "__main__":
    sys.exit(main())
