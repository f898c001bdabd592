#!/usr/bin/env python
"""Benchmark of the RS potential path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

One step = one whole solve of the workload (sinc factors, particle snapping, long-range
Gram matrices, RHOSVD eigen stage, Tucker core, full-grid reconstruction with the
short-range windows, interaction energy) with the particles already resident in HBM.
The metric is grid points per second (n^3 per solve).  For N > 1 (torchrun) every rank
solves its own seeded replica (independent problems, weak scaling, no data-path
collective); the reported value is the whole-job rate over the slowest rank's time.

The JSON line also carries sub-reports: the largest workload (the n = 1025 lattice) timed the
same way (``large``), the forces workload (``forces``), the plain GPU paths, and the serving
workload (``serving``: 256 requests through the library's request loop, replayed at their
Poisson arrival times and all at once for the loop's capacity, p50/p99 latency).

``--impl reference`` times the FP64 CPU oracle (full-rank canonical sum at sampled grid
points) on the host cores, on the same workload and metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RS potential grid pts/s vs plain GPU path at 1e-6 rel err; served p50/p99 ms"
UNIT = "grid_pts/s"
DEFAULT_WORKLOAD = "c2_protein1000_n513"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        d["source"] = "measured"
        return d
    return dict(FALLBACK_PEAKS)


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.fn = None

    def start(self):
        try:
            fd, self.fn = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.fn, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.fn):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), reasons=parts[4:9]))
            except ValueError:
                continue
        os.unlink(self.fn)
        if not rows:
            return None
        names = ["active_mask", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        seen = set()
        for r in rows:
            for nm, v in zip(names[1:], r["reasons"][1:]):
                if v.lower().startswith("active"):
                    seen.add(nm)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(seen), "samples": len(rows)}


def kernel_hash() -> str:
    """Hash of the assembly kernel's source (the tcgen05 helpers and rs_tc.cu without its T2 tile
    section): the recorded ncu traffic applies only to the code it was captured from."""
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_1606_09218_gb300", "csrc")
    h.update(open(os.path.join(csrc, "rs_tcgen05.cuh"), "rb").read())
    text = open(os.path.join(csrc, "rs_tc.cu"), "rb").read()
    a = text.find(b"// ------------------------------------------------------------------ T2 tiles")
    b = text.find(b"// ------------------------------------------------------------------ assembly kernel")
    if 0 <= a < b:
        text = text[:a] + text[b:]
    h.update(text)
    return h.hexdigest()[:12]


# DRAM bytes of one assembly launch on workload c2 from ncu (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by the source hash it was captured from; see profiles/.
NCU_TRAFFIC = {"0790a91b0d90": 567.9e6}


_WORKER_PROBLEM = None


def _oracle_worker_init(cfg, xyz, Z):
    """Pool initializer: one thread per process, and the oracle's problem built once."""
    global _WORKER_PROBLEM
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    from oracle import rs_oracle as O
    _WORKER_PROBLEM = O.Problem(cfg, xyz, Z)


def _oracle_chunk(idx):
    """Worker of the CPU baseline: the oracle's full-rank canonical sum at one chunk of grid
    points (one process per host core, numpy on one thread each)."""
    _WORKER_PROBLEM.P0_points(idx)
    return len(idx)


def host_cpu():
    """(cores usable by this process, CPU model name) of the host."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    import platform
    return cores, f"{model or 'unknown'} ({platform.machine()})"


class OraclePool:
    """The CPU oracle run over every host core: a process pool (spawn start) whose workers each
    evaluate the full-rank canonical sum on their share of a random sample of grid points."""

    def __init__(self, cfg, parts):
        import multiprocessing as mp
        self.cores, self.model = host_cpu()
        self.cfg, self.xyz, self.Z = dict(cfg), parts.xyz, parts.Z
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_worker_init,
                                                 initargs=(self.cfg, self.xyz, self.Z))
        self.per_point = None

    def close(self):
        self.pool.close()
        self.pool.join()

    def run(self, M: int, seed: int):
        """Wall time of the M-point sample over the pool."""
        import numpy as np
        rng = np.random.default_rng(seed)
        idx = rng.integers(0, int(self.cfg["n"]), (M, 3))
        chunks = np.array_split(idx, self.cores * 4)
        t0 = time.perf_counter()
        self.pool.map(_oracle_chunk, [c for c in chunks if len(c)])
        return time.perf_counter() - t0

    def rate(self, seconds: float, seed: int = 0):
        """Grid points per second over the pool on a random sample sized for about ``seconds``
        of wall time; returns (rate, points, wall seconds)."""
        if self.per_point is None:
            m = 64 * self.cores
            self.run(m, 12344)                     # the workers start and build the problem
            self.per_point = max(self.run(m, 12345), 1e-4) / m
        M = int(max(64 * self.cores, min(20_000_000, seconds / self.per_point)))
        dt = self.run(M, seed)
        self.per_point = dt / M
        return M / dt, M, dt


def workload_config(cfg, N):
    """The workload keys shared by both arms of the bench line."""
    return {"workload": cfg["name"], "N": int(N), "n": int(cfg["n"]), "R": int(cfg["R"]),
            "R_s": int(cfg["R_s"]), "eps": cfg["eps"], "precision": cfg.get("precision")}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from workloads import load_config, make_particles
    cfg = load_config(args.workload)
    parts = make_particles(cfg)
    per_step = float(os.environ.get("RS_REF_STEP_S", "2.0"))
    pool = OraclePool(cfg, parts)
    try:
        for w in range(args.warmup):
            pool.rate(0.2, seed=1000 + w)
        t_total, pts_total, M_last = 0.0, 0, 0
        for s in range(args.steps):
            r, M, dt = pool.rate(per_step, seed=s + 1)
            t_total += dt
            pts_total += M
            M_last = M
    finally:
        pool.close()
    value = pts_total / t_total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(cfg, len(parts.Z)),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "cpu_model": pool.model,
                             "kind": "oracle",
                             "sample": f"{M_last} random grid points per step, full-rank canonical sum "
                                       f"(N*R terms per point), numpy FP64, a process per core"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


SERVING_WORKLOAD = "c4_serving256"
FORCES_WORKLOAD = "c5_forces4096_n513"
LARGE_WORKLOAD = "c3_nacl28_n1025"


def serving_report(max_slots: int = 8, hbm_budget: int = 16 << 30, saturate: bool = False):
    """Replay the serving workload through the library's request loop (``rs_server_*``):
    requests of varying N and n arrive at their Poisson times with host inputs, each computes
    the potential into its own device buffer and the energy; latency is submit to result.
    With ``saturate`` every request is submitted at t = 0 (the loop's capacity: solves/s and
    latency under a full queue)."""
    import numpy as np
    import torch
    from paper_1606_09218_gb300 import RSServer, config_from_workload
    from workloads import load_config, make_serving_requests
    scfg = load_config(SERVING_WORKLOAD)
    sv = scfg["serving"]
    reqs = make_serving_requests(scfg)
    cfgs = {n: config_from_workload(scfg, n=n, max_particles=int(sv["N_max"])) for n in sv["n_choices"]}
    pots = [torch.empty((r.n,) * 3, dtype=torch.float32, device="cuda") for r in reqs]
    torch.cuda.synchronize()
    srv = RSServer(hbm_budget=hbm_budget, max_slots=max_slots)
    # warm-up: one request of each grid size creates a slot of each configuration
    for n in cfgs:
        r = next(q for q in reqs if q.n == n)
        warm = torch.empty((n,) * 3, dtype=torch.float32, device="cuda")
        srv.wait(srv.submit(cfgs[n], r.particles.xyz, r.particles.Z, potential=warm))
    t0 = time.perf_counter()
    tickets = []
    for r, pot in zip(reqs, pots):
        if not saturate:
            dt = t0 + r.arrival_s - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
        tickets.append(srv.submit(cfgs[r.n], r.particles.xyz, r.particles.Z, potential=pot))
    res = [srv.wait(t) for t in tickets]
    span = time.perf_counter() - t0
    info = srv.info()
    srv.close()
    lat = np.array([x["latency_ms"] for x in res])
    que = np.array([x["queue_ms"] for x in res])
    ok = sum(1 for x in res if x["status"] >= 0)
    errors = {}
    for x in res:
        if x["status"] < 0:
            errors[x["message"]] = errors.get(x["message"], 0) + 1
    pts = sum(r.n ** 3 for r in reqs)
    del pots
    arrivals = (f"all {len(reqs)} submitted at t = 0 (saturation)" if saturate else
                f"Poisson, mean gap {sv['mean_gap_ms']} ms, last at {reqs[-1].arrival_s:.3f} s")
    return {"workload": SERVING_WORKLOAD, "requests": len(reqs), "ok": ok, "errors": errors,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "queue_p50_ms": float(np.percentile(que, 50)),
            "queue_p99_ms": float(np.percentile(que, 99)), "span_s": span,
            "solves_per_s": len(reqs) / span, "grid_pts_per_s": pts / span,
            "arrivals": arrivals,
            "max_slots": max_slots, "hbm_budget_bytes": hbm_budget, "slots_at_end": info["slots"],
            "latency": "submit (host inputs) to result (energy on host, potential in a device buffer)"}


def timed_solves(ctx, xyz, Z, pot, steps, flush, stream, forces=False, forces_pair=False):
    """Device milliseconds of ``steps`` solves (CUDA events on the context stream, L2 flushed
    before each) and the per-stage milliseconds per solve."""
    import torch
    ctx.profile(True)
    ctx.profile_read()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    for s in range(steps):
        flush.zero_()
        starts[s].record(stream)
        ctx.solve(xyz, Z, potential=pot, energy=True, want_potential=pot is not None, forces=forces,
                  forces_pair=forces_pair)
        ends[s].record(stream)
    torch.cuda.synchronize()
    t_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    stages, nsolves = ctx.profile_read()
    ctx.profile(False)
    return t_ms, {k: v / max(nsolves, 1) for k, v in stages.items()}


def assembly_roofline(n, r1, per_launch_ms, pk, traffic=None):
    """Roofline of the assembly kernel (Tucker mode-1 product plus the short-range windows, one
    launch per solve): algorithmic bytes = the FP32 output written once, 4 n^3; the Tucker slab
    it reads (T2, r1 x n^2 values stored as FP16 hi/lo pairs, 4 r1 n^2 bytes) is an intermediate
    of this implementation and is reported beside it, not counted."""
    bytes_alg = 4 * n ** 3
    ach = bytes_alg / (per_launch_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": ach / pk["hbm_gbs"],
            "kernel": "assemble_kernel (tcgen05 kind::f16: FP16-split Tucker product and windows, one pass)",
            "traffic": traffic, "traffic_unit": "bytes per launch (ncu dram read + write)",
            "peak_source": pk["source"] + " hbm_gbs (copy, burst)",
            "ms_per_launch": per_launch_ms, "algorithmic_bytes": bytes_alg,
            "bytes_formula": "4*n^3 (FP32 output written once)",
            "t2_read_bytes": 4 * r1 * n * n}


def replica_seed(rank: int, index: int):
    """Particle seed of a rank's replica: rank 0 solves the workload itself (its own seed), every
    other rank an independent seeded problem of the same shape (weak scaling, no collective on
    the data path)."""
    return None if rank == 0 else 160609218 + 1000 * rank + index


def max_over_ranks(x: float, dist, device) -> float:
    """The largest of every rank's x (the slowest rank's time); x itself without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(points_per_step: float, steps: int, world: int, t_max_s: float) -> float:
    """Grid points per second of the whole job: every rank's points over the slowest rank's time."""
    return points_per_step * steps * world / t_max_s


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_1606_09218_gb300 import RSContext, config_from_workload
    from workloads import load_config, make_particles

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    cfg = load_config(args.workload)
    parts = make_particles(cfg, seed=replica_seed(rank, int(cfg["index"])))
    n = int(cfg["n"])
    N = int(len(parts.Z))
    ccfg = config_from_workload(cfg, max_particles=N)
    ctx = RSContext(ccfg)
    stream = torch.cuda.current_stream()
    xyz = torch.tensor(parts.xyz, device="cuda")
    Z = torch.tensor(parts.Z, device="cuda")
    pot = ctx.new_potential()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    pk = peaks()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(3, args.warmup)):
        ctx.solve(xyz, Z, potential=pot, energy=True)
    E = ctx.energy()
    rep = ctx.report()
    # timed region: device time of K solves, L2 flushed before each
    sampler = ClockSampler(local_rank)
    sampler.start()
    barrier()
    t_ms, stages = timed_solves(ctx, xyz, Z, pot, args.steps, flush, stream)
    barrier()
    clocks = sampler.stop()
    launches = ctx.report()["kernel_launches"] * args.steps
    t_ms = max_over_ranks(t_ms, dist, "cuda")
    value = whole_job_rate(n ** 3, args.steps, world, t_ms * 1e-3)

    # end to end through the C ABI with host buffers (pinned): the inputs copied in and the
    # energy read back every step, the potential left in the caller's device buffer
    hx = torch.tensor(parts.xyz).pin_memory()
    hz = torch.tensor(parts.Z).pin_memory()
    hxn, hzn = hx.numpy(), hz.numpy()
    e2e_steps = max(3, min(args.steps, 50))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.solve(hxn, hzn, potential=pot, energy=True)
        ctx.energy()
    t_e2e = time.perf_counter() - t0
    e2e_value = whole_job_rate(n ** 3, e2e_steps, world, max_over_ranks(t_e2e, dist, "cuda"))
    # the same with the whole potential grid copied back to pinned host memory every step
    hpot = torch.empty(pot.shape, dtype=pot.dtype).pin_memory()
    grid_steps = max(3, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for _ in range(grid_steps):
        ctx.solve(hxn, hzn, potential=pot, energy=True)
        hpot.copy_(pot, non_blocking=True)
        ctx.energy()
        torch.cuda.current_stream().synchronize()
    t_grid = time.perf_counter() - t0
    e2e_grid_value = whole_job_rate(n ** 3, grid_steps, world, max_over_ranks(t_grid, dist, "cuda"))
    del hpot

    # plain RS path on the same GPU: every stage in FP64
    plain = None
    if rank == 0 and not args.no_plain:
        pcfg = dict(cfg)
        pcfg["precision"] = "fp64"
        pctx = RSContext(config_from_workload(pcfg, max_particles=N))
        ppot = pctx.new_potential()
        for _ in range(2):
            pctx.solve(xyz, Z, potential=ppot, energy=True)
        ps = max(3, min(args.steps, 10))
        tp, _ = timed_solves(pctx, xyz, Z, ppot, ps, flush, stream)
        plain = {"value": n ** 3 * ps / (tp * 1e-3), "unit": UNIT, "ms_per_step": tp / ps,
                 "path": "same RS pipeline with every stage in FP64 (Tucker core, mode products, output)"}
        pctx.close()
        del ppot

    if rank != 0:
        ctx.close()
        if dist is not None:
            dist.destroy_process_group()
        return 0

    roof = assembly_roofline(n, rep["ranks"][0], stages["reconstruct"], pk,
                             NCU_TRAFFIC.get(kernel_hash()) if args.workload == DEFAULT_WORKLOAD else None)

    # plain-method GPU paths on the same particles and grid: direct sum and full-rank
    # canonical sum (one timed run each after a warm-up), with the RS grid's relative
    # difference from the canonical sum over the whole grid
    plain_methods = None
    if not args.no_plain:
        plain_methods = {}
        ctx.solve(xyz, Z, potential=pot, energy=True)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        outp = torch.empty((n,) * 3, dtype=torch.float32, device="cuda")
        for name, fn, flops in (("direct_sum", ctx.plain_direct, "n^3 N pair terms"),
                                ("canonical_sum", ctx.plain_canonical, "2 n^3 N R")):
            fn(outp)
            torch.cuda.synchronize()
            flush.zero_()
            a.record(stream)
            fn(outp)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            entry = {"ms_per_step": ms, "value": n ** 3 / (ms * 1e-3), "unit": UNIT, "work": flops}
            if name == "canonical_sum":
                entry["rs_rel_diff_full_grid"] = float((pot.double() - outp.double()).norm() / outp.double().norm())
            plain_methods[name] = entry
        del outp

    # two independent solves of the workload at a time, each context on its own stream (the
    # eigen stage leaves most SMs idle): the combined rate of the GPU, beside the sequential
    # per-solve rate of the headline
    concurrent = None
    if not args.no_plain:
        try:
            streams = [torch.cuda.Stream() for _ in range(2)]
            cctx, cpots = [], []
            for st in streams:
                with torch.cuda.stream(st):
                    cctx.append(RSContext(ccfg, stream=st))
                    cpots.append(cctx[-1].new_potential())
            for _ in range(2):
                for cx, pt in zip(cctx, cpots):
                    cx.solve(xyz, Z, potential=pt, energy=True)
            torch.cuda.synchronize()
            csteps = max(4, min(args.steps, 20))
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for i in range(csteps):
                cctx[i & 1].solve(xyz, Z, potential=cpots[i & 1], energy=True)
            torch.cuda.synchronize()
            tc = time.perf_counter() - t0
            concurrent = {"solves": csteps, "streams": 2, "ms_per_solve": 1e3 * tc / csteps,
                          "value": n ** 3 * csteps / tc, "unit": UNIT,
                          "timing": "host wall clock around the solves (synchronised), no L2 flush between them",
                          "energies_equal": cctx[0].energy() == cctx[1].energy() == E}
            for cx in cctx:
                cx.close()
            del cpots
        except Exception as e:  # reported, not fatal to the bench line
            concurrent = {"error": str(e)}

    # the largest workload (lattice, n = 1025, N = 19,757, eps = 1e-5): whole solves timed the
    # same way, with its stage breakdown and the assembly roofline
    large = None
    if not args.no_plain and args.workload != LARGE_WORKLOAD:
        try:
            lcfg = load_config(LARGE_WORKLOAD)
            lp = make_particles(lcfg)
            lctx = RSContext(config_from_workload(lcfg))
            lx = torch.tensor(lp.xyz, device="cuda")
            lz = torch.tensor(lp.Z, device="cuda")
            lpot = lctx.new_potential()
            for _ in range(2):
                lctx.solve(lx, lz, potential=lpot, energy=True)
            lrep = lctx.report()
            ls = 5
            tl, lst = timed_solves(lctx, lx, lz, lpot, ls, flush, stream)
            ln = int(lcfg["n"])
            large = {"workload": LARGE_WORKLOAD, "N": int(len(lp.Z)), "n": ln, "eps": lcfg["eps"],
                     "ms_per_step": tl / ls, "value": ln ** 3 * ls / (tl * 1e-3), "unit": UNIT,
                     "ranks": lrep["ranks"], "subspace": lrep["subspace"], "status": lrep["status"],
                     "energy": lctx.energy(), "stages_ms_per_step": lst,
                     "roofline": assembly_roofline(ln, lrep["ranks"][0], lst["reconstruct"], pk)}
            lctx.close()
            del lpot
        except Exception as e:  # reported, not fatal to the bench line
            large = {"error": str(e)}

    # forces workload (N = 4096, Z = +-1): the RS solve with forces at snapped centres (adjoint,
    # Sec. 4.3), and energy and forces at centres off the grid (the RS kernel in pair form)
    forces = None
    if not args.no_plain:
        fcfg = load_config(FORCES_WORKLOAD)
        fp = make_particles(fcfg)
        fN = int(len(fp.Z))
        fctx = RSContext(config_from_workload(dict(fcfg, snap=True), max_particles=fN))
        fx = torch.tensor(fp.xyz, device="cuda")
        fz = torch.tensor(fp.Z, device="cuda")
        fn_ = int(fcfg["n"])
        fpot = fctx.new_potential()
        for _ in range(2):
            fctx.solve(fx, fz, potential=fpot, energy=True, forces=True)
        fs = 5
        tf, fst = timed_solves(fctx, fx, fz, fpot, fs, flush, stream, forces=True)
        frep = fctx.report()
        tpf, pst = timed_solves(fctx, fx, fz, fpot, 2, flush, stream, forces=True, forces_pair=True)
        fctx.pair_energy_forces(fx, fz)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(torch.cuda.current_stream())
        fE, _ = fctx.pair_energy_forces(fx, fz)
        b.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        fms = a.elapsed_time(b)
        forces = {"workload": FORCES_WORKLOAD, "N": fN, "n": fn_,
                  "solve_with_forces": {"ms_per_step": tf / fs, "value": fn_ ** 3 * fs / (tf * 1e-3),
                                        "unit": UNIT, "ranks": frep["ranks"], "stages_ms_per_step": fst,
                                        "path": "rs_solve with RS_POTENTIAL | RS_ENERGY | RS_FORCES at "
                                                "snapped centres (discrete gradient of the RS-Tucker "
                                                "tensor, Sec. 4.3)"},
                  "solve_with_pair_forces": {"ms_per_step": tpf / 2, "value": fn_ ** 3 * 2 / (tpf * 1e-3),
                                             "unit": UNIT,
                                             "path": "the same with RS_FORCES_PAIR (untruncated long-range "
                                                     "pair kernel, O(N^2 R_l), on the second stream)"},
                  "offgrid_pair": {"ms": fms, "pairs_per_s": fN * (fN - 1) / (fms * 1e-3), "energy": fE,
                                   "path": "rs_pair_energy_forces: RS kernel in pair form at unsnapped "
                                           "centres, FP32 factors, FP64 sums (energy and forces, one call)"}}
        fctx.close()
        del fpot

    # the RS interaction matrix of the grid (Sec. 4.1, case (A)): one product A X with a random
    # X (all R terms, 3R FFT mode passes), and the energy 1/2 <(A - diag A) z, z> (Eq. (4.6)) of
    # the workload's charges through it
    matvec = None
    if not args.no_plain:
        try:
            ctx.solve(xyz, Z, potential=pot, energy=True)
            Xm = torch.randn((n,) * 3, device="cuda", dtype=pot.dtype)
            Ym = ctx.matvec(Xm)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(ctx.stream)
            ctx.matvec(Xm, Ym)
            b.record(ctx.stream)
            torch.cuda.synchronize()
            mv_ms = a.elapsed_time(b)
            Em = ctx.energy_matvec()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Em = ctx.energy_matvec()
            em_ms = 1e3 * (time.perf_counter() - t0)
            R_all = int(cfg["R"])
            mv_bytes = R_all * 3 * 8 * n ** 3 + R_all * 4 * n ** 3     # read + write per pass, + Y reads
            matvec = {"ms": mv_ms, "terms": R_all, "mode_passes": 3 * R_all,
                      "grid_pts_per_s": n ** 3 / (mv_ms * 1e-3),
                      "achieved_gbs": mv_bytes / (mv_ms * 1e-3) / 1e9, "bytes": mv_bytes,
                      "bytes_formula": "3R passes x (read + write of n^3 FP32) + R reads of Y",
                      "energy_matvec_ms": em_ms, "energy_matvec": Em, "energy_rs_tucker": E,
                      "path": "rs_matvec: Kronecker-Toeplitz terms by batched 1-D FFT convolutions "
                              "(circulant size M = 2n - 2); rs_energy_matvec: charges embedded, A - diag A"}
            del Xm, Ym
        except Exception as e:  # reported, not fatal to the bench line
            matvec = {"error": str(e)}

    # RS-canonical form of the last solve (Def. 3.7): the Tucker-to-canonical transform at the
    # accuracy the paper's RS-canonical ranks are quoted at (eps_T2C = 4e-6), and point values of
    # the canonical form (3 R* products per point, Lemma 3.8) against those of the Tucker form
    # (r1 r2 per point, Lemma 3.10), both with the windows, on 2^20 random grid points
    canonical = None
    if not args.no_plain:
        ctx.solve(xyz, Z, potential=pot, energy=True)
        eps_c = 4e-6
        ctx.canonical(eps_c)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Rc = ctx.canonical(eps_c)                    # synchronises
        t2c_ms = 1e3 * (time.perf_counter() - t0)
        g = torch.Generator(device="cuda")
        g.manual_seed(11)
        pts = torch.randint(0, n, (1 << 20, 3), device="cuda", dtype=torch.int32, generator=g)
        rates = {}
        for nm, fn in (("canonical", ctx.canonical_eval_points), ("tucker", ctx.eval_points)):
            fn(pts)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(ctx.stream)
            vals = fn(pts)
            b.record(ctx.stream)
            torch.cuda.synchronize()
            rates[nm] = (vals, pts.shape[0] / (a.elapsed_time(b) * 1e-3))
        canonical = {"eps_t2c": eps_c, "rank": Rc, "tucker_ranks": rep["ranks"], "t2c_ms": t2c_ms,
                     "points": int(pts.shape[0]),
                     "canonical_points_per_s": rates["canonical"][1], "tucker_points_per_s": rates["tucker"][1],
                     "max_abs_diff_vs_tucker": float((rates["canonical"][0] - rates["tucker"][0]).abs().max()),
                     "path": "rs_canonical (FP64 one-sided Jacobi SVD of the core slices), "
                             "rs_canonical_eval_points vs rs_eval_points"}

    # ALS refinement of the canonical-to-Tucker transform (Sec. 6, steps (III)-(V)): one sweep with
    # eps-truncated ranks after a fresh solve, timed as one call (it synchronises once per mode
    # update to read the ranks), the refined grid against the full-rank canonical sum
    als = None
    if not args.no_plain:
        try:
            ctx.solve(xyz, Z, potential=pot, energy=True)
            ctx.tucker_als(1, potential=pot)           # the first call allocates its buffers
            ctx.solve(xyz, Z, potential=pot, energy=True)
            r_rhosvd = ctx.report()["ranks"]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.tucker_als(1, potential=pot)
            torch.cuda.synchronize()
            als_ms = 1e3 * (time.perf_counter() - t0)
            rep_als = ctx.report()
            outp = torch.empty((n,) * 3, dtype=torch.float32, device="cuda")
            ctx.plain_canonical(outp)
            torch.cuda.synchronize()
            als = {"sweeps": 1, "ms": als_ms, "ranks_rhosvd": r_rhosvd, "ranks_als": rep_als["ranks"],
                   "energy": ctx.energy(),
                   "rel_diff_vs_canonical_sum_full_grid":
                       float((pot.double() - outp.double()).norm() / outp.double().norm()),
                   "path": "rs_tucker_als: FP64 mode matrices M = P A over (charged coordinate, k) rows, "
                           "M M^T, the solve's eigen stage and core contraction"}
            del outp
        except Exception as e:  # reported, not fatal to the bench line
            als = {"error": str(e)}

    serving = None
    if not args.no_serving:
        serving = {"poisson": serving_report(), "saturation": serving_report(saturate=True)}

    cpu = None
    if not args.no_cpu:
        pool = OraclePool(cfg, parts)
        try:
            r, M, dt = pool.rate(float(os.environ.get("RS_CPU_SAMPLE_S", "12")))
        finally:
            pool.close()
        cpu = {"value": r, "unit": UNIT, "cores": pool.cores, "cpu_model": pool.model, "kind": "oracle",
               "sample": f"{M} random grid points, full-rank canonical sum (N*R terms per point), "
                         f"numpy FP64, a process per core, {dt:.1f} s"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": dict(workload_config(cfg, N), l2="256 MiB written before every timed step",
                       replicas="one independent seeded problem per rank"),
        "solve": {"ranks": rep["ranks"], "subspace": rep["subspace"], "gamma": rep["gamma"],
                  "status": rep["status"], "energy": E},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(N * 4 * 8),
                "d2h_bytes_per_step": 16, "steps": e2e_steps,
                "output": "potential device-resident (caller's buffer); energy and status read back"},
        "e2e_host_grid": {"value": e2e_grid_value, "unit": UNIT, "h2d_bytes_per_step": int(N * 4 * 8),
                          "d2h_bytes_per_step": int(pot.numel() * pot.element_size()) + 16, "steps": grid_steps,
                          "output": "potential copied to pinned host memory every step"},
        "gpu_launches": launches,
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "stages_ms_per_step": stages,
        "plain_gpu": plain,
        "plain_methods": plain_methods,
        "concurrent": concurrent,
        "large": large,
        "forces": forces,
        "canonical": canonical,
        "matvec": matvec,
        "als": als,
        "serving": serving,
        "energy": E,
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-plain", action="store_true", help="skip the FP64 plain-path comparison")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving replay")
    args = ap.parse_args()
    rank = env_int("RANK", 0)
    world = env_int("WORLD_SIZE", 1)
    local_rank = env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
