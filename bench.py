"""Benchmark of the fused pseudopotential MRT-LBM step (arXiv:1605.01800) on GB300.

Workload (default): the coexistence-curve batch, 32 independent flat liquid
slabs of 256x64 periodic nodes at T/Tc = 0.5 .. 0.95, FP32 deviation storage,
advanced together by one kernel launch per time step. One bench step is one
time step of the whole batch.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Timing: the working set (37.7 MB) fits in the 129 MB L2, so before every timed
step (outside the timed events) a 256 MiB buffer is written and another 256 MiB
buffer is read (evicting the written lines, so their write-back does not land
in the timed step); each step is timed alone with CUDA events on the library's
stream. The FP64-storage path (the plain comparator) is timed the same way.
`sustained` times back-to-back steps (CUDA-graph replay, events around the
whole replay, no flush) on workloads larger than L2, among them the 4096^2
lattice (1.2 GB) on which the sustained HBM fraction is measured. `e2e` times
the public C ABI with host buffers: upload of every density field, one step,
download of every density field. `cpu_baseline` times the FP64 CPU oracle on a
bounded sample, on every host core. Under torchrun every rank advances its own
copy of the batch (weak scaling, no collective on the data path); the
48-lattice Laplace batch is also split across the ranks by node count
(`sharded`, strong scaling), and the collapse lattice into one x-slab per rank
with a halo exchange after every step (`xslab`, strong scaling).
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ALG_BYTES_FP32 = 72   # 9 reads + 9 writes of 4 B per node update
ALG_BYTES_FP64 = 144
# in-place storage: psi pass (9 reads, 1 psi write) + collision (9 reads, the
# node's psi, 9 writes; the neighbours' psi come from L1/L2), 4 B each
ALG_BYTES_INPLACE = 116
WORKLOAD = "coexistence_batch"
PROFILE = os.path.join(ROOT, "profiles", "step_fp32_coexistence_batch.md")
# ncu DRAM bytes of one step of the sustained workloads (same summary format)
SUSTAINED_PROFILES = {"roofline_4096": os.path.join(ROOT, "profiles", "step_fp32_roofline_4096.md")}
INPLACE_PROFILE = os.path.join(ROOT, "profiles", "step_fp32_inplace_roofline_4096.md")
SUSTAINED = ("laplace_batch", "collapse_2048x1024", "roofline_4096", "collapse_x8")
# device sources of each step-kernel kind whose ncu traffic the profile records
# (a pipelined step also launches the plain kernel on its other tiles)
_PLAIN = ("lbm_step.cuh", "lbm_device.cuh", "lbm_step_f32.cu", "lbm_step_f32.inc")
KERNEL_SOURCES = {kind: [os.path.join(ROOT, "paper_1605_01800_gb300", "csrc", f) for f in files]
                  for kind, files in (("plain", _PLAIN), ("pipelined", _PLAIN + ("lbm_step_pipe.cu",)),
                                      ("inplace", ("lbm_device.cuh", "lbm_step_inplace.cu")))}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="time budget of the oracle sample for cpu_baseline")
    ap.add_argument("--profile", default=None, metavar="WORKLOAD",
                    help="profiling mode for ncu: only init and --steps FP32 steps of WORKLOAD "
                         "(coexistence_batch, laplace_batch, collapse_2048x1024, ...) with --tile")
    ap.add_argument("--tile", type=int, default=None, help="step-kernel tile index for --profile")
    ap.add_argument("--precision", default="fp32_dev", help="storage for --profile (fp32_dev, fp32_dev_inplace, ...)")
    return ap.parse_args()


def run_profile(args):
    """A minimal launch sequence for ncu: one context, init, --steps steps."""
    import torch
    from paper_1605_01800_gb300 import inputs, lbm
    torch.cuda.set_device(0)
    specs = inputs.WORKLOADS[args.profile]()
    b = lbm.Batch(specs, args.precision)
    if args.tile is not None:
        lbm.lbm_set_tile(b.ctx, args.tile)
    b.init()
    b.step(args.steps)
    lbm.lbm_sync(b.ctx)
    info = b.info()
    print(json.dumps({"profile": args.profile, "precision": args.precision, "tile_index": args.tile,
                      "tile": [info["tile_x"], info["tile_y"]],
                      "steps": args.steps, "nodes": info["nodes"], "launches": info["kernel_launches"]}))
    b.close()


def kernel_source_hash(kind):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kind]:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(tile, kind, profile=None):
    """DRAM bytes of one step with tile index `tile` (a step kernel of `kind`,
    "plain" or "pipelined") from a committed ncu summary (default: the bench
    workload's), or None when that kernel's source changed since the capture
    or the tile was not captured."""
    profile = profile or PROFILE
    if kind not in KERNEL_SOURCES or not os.path.exists(profile):
        return None
    text = open(profile).read()
    m_hash = re.search(r"kernel_source_sha\[%s\]:\s*([0-9a-f]+)" % kind, text)
    m_bytes = re.search(r"dram_bytes_per_launch\[%d\]:\s*([0-9.eE+]+)" % tile, text)
    if not m_hash or not m_bytes or m_hash.group(1) != kernel_source_hash(kind):
        return None
    return float(m_bytes.group(1))


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of the SM clock, its limit, the throttle reasons and
    the GPU utilisation, taken every `period_ms` until stop(); the summary
    gives the median SM clock over the samples under load (utilisation of
    50% or more; all samples when none is) and every throttle reason seen."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, gpu_index, period_ms=50):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(period_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, loaded, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            try:
                if float(parts[9]) >= 50.0:
                    loaded.append(sm[-1])
            except (IndexError, ValueError):
                pass
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(loaded or sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "samples_under_load": len(loaded), "reasons": sorted(reasons)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle(specs, seconds, threads=1, min_steps=1):
    """FP64 oracle over the whole batch on `threads` host threads, whole time
    steps until `seconds` pass; returns (MLUPS, steps, seconds, threads used)."""
    from oracle import d2q9
    threads = threads if d2q9.set_threads(threads) else 1
    lats = []
    for s in specs:
        L = d2q9.Lattice(s.nx, s.ny, a=s.a, b=s.b, R=s.R, T=s.T, G=s.G, s=s.s, eps=s.eps, solid=s.solid)
        L.init(s.rho)
        lats.append(L)
    nodes = sum(s.nodes for s in specs)
    steps = 0
    t0 = time.perf_counter()
    while True:
        for L in lats:
            L.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if steps >= min_steps and el >= seconds:
            break
    d2q9.set_threads(1)
    return nodes * steps / el / 1e6, steps, el, threads


def run_reference(args, budget_s=150.0):
    """The reference arm: the FP64 CPU oracle as it stands, on the host cores.
    Each of the --warmup + --steps steps advances a bounded sample of the
    workload, the next k of its 32 lattices by one time step (round-robin),
    with k chosen from a one-lattice calibration step so that the whole run
    takes about `budget_s` seconds; MLUPS counts the node updates done."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    from paper_1605_01800_gb300 import inputs
    specs = inputs.coexistence_batch()
    from oracle import d2q9
    cores = host_cores()
    cores = cores if d2q9.set_threads(cores) else 1
    lats = []
    for s in specs:
        L = d2q9.Lattice(s.nx, s.ny, a=s.a, b=s.b, R=s.R, T=s.T, G=s.G, s=s.s, eps=s.eps, solid=s.solid)
        L.init(s.rho)
        lats.append(L)
    t0 = time.perf_counter()
    lats[0].step(1)
    t_lat = time.perf_counter() - t0
    per_step = max(1, min(len(lats), int(budget_s / max(1, args.steps + args.warmup) / t_lat)))
    nxt = [1]

    def one_step():
        done = 0
        for _ in range(per_step):
            L = lats[nxt[0] % len(lats)]
            L.step(1)
            done += L.nx * L.ny
            nxt[0] += 1
        return done

    for _ in range(args.warmup):
        one_step()
    t0 = time.perf_counter()
    updates = sum(one_step() for _ in range(args.steps))
    el = time.perf_counter() - t0
    mlups = updates / el / 1e6
    d2q9.set_threads(1)
    sample = (f"{args.steps} steps of {per_step} of the {len(lats)} lattices each (round-robin), "
              f"{updates} node updates in {el:.1f} s, {cores} thread(s) (OpenMP over the nodes of a lattice)")
    line = {
        "impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattices": len(specs), "nx": 256, "ny": 64,
                   "nodes_per_step": per_step * specs[0].nodes, "precision": "fp64 CPU oracle"},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def flush_l2(flush, sink):
    """Write a buffer larger than L2, then read another one: the write evicts
    the lattice data, the read evicts the dirty lines of the write, so the
    timed step neither hits L2 nor pays for the flush's write-back."""
    flush[0].zero_()
    torch_sum = flush[1].sum(dtype=sink.dtype)
    sink.copy_(torch_sum)


def timed_steps(torch, ctx, lbm, stream, flush, steps):
    """Per-step CUDA-event times (ms) of lbm_step(ctx, 1), L2 flushed before each."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    sink = torch.zeros((), dtype=torch.float32, device=flush[0].device)
    with torch.cuda.stream(stream):
        for e0, e1 in ev:
            flush_l2(flush, sink)
            e0.record(stream)
            lbm.lbm_step(ctx, 1)
            e1.record(stream)
    stream.synchronize()
    return [e0.elapsed_time(e1) for e0, e1 in ev]


def sustained_steps(torch, lbm, specs, stream, tiles, steps=256, warm=32, precision="fp32_dev"):
    """Back-to-back steps of one batch on its own, no flush: CUDA-graph replay
    of `steps` steps with CUDA events around the whole replay, for the fastest
    of `tiles` (each tried on 64 steps from a fresh state). Returns
    (ms per step, tile index, {tile: ms per step of the trial})."""
    b = lbm.Batch(specs, precision, stream=stream)

    def replay(n):
        with torch.cuda.stream(stream):
            lbm.lbm_step(b.ctx, warm)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lbm.lbm_step(b.ctx, n)
            e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / n

    trial = {}
    for t in tiles:
        b.init()
        lbm.lbm_set_tile(b.ctx, t)
        trial[t] = replay(64)
    best = min(trial, key=trial.get)
    b.init()
    lbm.lbm_set_tile(b.ctx, best)
    ms = replay(steps)
    lbm.lbm_sync(b.ctx, allow_flags=True)
    b.close()
    return ms, best, trial


def main():
    args = parse_args()
    if args.profile:
        run_profile(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return

    import numpy as np
    import torch

    world, rank, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    from paper_1605_01800_gb300 import inputs, lbm
    lbm.load()
    specs = inputs.coexistence_batch()
    nodes = sum(s.nodes for s in specs)
    stream = torch.cuda.Stream()
    flush = [torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev),   # 256 MiB > L2
             torch.ones(64 * 1024 * 1024, dtype=torch.float32, device=dev)]

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v):
        if world > 1:
            t = torch.tensor([v], device=dev, dtype=torch.float64)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            v = float(t.item())
        return v

    # clocks over the GPU-busy part of the run: the tile sweep, the timed
    # steps and the sustained runs (the timed steps alone last milliseconds)
    clocks = ClockSampler(dev)

    # ---- FP32 deviation storage (the product path)
    b32 = lbm.Batch(specs, "fp32_dev", stream=stream)
    b32.init()
    # tile shape: the fastest of every shape on flushed single steps (after a
    # warm-up, so the first shape measured pays no first-launch cost)
    timed_steps(torch, b32.ctx, lbm, stream, flush, 30)
    sweep = list(range(lbm.lbm_tile_count()))
    plain = [t for t in sweep if lbm.lbm_tile_kind(t) == lbm.LBM_TILE_PLAIN]
    tile_ms = {}
    for t in sweep:
        lbm.lbm_set_tile(b32.ctx, t)
        tile_ms[t] = statistics.mean(timed_steps(torch, b32.ctx, lbm, stream, flush, 60))
    best_tile = min(tile_ms, key=tile_ms.get)
    lbm.lbm_set_tile(b32.ctx, best_tile)
    b32.init()
    timed_steps(torch, b32.ctx, lbm, stream, flush, max(args.warmup, 3))
    launches0 = b32.info()["kernel_launches"]
    barrier()
    t_wall0 = time.perf_counter()
    ms = timed_steps(torch, b32.ctx, lbm, stream, flush, args.steps)
    barrier()
    t_wall = time.perf_counter() - t_wall0
    launches = b32.info()["kernel_launches"] - launches0
    total_ms = max_over_ranks(sum(ms))
    ms_per_step = total_ms / args.steps
    mlups = world * nodes * args.steps / (total_ms * 1e-3) / 1e6
    lbm.lbm_sync(b32.ctx)

    # steady state with the working set resident in L2 (no flush), for context
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        lbm.lbm_step(b32.ctx, 64)
        e0.record(stream)
        lbm.lbm_step(b32.ctx, 256)
        e1.record(stream)
    stream.synchronize()
    l2_mlups = nodes * 256 / (e0.elapsed_time(e1) * 1e-3) / 1e6

    # ---- sustained steps on workloads larger than L2 (no flush needed)
    peak, peak_kind = measured_peak_hbm()
    kinds = {lbm.LBM_TILE_PLAIN: "plain", lbm.LBM_TILE_PIPELINED: "pipelined"}
    sustained = {}
    for name in SUSTAINED:
        lspecs = inputs.WORKLOADS[name]()
        lnodes = sum(s.nodes for s in lspecs)
        # every shape, the TMA-staged ones too where the batch allows them
        tiles = sweep if len(lspecs) <= 64 else [t for t in sweep if lbm.lbm_tile_kind(t) != lbm.LBM_TILE_TMA]
        lms, lt, trial = sustained_steps(torch, lbm, lspecs, stream, tiles)
        gbs = ALG_BYTES_FP32 * lnodes / (lms * 1e-3) / 1e9
        entry = {"nodes": lnodes, "working_set_bytes": 2 * 36 * lnodes, "tile": lbm.lbm_tile_shape(lt),
                 "tile_index": lt, "steps": 256, "ms_per_step": lms, "MLUPS": lnodes / (lms * 1e-3) / 1e6,
                 "achieved_gbs": gbs, "frac": gbs / peak,
                 "tile_trial_us": {str(t): round(1e3 * v, 2) for t, v in trial.items()}}
        if name in SUSTAINED_PROFILES:
            tr = profiled_traffic(lt, kinds.get(lbm.lbm_tile_kind(lt)), SUSTAINED_PROFILES[name])
            entry["dram_bytes_per_node"] = None if tr is None else tr / lnodes
        sustained[name] = entry
        del lspecs

    # ---- in-place storage on the 4096^2 lattice (one distribution array)
    ispecs = inputs.WORKLOADS["roofline_4096"]()
    inodes = sum(s.nodes for s in ispecs)
    ims, it, itrial = sustained_steps(torch, lbm, ispecs, stream, plain, precision="fp32_dev_inplace")
    igbs = ALG_BYTES_INPLACE * inodes / (ims * 1e-3) / 1e9
    inplace = {"workload": "roofline_4096", "nodes": inodes, "distribution_bytes": 36 * inodes,
               "tile": lbm.lbm_tile_shape(it), "tile_index": it, "steps": 256, "ms_per_step": ims,
               "MLUPS": inodes / (ims * 1e-3) / 1e6, "alg_bytes_per_node": ALG_BYTES_INPLACE,
               "achieved_gbs": igbs, "frac": igbs / peak,
               "vs_two_buffers": sustained["roofline_4096"]["ms_per_step"] / ims,
               "dram_bytes_per_node": (lambda tr: None if tr is None else tr / inodes)(
                   profiled_traffic(it, "inplace", INPLACE_PROFILE)),
               "tile_trial_us": {str(t): round(1e3 * v, 2) for t, v in itrial.items()},
               "note": "LBM_INPLACE: one array, psi pass + in-place collision per step, CUDA-graph replay"}
    del ispecs
    clk = clocks.stop()

    # ---- the Laplace batch split across the ranks by node count (strong
    # scaling; one rank alone advances the whole batch)
    sharded = None
    if world > 1:
        try:
            from paper_1605_01800_gb300 import sharding
            lspecs = inputs.laplace_batch()
            mine = sharding.shard(lspecs, rank, world)
            barrier()
            sms = sustained_steps(torch, lbm, mine, stream, [3])[0] if mine else 0.0
            sms = max_over_ranks(sms)
            lnodes = sum(s.nodes for s in lspecs)
            sharded = {"workload": "laplace_batch", "lattices": len(lspecs), "ranks": world,
                       "ms_per_step": sms, "MLUPS": lnodes / (sms * 1e-3) / 1e6,
                       "note": "LPT shares by node count, each rank steps its own share, max over ranks"}
        except Exception as exc:  # the headline line must still be printed
            sharded = {"error": f"{type(exc).__name__}: {exc}"[:300]}

    # ---- one lattice split into x-slabs across the ranks (strong scaling):
    # the collapse lattice, each rank its slab, a halo exchange after every
    # step (NCCL point-to-point); reported, not fatal, if it fails
    xsl = None
    if world > 1:
        try:
            from paper_1605_01800_gb300 import xslab
            (cspec,) = inputs.collapse()
            rs = xslab.RankSlab(cspec, "fp32_dev", stream=stream, overlap=True)
            rs.step(10)
            barrier()
            t0 = time.perf_counter()
            k_x = 200
            rs.step(k_x)
            barrier()
            xs = max_over_ranks(time.perf_counter() - t0)
            rs.close()
            xsl = {"workload": "collapse_2048x1024", "ranks": world, "steps": k_x, "ms_per_step": 1e3 * xs / k_x,
                   "MLUPS": cspec.nodes * k_x / xs / 1e6,
                   "note": "x-slabs, one per rank, halo exchange (12 values per row and face) every step, "
                           "overlapped with the interior tiles (split step), wall-clock over the ranks"}
        except Exception as exc:  # the headline line must still be printed
            xsl = {"error": f"{type(exc).__name__}: {exc}"[:300]}

    # ---- e2e through the C ABI with host buffers
    rho_in = torch.empty(nodes, dtype=torch.float64, pin_memory=True).numpy()
    rho_in[:] = np.concatenate([s.rho.ravel() for s in specs])
    rho_out = torch.empty(nodes, dtype=torch.float64, pin_memory=True).numpy()
    e2e_steps = max(3, min(args.steps, 50))
    for _ in range(2):
        lbm.lbm_init_fields_all(b32.ctx, rho_in)
        lbm.lbm_step(b32.ctx, 1)
        lbm.lbm_read_moments_all(b32.ctx, rho_out)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        lbm.lbm_init_fields_all(b32.ctx, rho_in)
        lbm.lbm_step(b32.ctx, 1)
        lbm.lbm_read_moments_all(b32.ctx, rho_out)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e_mlups = world * nodes * e2e_steps / e2e_s / 1e6
    b32.close()

    # ---- FP64 plain storage (the comparator)
    b64 = lbm.Batch(specs, "fp64", stream=stream)
    b64.init()
    timed_steps(torch, b64.ctx, lbm, stream, flush, 3)
    k64 = max(3, min(args.steps, 50))
    ms64 = timed_steps(torch, b64.ctx, lbm, stream, flush, k64)
    fp64_ms = sum(ms64) / k64
    fp64_mlups = nodes / (fp64_ms * 1e-3) / 1e6
    b64.close()

    # ---- the error that goes with the FP32 number: fresh FP32 and FP64 runs
    # of the same batch for the same steps, densities compared node by node
    acc_steps = 500
    rho = {}
    for prec in ("fp32_dev", "fp64"):
        ba = lbm.Batch(specs, prec, stream=stream)
        ba.init()
        ba.step(acc_steps)
        out = np.empty(nodes)
        lbm.lbm_read_moments_all(ba.ctx, out)
        rho[prec] = out
        ba.close()
    acc = {"steps": acc_steps, "max_rel_rho": float(np.max(np.abs(rho["fp32_dev"] / rho["fp64"] - 1.0))),
           "mean_rel_rho": float(np.mean(np.abs(rho["fp32_dev"] / rho["fp64"] - 1.0))),
           "note": "FP32 deviation storage against FP64 storage, every node of the batch"}

    # ---- context: a plain device copy of the same bytes under the same flush
    src = torch.empty(nodes * 9, dtype=torch.float32, device=dev)
    dst = torch.empty_like(src)
    cev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(30)]
    sink = torch.zeros((), dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        for e0, e1 in cev:
            flush_l2(flush, sink)
            e0.record(stream)
            dst.copy_(src)
            e1.record(stream)
    stream.synchronize()
    copy_ms = statistics.mean([a.elapsed_time(b) for a, b in cev])
    copy_gbs = 2 * src.numel() * 4 / (copy_ms * 1e-3) / 1e9
    del src, dst

    achieved = ALG_BYTES_FP32 * nodes / (ms_per_step * 1e-3) / 1e9
    traffic = profiled_traffic(best_tile, kinds.get(lbm.lbm_tile_kind(best_tile)))

    line = {
        "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattices": len(specs), "nx": 256, "ny": 64,
                   "nodes_per_step_per_gpu": nodes, "precision": "fp32 deviation storage",
                   "tile": lbm.lbm_tile_shape(best_tile),
                   "tile_sweep_us": {"x".join(map(str, lbm.lbm_tile_shape(t))) + f"/{t}": round(1e3 * v, 2)
                                     for t, v in tile_ms.items()},
                   "l2": "before every timed step: 256 MiB buffer written, then another 256 MiB read",
                   "parallelism": f"{world} independent batch replica(s), no collective"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"{peak_kind} hbm_gbs", "alg_bytes_per_node": ALG_BYTES_FP32},
        "sustained": dict(sustained, note="back-to-back steps, CUDA-graph replay of 256 steps, events around "
                                          "the replay, no flush; working sets larger than L2 (129 MB)"),
        "inplace": inplace,
        "copy_same_bytes": {"achieved_gbs": copy_gbs, "ms": copy_ms, "frac": copy_gbs / peak,
                            "note": "torch device copy of 9 x 4 B per node, same flush"},
        "fp32_vs_fp64": acc,
        "fp64_plain": {"value": fp64_mlups, "unit": "MLUPS", "ms_per_step": fp64_ms, "steps": k64,
                       "achieved_gbs": ALG_BYTES_FP64 * nodes / (fp64_ms * 1e-3) / 1e9},
        "l2_resident": {"value": l2_mlups, "unit": "MLUPS",
                        "note": "256 back-to-back steps in CUDA graphs without flushing L2"},
        "e2e": {"value": e2e_mlups, "unit": "MLUPS", "steps": e2e_steps,
                "h2d_bytes_per_step": nodes * 8, "d2h_bytes_per_step": nodes * 8,
                "path": "lbm_init_fields_all(host rho) + lbm_step(1) + lbm_read_moments_all(host rho)"},
        "gpu_launches": launches,
        "clocks": clk,
        "wall_s_timed_loop": t_wall,
    }
    if sharded is not None:
        line["sharded"] = sharded
    if xsl is not None:
        line["xslab"] = xsl
    if rank == 0 and world == 1:
        cores = host_cores()
        cpu_mlups, cpu_steps, cpu_s, used = time_oracle(specs, args.cpu_seconds, threads=cores)
        one_mlups, one_steps, one_s, _ = time_oracle(specs, max(2.0, args.cpu_seconds / 4), threads=1)
        line["cpu_baseline"] = {"value": cpu_mlups, "unit": "MLUPS", "cores": used, "kind": "oracle",
                                "sample": f"{cpu_steps} whole time steps of all {len(specs)} lattices "
                                          f"({cpu_s:.1f} s, {used} threads, OpenMP over the nodes)",
                                "single_thread": {"value": one_mlups, "steps": one_steps, "seconds": one_s}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
