"""Throughput of the sparse FastTucker SGD hot path on GB300.

One step = one epoch of Algorithm 2 over a Netflix-shaped synthetic ratings
tensor (480000 x 17800 x 2200, 100M nonzeros, Zipf(1.1) user / item modes,
integer values 1-5, J = R = 16, float32; 90M train / 10M test):
  for every mode: factor pass + refresh of C^(n);
  for every mode: core pass (gradient accumulated over the whole pass and one
  update, Algorithm 5) + refresh of C^(n);
  then the test-set residual sums (RMSE / MAE).
Default path: the nonzeros of each mode are kept in its slice layout (the CSF
slices of Section "Tensor Storage Format", built once before timing) and the
factor pass runs every slice element by element (Algorithm 4 order); with
--path coo the factor pass is the Hogwild COO kernel instead.
value = training nonzeros / epoch time.  Inputs live in HBM (several GB,
larger than L2); `e2e` repeats the step with the step's inputs (each slice
layout as values, row pointers, fiber ids and fiber coordinates, whose
coordinate arrays the step rebuilds on the device, and the test set) copied
from pinned host memory inside the timed region and the loss read back;
`e2e_raw` starts from the raw COO and also builds every layout each step.

--impl reference times the FP64 CPU oracle on a bounded prefix of the same
workload (the only CPU code this script runs).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_PATH = os.path.join(ROOT, "profiles", "dram_traffic.json")
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--nnz", type=int, default=100_000_000)
    p.add_argument("--core-batch", type=int, default=0, help="0 = whole pass (Algorithm 5)")
    p.add_argument("--cpu-sample", type=int, default=2_000_000,
                   help="nonzeros of the oracle's bounded CPU sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--path", default="slices", choices=["slices", "coo"])
    p.add_argument("--prec", default="fp32", choices=["fp32", "bf16"],
                   help="storage of the cached products C (arithmetic is float32 either way)")
    p.add_argument("--workload", default="ratings",
                   choices=["ratings", "order8", "autograd", "batch", "sparsity"],
                   help="ratings: 480000x17800x2200, 100M nnz, J=R=16; order8: 8 modes of "
                        "10000, 50M nnz, J=R=32; autograd: loss forward + backward over 4 "
                        "modes of 100000, 20M nnz, J=R=32; batch: 64 independent problems "
                        "(order 3-6, dims 1k-200k, nnz 10k-5M, J=R in 4..32) in one "
                        "persistent launch per epoch; sparsity: order 3, 1000^3, 20M..100M nnz "
                        "(2%%..10%% dense), J=R=16, one line with every density")
    p.add_argument("--lr", type=float, default=0.0,
                   help="SGD step for A and B (0 = 0.01 for ratings, 1e-5 for order8)")
    p.add_argument("--fibers", default="auto", choices=["auto", "on", "off"],
                   help="form v once per fiber (tuple of the other modes' coordinates) in the "
                        "factor pass: on, off, or auto = for modes with at most nnz/2 fibers")
    p.add_argument("--epochs-rmse", type=int, default=10,
                   help="epochs of the per-epoch test-RMSE curves (float32 and bfloat16 C, "
                        "same init; 0 = skip the curves and the bfloat16 block)")
    p.add_argument("--no-e2e-raw", action="store_true",
                   help="skip the end-to-end figure that rebuilds the slice layouts and fiber "
                        "tables from raw COO every step")
    p.add_argument("--order", default="storage", choices=["csf", "storage"],
                   help="visit order of the nonzeros inside each slice: the paper's B-CSF "
                        "traversal (sorted by the other modes' coordinates) or storage order")
    p.add_argument("--blocked-chains", default="on", choices=["on", "off"],
                   help="chains of 256+ nonzeros of the fiber pass in 32-position blocks "
                        "(Gram matrix on the tensor cores + triangular solve) or element by "
                        "element")
    p.add_argument("--long-slices", default="maps", choices=["maps", "subslices"],
                   help="long slices exactly through composed maps (Algorithm 4 order), or as "
                        "concurrent sub-slices merged with atomic adds (the paper's B-CSF manner)")
    p.add_argument("--slice-tile", type=int, default=0, help="slice tile length (0 = automatic)")
    p.add_argument("--slice-max-direct", type=int, default=0,
                   help="longest crossing slice run element by element (0 = automatic)")
    return p.parse_args()


# ----------------------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi samples (SM clock, throttle reasons) during the timed region.
    Sampling runs every 50 ms; __enter__ returns once the first sample has
    arrived (so the sampler is running when the timed region starts), and
    summary() keeps the samples that arrived between __enter__ and __exit__."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.lines = []  # (arrival time, csv line)
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            deadline = time.time() + 5.0
            while not self.lines and time.time() < deadline and self.proc.poll() is None:
                time.sleep(0.01)
        except FileNotFoundError:
            self.proc = None
        self.t0 = time.time()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def __exit__(self, *a):
        self.t1 = time.time()
        if self.proc:
            time.sleep(0.06)  # the sample that covers the end of the region
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t1 = (self.t1 or time.time()) + 0.06
        for ts, ln in self.lines:
            if self.t0 is not None and not (self.t0 <= ts <= t1):
                continue
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- helpers


def source_digest(paths) -> str:
    """sha256 over the bytes of the given repository files, in the given order."""
    import hashlib
    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(rel.encode() + b"\0" + f.read())
    return h.hexdigest()


def measured_traffic(key: str):
    """DRAM bytes (read + write) per launch of a timed unit, from the committed
    record of an ncu capture (profiles/dram_traffic.json), or None when there is
    no record for `key` or the kernels' sources changed since it was taken."""
    try:
        with open(TRAFFIC_PATH) as f:
            rec = json.load(f)[key]
        if source_digest(rec["sources"]) != rec["digest"]:
            return None
        return float(rec["bytes_per_launch"])
    except (OSError, KeyError, ValueError, TypeError):
        return None


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


_REDUCE_DEVICE = "cpu"


def dist_setup(args=None):
    """One process per GPU (torchrun env vars); NCCL with GPUs, gloo without.
    Returns (world, rank, local_rank)."""
    global _REDUCE_DEVICE
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            _REDUCE_DEVICE = "cuda"
        if not dist.is_initialized():
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """Timing is the slowest rank's (max over ranks)."""
    if world == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_REDUCE_DEVICE)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world):
    """Work is summed over ranks (each rank runs its own replica)."""
    if world == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_REDUCE_DEVICE)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def replica_rate(local_units, local_seconds, world):
    """Whole-job throughput of independent replicas: all ranks' units over the
    slowest rank's time (weak scaling)."""
    return sum_over_ranks(float(local_units), world) / max_over_ranks(float(local_seconds), world)


def algorithmic_bytes(N, J, R, path="coo", rows_per_nnz=1.0, c_bytes=4):
    """Bytes per nonzero of one factor / core pass: the COO entry, the N-1
    gathered C rows (c_bytes per entry: 4 float32, 2 bfloat16), and the float32
    factor row (read + write for the factor pass, read for the core pass).  On
    the slice layout a factor row is read and written once per slice instead of
    once per nonzero, so its bytes are scaled by rows_per_nnz = rows / nnz."""
    coo = 4 * N + 4
    gather = (N - 1) * R * c_bytes
    f = rows_per_nnz if path == "slices" else 1.0
    return coo + gather + 2 * J * 4 * f, coo + gather + J * 4 * f


# ----------------------------------------------------------------------------- e2e inputs


def e2e_groups(inp, N: int):
    """The device tensors an end-to-end step copies from the host, one group per
    mode and one for the test set (a mode's pass waits only for its group).
    A slice layout ships its values, row_ptr and, with fibers, its fiber ids
    and the first nfibers entries of its fiber coordinates.  Its coordinate
    arrays are not shipped where the step rebuilds them on the device: the
    own mode's from row_ptr (sft_slices_expand_rows), the other modes' from
    fid and fcoord (sft_fibers_expand_coords) when the mode has fibers.  On
    the COO path the whole set is the first group."""
    if inp["slices"]:
        gs = [([t for k, t in enumerate(sl.idx) if k != sl.mode]
               if sl.fid is None else []) + [sl.val, sl.row_ptr]
              + ([sl.fid] + [c[:sl.nfibers] for c in sl.fcoord if c is not None]
                 if sl.fid is not None else [])
              for sl in inp["slices"]]
    else:
        gs = [list(inp["idx"]) + [inp["val"]]] + [[] for _ in range(N - 1)]
    return gs + [list(inp["tidx"]) + [inp["tval"]]]


def e2e_clone_set(inp):
    """A second set of device buffers shaped like `inp` (the e2e steps
    alternate between two, so that step k+1's copies overlap step k)."""
    import copy as copy_mod
    out = dict(inp)
    if inp["slices"]:
        sl2 = []
        for sl in inp["slices"]:
            c = copy_mod.copy(sl)
            c.idx = [torch.empty_like(t) for t in sl.idx]
            c.val = torch.empty_like(sl.val)
            c.row_ptr = torch.empty_like(sl.row_ptr)
            if sl.fid is not None:
                c.fid = torch.empty_like(sl.fid)
                c.fcoord = [None if t is None else torch.empty_like(t) for t in sl.fcoord]
            sl2.append(c)
        out["slices"] = sl2
    else:
        out["idx"] = [torch.empty_like(t) for t in inp["idx"]]
        out["val"] = torch.empty_like(inp["val"])
    out["tidx"] = [torch.empty_like(t) for t in inp["tidx"]]
    out["tval"] = torch.empty_like(inp["tval"])
    return out


# ----------------------------------------------------------------------------- CPU oracle


def cpu_oracle_grad_rate(T, sample: int):
    """Oracle loss and gradient (FP64, single thread) over the first `sample`
    nonzeros; returns (nonzeros per second, seconds, sample)."""
    import oracle
    oracle.build()
    S = min(sample, T.nnz)
    idx = [i[:S].cpu().numpy() for i in T.idx]
    val = T.val[:S].cpu().numpy()
    m = oracle.Model([a.cpu().numpy() for a in T.A0], [b.cpu().numpy() for b in T.B0])
    t0 = time.perf_counter()
    m.refresh_all()
    m.loss_grad(idx, val)
    dt = time.perf_counter() - t0
    return S / dt, dt, S


def cpu_oracle_epoch_rate(T, sample: int, order: str = "storage"):
    """Oracle (FP64, single thread) on the first `sample` training nonzeros with
    the same schedule (factor rows element by element in the same visit order,
    core once per pass); returns (nonzeros per second, seconds, sample)."""
    import numpy as np
    import oracle
    from paper_2210_06014_gb300 import synth
    oracle.build()
    S = min(sample, T.nnz)
    idx = [i[:S].cpu().numpy() for i in T.idx]
    val = T.val[:S].cpu().numpy()
    pf = None
    if order == "csf":
        tix = [i[:S].cpu() for i in T.idx]
        pf = [synth.csf_order(tix, n).numpy().astype(np.uint32) for n in range(len(idx))]
    m = oracle.Model([a.cpu().numpy() for a in T.A0], [b.cpu().numpy() for b in T.B0])
    t0 = time.perf_counter()
    m.epoch(idx, val, pf, None, batch_factor=1, batch_core=S)
    dt = time.perf_counter() - t0
    return S / dt, dt, S


# ----------------------------------------------------------------------------- batch


def stable_lrs(Ts, cap, c=0.5):
    """Per-problem SGD step kept below c / max_s |v_s|^2 at the initial
    parameters (one step scales a row along v by 1 - lr |v|^2; the products of
    N - 1 cached rows are heavy-tailed at high order and rank).  Setup only."""
    out = []
    for T in Ts:
        A = [a.double() for a in T.A0]
        B = [b.double() for b in T.B0]
        C = [a @ b for a, b in zip(A, B)]
        vmax = 0.0
        for n in range(len(A)):
            p = None
            for k in range(len(A)):
                if k != n:
                    rows = C[k][T.idx[k].long()]
                    p = rows if p is None else p * rows
            v = p @ B[n].T
            vmax = max(vmax, float((v * v).sum(1).max()))
            del p, v
        out.append(min(cap, c / vmax) if vmax > 0 else cap)
    return out


def run_batch(args, world, rank, lr):
    """One step = one epoch of Algorithm 2 for each of 64 independent problems
    (one graph launch of the persistent kernel; tiles autotuned first)."""
    from paper_2210_06014_gb300 import synth
    specs = synth.spec_batch(64, seed=0)
    total_nnz = sum(s.nnz for s in specs)
    metric = "SGD nonzeros/s (factor+core updates)"
    unit = "nnz/s"
    workload = f"batch64-order3to6-dims1k-200k-nnz10k-5M-R4to32 ({total_nnz} nnz)"
    if args.impl == "reference":
        if rank != 0:
            return
        big = max(specs, key=lambda s: s.nnz)
        T = synth.make_tensor(big, device="cuda" if torch.cuda.is_available() else "cpu")
        steps = []
        for i in range(args.warmup + args.steps):
            rate, dt, S = cpu_oracle_epoch_rate(T, max(10_000, args.cpu_sample // 4))
            if i >= args.warmup:
                steps.append((rate, dt))
        rate = statistics.median(r for r, _ in steps)
        print(json.dumps({
            "impl": "reference", "metric": metric, "value": rate, "unit": unit, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.median(d for _, d in steps) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload, "sample_nnz": S},
            "cpu_baseline": {"value": rate, "unit": unit, "cores": 1, "kind": "oracle",
                             "sample": f"first {S} nonzeros of the largest problem, one epoch"},
            "e2e": {"value": rate, "unit": unit, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}))
        return
    from paper_2210_06014_gb300 import sft
    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = time.perf_counter()
    Ts = [synth.make_tensor(s, device=dev) for s in specs]
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    prec = sft.SFT_BF16 if args.prec == "bf16" else sft.SFT_FP32
    lrs = stable_lrs(Ts, lr)
    b = sft.Batch([(T.A0, T.B0, list(T.idx), T.val) for T in Ts], prec=prec, min_chunk=1024,
                  lr=lrs, lam=0.01)
    t0 = time.perf_counter()
    chunk, bps = b.autotune(epochs=2)
    tune_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        b.epoch()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    l0 = b.launches
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        torch.cuda.nvtx.range_push("timed")
        start.record(stream)
        for _ in range(args.steps):
            b.epoch()
        end.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    barrier(world)
    launches = (b.launches - l0) * 2  # counter reset + persistent kernel per graph
    b.sync(600_000)
    elapsed = start.elapsed_time(end) / 1e3
    elapsed_max = max_over_ranks(elapsed, world)
    value = replica_rate(total_nnz * args.steps, elapsed, world)
    c_bytes = 2 if args.prec == "bf16" else 4
    byts = 0.0
    for s in specs:
        fac, core = algorithmic_bytes(s.order, s.R, s.R, "coo", 1.0, c_bytes)
        byts += s.order * s.nnz * (fac + core)
        byts += 2 * sum(I * (s.R + s.R) * 4 for I in s.dims)  # two refreshes per mode
    ep_s = elapsed / args.steps
    peak, peak_kind = peaks()
    ach = byts / ep_s / 1e9
    rmse = b.rmse()

    e2e = None
    if not args.no_e2e:
        dev_in = [t for T in Ts for t in list(T.idx) + [T.val]]
        host_in = [t.cpu().pin_memory() for t in dev_in]
        h2d = sum(t.numel() * t.element_size() for t in host_in)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(args.steps):
            for d, h in zip(dev_in, host_in):
                d.copy_(h, non_blocking=True)
            b.epoch()
            b.loss()  # synchronises and reads the per-problem sums back
        et = max_over_ranks(time.perf_counter() - t1, world)
        e2e = {"value": sum_over_ranks(float(total_nnz * args.steps), world) / et, "unit": unit,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 16 * len(specs),
               "includes": "input copies, epoch, loss pass and its readback"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        big = max(range(len(specs)), key=lambda i: specs[i].nnz)
        rate, dt, S = cpu_oracle_epoch_rate(Ts[big], args.cpu_sample)
        cpu = {"value": rate, "unit": unit, "cores": 1, "kind": "oracle",
               "sample": f"first {S} nonzeros of the largest problem, one epoch ({dt:.1f} s)"}
    if rank == 0:
        print(json.dumps({
            "metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_max / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "c_storage": args.prec,
            "config": {
                "workload": workload, "problems": len(specs), "nnz": total_nnz,
                "parallelism": "replicas only" if world > 1 else "single GPU",
                "schedule": "per problem: Hogwild factor pass + refresh per mode, then whole-pass "
                            "core update + refresh per mode; all problems in one persistent "
                            "launch (CUDA graph)",
                "autotuned": {"chunk": chunk, "blocks_per_sm": bps, "seconds": round(tune_s, 2)},
                "epoch_tasks": b.epoch_tasks,
                "lr": {"rule": "min(cap, 0.5 / max |v|^2 at init) per problem", "cap": lr,
                       "min": min(lrs), "max": max(lrs)},
                "lambda": 0.01,
                "l2": "inputs larger than L2", "generation_s": round(gen_s, 2),
                "train_rmse_after": {"min": min(rmse), "median": statistics.median(rmse),
                                     "max": max(rmse)},
            },
            "roofline": {"bound": "hbm", "kernel": "persistent batch kernel", "achieved": ach,
                         "peak": peak, "unit": "GB/s", "frac": ach / peak, "traffic": None,
                         "peak_source": peak_kind},
            "clocks": clk.summary(),
            "gpu_launches": launches,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- sparsity


def run_sparsity(args, world, rank, lr):
    """The SGD epoch on order-3 1000^3 tensors with 20M, 40M, ..., 100M nonzeros
    (Synthetic(Sparsity)); the line's value is the 100M tensor, config.sweep has
    every density (factor and core time per epoch separately)."""
    from paper_2210_06014_gb300 import synth
    metric = "SGD nonzeros/s (factor+core updates)"
    unit = "nnz/s"
    if args.impl == "reference":
        if rank != 0:
            return
        T = synth.make_tensor(synth.spec_sparsity(100_000_000),
                              device="cuda" if torch.cuda.is_available() else "cpu")
        steps = []
        for i in range(args.warmup + args.steps):
            rate, dt, S = cpu_oracle_epoch_rate(T, max(10_000, args.cpu_sample // 4))
            if i >= args.warmup:
                steps.append((rate, dt))
        rate = statistics.median(r for r, _ in steps)
        print(json.dumps({
            "impl": "reference", "metric": metric, "value": rate, "unit": unit, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.median(d for _, d in steps) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "sparsity-1000^3-100M-J16R16", "sample_nnz": S},
            "cpu_baseline": {"value": rate, "unit": unit, "cores": 1, "kind": "oracle",
                             "sample": f"first {S} training nonzeros, one epoch"},
            "e2e": {"value": rate, "unit": unit, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}))
        return
    from paper_2210_06014_gb300 import sft
    dev = torch.device("cuda", torch.cuda.current_device())
    sweep, last = [], None
    sizes = [20_000_000, 40_000_000, 60_000_000, 80_000_000, 100_000_000]
    for i, nz in enumerate(sizes):
        spec = synth.spec_sparsity(nz)
        t0 = time.perf_counter()
        T = synth.make_tensor(spec, device=dev)
        torch.cuda.synchronize()
        gen_s = time.perf_counter() - t0
        final = i == len(sizes) - 1
        line = run_sgd(args, world, rank, sft, T, spec, metric, unit, gen_s, lr, print_line=False,
                       extras=final)
        if rank == 0:
            c = line["config"]
            sweep.append({"nnz": nz, "density": nz / 1e9, "value": line["value"],
                          "ms_per_step": line["ms_per_step"],
                          "factor_ms": c["per_step_ms"]["factor"],
                          "core_ms": c["per_step_ms"]["core"],
                          "factor_nnz_per_s": c["train_nnz"] * spec.order
                          / (c["per_step_ms"]["factor"] / 1e3),
                          "core_nnz_per_s": c["train_nnz"] * spec.order
                          / (c["per_step_ms"]["core"] / 1e3),
                          "test_rmse_after": c["test_rmse_after"]})
            last = line
        del T
        torch.cuda.empty_cache()
    if rank == 0:
        last["config"]["sweep"] = sweep
        last["config"]["workload"] = "sparsity-1000^3-20M..100M-J16R16 (value: 100M)"
        print(json.dumps(last))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- autograd


def run_autograd(args, world, rank, sft, T, spec, metric, unit, gen_s):
    """One step = forward + backward of the sampled loss L = 1/2 sum e^2 over
    every nonzero through sft.SampledLoss (refresh of every C^(n), the fused
    loss + dL/dC pass, then dL/dA and dL/dB for every mode)."""
    dev = T.val.device
    N, J, R = spec.order, spec.J[0], spec.R
    nnz = T.nnz
    idx, val = list(T.idx), T.val
    prec = sft.SFT_BF16 if args.prec == "bf16" else sft.SFT_FP32
    mod = sft.SampledLoss(T.A0, T.B0, prec=prec)
    stream = torch.cuda.current_stream()
    fw, bw = [], []

    def step(timed, src=None):
        if src is not None:
            for d, h in zip(src[0], src[1]):
                d.copy_(h, non_blocking=True)
        for p in mod.parameters():
            p.grad = None
        if timed:
            a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record(stream)
        loss = mod(idx, val)
        if timed:
            b.record(stream)
        loss.backward()
        if timed:
            c.record(stream)
            fw.append((a, b))
            bw.append((b, c))
        return loss

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    launches0 = mod.dec.launches
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        torch.cuda.nvtx.range_push("timed")
        start.record(stream)
        for _ in range(args.steps):
            loss = step(True)
        end.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    barrier(world)
    launches = mod.dec.launches - launches0
    mod.dec.sync(600_000)
    elapsed = start.elapsed_time(end) / 1e3
    elapsed_max = max_over_ranks(elapsed, world)
    total_nnz = sum_over_ranks(float(nnz * args.steps), world)
    value = replica_rate(nnz * args.steps, elapsed, world)
    f_ms = sum(a.elapsed_time(b) for a, b in fw) / len(fw)
    b_ms = sum(a.elapsed_time(b) for a, b in bw) / len(bw)
    # forward: COO entry, N gathered C rows, one R-float gradient row per mode
    # per nonzero; the C tables and the dL/dC accumulators (N I R floats each)
    # stay in L2, so of these only the COO stream and one read of C plus one
    # write of dL/dC must reach DRAM: the roofline counts those bytes (the
    # kernel is bound by its dependent L2 gathers, not by DRAM)
    fwd_bytes = 4 * N + 4 + N * R * 4 + N * R * 4
    table_bytes = 2 * sum(int(d) for d in spec.dims) * R * 4
    dram_bytes = (4 * N + 4) * nnz + table_bytes
    peak, peak_kind = peaks()
    ach = dram_bytes / (f_ms / 1e3) / 1e9
    loss_v = float(loss.item())

    e2e = None
    if not args.no_e2e:
        dev_in = idx + [val]
        host_in = [t.cpu().pin_memory() for t in dev_in]
        h2d = sum(t.numel() * t.element_size() for t in host_in)
        hl = torch.zeros(1, dtype=torch.float64).pin_memory()
        step(False, (dev_in, host_in))
        torch.cuda.synchronize()
        barrier(world)
        s2, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s2.record(stream)
        for _ in range(args.steps):
            loss = step(False, (dev_in, host_in))
            hl.copy_(loss.detach().reshape(1), non_blocking=True)
        e2.record(stream)
        torch.cuda.synchronize()
        et = max_over_ranks(s2.elapsed_time(e2) / 1e3, world)
        e2e = {"value": total_nnz / et, "unit": unit, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": 8}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, dt, S = cpu_oracle_grad_rate(T, args.cpu_sample)
        cpu = {"value": rate, "unit": unit, "cores": 1, "kind": "oracle",
               "sample": f"first {S} nonzeros, refresh + loss + gradient ({dt:.1f} s)"}
    if rank == 0:
        line = {
            "metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_max / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "c_storage": args.prec,
            "config": {
                "workload": spec.name, "nnz": nnz, "J": J, "R": R,
                "parallelism": "replicas only" if world > 1 else "single GPU",
                "schedule": "SampledLoss forward (refresh C, fused loss + dL/dC) and backward "
                            "(dL/dA, dL/dB) over every nonzero",
                "l2": "inputs larger than L2 (COO 400 MB)", "generation_s": round(gen_s, 2),
                "loss": loss_v,
                "per_step_ms": {"forward": f_ms, "backward": b_ms},
                "algorithmic_bytes_per_nnz": {"forward": fwd_bytes},
                "l2_served_bytes_per_step": fwd_bytes * nnz - dram_bytes,
            },
            "roofline": {"bound": "hbm", "kernel": "forward (loss + dL/dC scatter)",
                         "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "traffic": None, "peak_source": peak_kind,
                         "bytes": "DRAM-compulsory: COO stream + one read of C + one write "
                                  "of dL/dC per forward; the gathered rows and red.add rows "
                                  "are L2-served"},
            "clocks": clk.summary(),
            "gpu_launches": launches,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- main


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    from paper_2210_06014_gb300 import synth

    lr = args.lr
    if args.workload == "order8":
        spec = synth.spec_order(8, 10_000, args.nnz if args.nnz != 100_000_000 else 50_000_000, 32)
        spec.test_fraction = 0.1
        # the products of 7 cached rows are heavy-tailed (max |v|^2 ~ 3e4 per 2M
        # nonzeros at this init); per-element SGD needs lr |v|^2 < 2
        lr = lr or 1e-5
    elif args.workload == "batch":
        spec = None
        lr = lr or 0.01
    elif args.workload == "sparsity":
        return run_sparsity(args, world, rank, lr or 0.01)
    elif args.workload == "autograd":
        spec = synth.spec_order(4, 100_000, args.nnz if args.nnz != 100_000_000 else 20_000_000, 32)
        spec.test_fraction = 0.0
    else:
        spec = synth.spec_ratings(nnz=args.nnz)
        lr = lr or 0.01
    if args.workload == "batch":
        return run_batch(args, world, rank, lr)
    workload = spec.name
    N, J, R = spec.order, spec.J[0], spec.R
    metric = "SGD nonzeros/s (factor+core updates)"
    if args.workload == "autograd":
        metric = "loss forward+backward nonzeros/s"
    unit = "nnz/s"

    if args.impl == "reference":
        if rank != 0:
            return
        t0 = time.perf_counter()
        T = synth.make_tensor(spec, device="cuda" if torch.cuda.is_available() else "cpu")
        gen_s = time.perf_counter() - t0
        steps = []
        for i in range(args.warmup + args.steps):
            if args.workload == "autograd":
                rate, dt, S = cpu_oracle_grad_rate(T, max(10_000, args.cpu_sample // 4))
            else:
                rate, dt, S = cpu_oracle_epoch_rate(T, max(10_000, args.cpu_sample // 4),
                                                    args.order)
            if i >= args.warmup:
                steps.append((rate, dt))
        rate = statistics.median(r for r, _ in steps)
        ms = statistics.median(d for _, d in steps) * 1e3
        line = {"impl": "reference", "metric": metric, "value": rate, "unit": unit, "n_gpus": 1,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": workload, "sample_nnz": S, "generation_s": gen_s},
                "cpu_baseline": {"value": rate, "unit": unit, "cores": 1, "kind": "oracle",
                                 "sample": f"first {S} training nonzeros, " + (
                                     "loss and gradient" if args.workload == "autograd"
                                     else "one epoch")},
                "e2e": {"value": rate, "unit": unit, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    from paper_2210_06014_gb300 import sft
    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = time.perf_counter()
    T = synth.make_tensor(spec, device=dev)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    if args.workload == "autograd":
        return run_autograd(args, world, rank, sft, T, spec, metric, unit, gen_s)
    line = run_sgd(args, world, rank, sft, T, spec, metric, unit, gen_s, lr)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_sgd(args, world, rank, sft, T, spec, metric, unit, gen_s, lr, print_line=True,
            extras=True):
    """One step = one epoch of Algorithm 2 on tensor T (factor pass + refresh per
    mode, then core pass + refresh per mode, then the test-set residual sums).
    Returns the JSON line (rank 0)."""
    from paper_2210_06014_gb300 import synth
    dev = T.val.device
    workload = spec.name
    N, J, R = spec.order, spec.J[0], spec.R
    if not extras:
        args = argparse.Namespace(**{**vars(args), "no_e2e": True, "no_cpu_baseline": True})
    idx, val = T.idx, T.val
    tidx, tval = T.test_idx, T.test_val
    nnz, ntest = T.nnz, int(tval.numel())
    core_batch = args.core_batch if args.core_batch > 0 else nnz
    stream = torch.cuda.current_stream()
    prec = sft.SFT_BF16 if args.prec == "bf16" else sft.SFT_FP32
    dec = sft.Decomposition(T.A0, T.B0, deterministic=False, max_batch=4096, prec=prec)
    loss_out = torch.zeros(2, dtype=torch.float64, device=dev)
    slices = []
    layout_s = 0.0
    rows_per_nnz = 1.0
    if args.path == "slices":
        dec.set_slice_tiling(args.slice_tile, args.slice_max_direct)
        if args.long_slices == "subslices":
            dec.set_long_slices(sft.SFT_LONG_SUBSLICES)
        dec.set_blocked_chains(args.blocked_chains == "on")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        orders = ([synth.csf_order(idx, n) for n in range(N)] if args.order == "csf"
                  else [None] * N)
        slices = [dec.slices(n, idx, val, orders[n]) for n in range(N)]
        del orders
        torch.cuda.synchronize()
        layout_s = time.perf_counter() - t0
        for sl in slices:
            sl._scratch = None  # sort keys are no longer needed
        touched = [int((sl.row_ptr[1:] > sl.row_ptr[:-1]).sum()) for sl in slices]
        rows_per_nnz = sum(touched) / (N * nnz)
        if args.fibers != "off":
            t0 = time.perf_counter()
            for sl in slices:
                try:
                    nf = sl.build_fibers(dec)
                except sft.SftError:  # fiber key does not fit 64 bits
                    continue
                if args.fibers == "auto" and nf > nnz // 2:
                    sl.drop_fibers()
            torch.cuda.synchronize()
            layout_s += time.perf_counter() - t0
    chain_limits = []
    if slices and args.slice_max_direct == 0 and args.slice_tile == 0:
        # per-mode choice of the longest slice run whole (setup, untimed; A restored)
        t0 = time.perf_counter()
        chain_limits = [dec.autotune_slices(sl, lr=lr, lam=0.01) for sl in slices]
        torch.cuda.synchronize()
        tune_s = time.perf_counter() - t0
    fibers = [{"mode": n, "fibers": sl.nfibers if sl.fid is not None else None,
               "used": sl.fid is not None, "core": sl.P is not None}
              for n, sl in enumerate(slices)]

    ev = {}

    def ev_pair(key):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        ev.setdefault(key, []).append((a, b))
        return a, b

    resident = {"slices": slices, "idx": idx, "val": val, "tidx": tidx, "tval": tval,
                "ready": None}

    def step(timed: bool, inp=resident, d=None, lout=None):
        """One epoch over the inputs `inp` on decomposition d (default: dec).
        inp["ready"]: None, or per mode and for the test set a list of events
        recorded after that input's host-to-device copies; the step waits on
        them before it first reads that input."""
        d = d or dec
        lout = loss_out if lout is None else lout
        ready = inp["ready"]
        sls = inp["slices"]
        def wait_ready(i):
            if ready is not None:
                for e in ready[i]:
                    stream.wait_event(e)

        for n in range(N):
            wait_ready(n)
            if inp.get("expand_rows"):
                sl = sls[n]
                sft.sft_slices_expand_rows(d.ctx, n, sl.row_ptr, sl.nnz, sl.idx[n])
                if sl.fid is not None:
                    sft.sft_fibers_expand_coords(d.ctx, n, sl.fid, sl.nnz, sl.fcoord, sl.nfibers,
                                                 sl.idx)
            if timed:
                a, b = ev_pair("factor")
                a.record(stream)
            if sls:
                d.update_factors_slices(sls[n], lr=lr, lam=0.01)
            else:
                d.update_factors(n, inp["idx"], inp["val"], None, batch=4096, lr=lr, lam=0.01)
            if timed:
                b.record(stream)
                a, b = ev_pair("refresh")
                a.record(stream)
            d.refresh(n)
            if timed:
                b.record(stream)
        for n in range(N):
            if timed:
                a, b = ev_pair("core")
                a.record(stream)
            if sls:
                d.update_core_slices(sls[n], batch=core_batch, lr=lr, lam=0.01)
            else:
                d.update_core(n, inp["idx"], inp["val"], None, batch=core_batch, lr=lr,
                                lam=0.01)
            if timed:
                b.record(stream)
                a, b = ev_pair("refresh")
                a.record(stream)
            d.refresh(n)
            if timed:
                b.record(stream)
        wait_ready(N)
        if timed:
            a, b = ev_pair("loss")
            a.record(stream)
        sft.sft_loss_async(d.ctx, inp["tidx"], inp["tval"], ntest, lout)
        if timed:
            b.record(stream)

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    launches0 = dec.launches
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed epochs
        start.record(stream)
        for _ in range(args.steps):
            step(True)
        end.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    barrier(world)
    launches = dec.launches - launches0
    dec.sync(600_000)
    elapsed = start.elapsed_time(end) / 1e3
    elapsed_max = max_over_ranks(elapsed, world)
    total_nnz = sum_over_ranks(float(nnz * args.steps), world)
    value = replica_rate(nnz * args.steps, elapsed, world)
    ms_per_step = elapsed_max / args.steps * 1e3

    def avg_ms(key, per_step):
        xs = [a.elapsed_time(b) for a, b in ev[key]]
        return sum(xs) / len(xs), sum(xs) / args.steps

    f_ms, f_step = avg_ms("factor", N)
    f_mode = [sum(a.elapsed_time(b) for a, b in ev["factor"][k::N]) / args.steps
              for k in range(N)]
    c_mode = [sum(a.elapsed_time(b) for a, b in ev["core"][k::N]) / args.steps
              for k in range(N)]
    c_ms, c_step = avg_ms("core", N)
    r_ms, r_step = avg_ms("refresh", 2 * N)
    l_ms, l_step = avg_ms("loss", 1)
    c_bytes = 2 if args.prec == "bf16" else 4
    fac_bytes, core_bytes = algorithmic_bytes(N, J, R, args.path, rows_per_nnz, c_bytes)
    # factor bytes of one epoch, mode by mode: a mode with fibers reads its
    # fiber id and v (J floats) per nonzero instead of the N-1 cached rows, and
    # first forms v per fiber (N-1 coordinates and rows in, J floats out)
    fac_epoch = core_epoch = 0.0
    for fb in fibers or [{"used": False}] * N:
        gathers = 4 * (N - 1) + (N - 1) * R * c_bytes  # other coordinates + cached rows
        if fb["used"]:
            nf = fb["fibers"]
            # per nonzero: fiber id and v (J) / p (R) instead of the cached rows;
            # per fiber: its coordinates and rows in, v or p out
            fac_epoch += nnz * (fac_bytes - gathers + 4 + J * 4) + nf * (4 + gathers + J * 4)
            if fb["core"]:
                core_epoch += nnz * (core_bytes - gathers + 4 + R * 4) + nf * (4 + gathers + R * 4)
            else:
                core_epoch += nnz * core_bytes
        else:
            fac_epoch += nnz * fac_bytes
            core_epoch += nnz * core_bytes
    peak, peak_kind = peaks()
    kernels = {
        "factor": (f_ms, fac_epoch / N / (f_ms / 1e3) / 1e9),
        "core": (c_ms, core_epoch / N / (c_ms / 1e3) / 1e9),
    }
    dom = "factor" if f_step >= c_step else "core"
    ach = kernels[dom][1]
    sse, sae = loss_out.tolist()
    test_rmse = (sse / ntest) ** 0.5 if ntest else None

    # end to end through the public API from pinned host buffers: every step's
    # inputs (what the step's passes read of each slice layout, or the COO set,
    # and the test set) are copied from pinned host memory inside the timed
    # region and the loss is read back.  Two device copies of the inputs
    # alternate: step k+1's copies run on a copy stream while step k computes,
    # each mode's pass waits only for its own layout, and a copy into a buffer
    # set starts only after the step that last read it (k-1) has finished.
    e2e = None
    if not args.no_e2e:
        def groups_of(inp):
            return e2e_groups(inp, N)

        sets = [dict(resident), e2e_clone_set(resident)]
        for st_ in sets:
            st_["expand_rows"] = bool(st_["slices"])
        host = [[t.cpu().pin_memory() for t in g] for g in groups_of(sets[0])]
        h2d = sum(t.numel() * t.element_size() for g in host for t in g)
        hloss = torch.zeros(2, dtype=torch.float64).pin_memory()
        # one copy stream: a second one gains no bandwidth on the host link,
        # and with one the sets arrive strictly in step order (step k+1's
        # copies never compete with step k's); a group is ready at its event
        copy_stream = torch.cuda.Stream()
        done = [torch.cuda.Event(), torch.cuda.Event()]

        # timing events of the timed run: per set, its copies on the copy
        # stream; per step, its work on the compute stream (reported as medians
        # so that a slow host link shows as such)
        spans = {"copy": [], "step": []}

        def span(kind, st):
            a = torch.cuda.Event(enable_timing=True)
            a.record(st)
            spans[kind].append(a)

        def enqueue_copies(k):
            inp = sets[k % 2]
            ready = []
            copy_stream.wait_event(done[k % 2])  # the step that last read this set
            span("copy", copy_stream)
            with torch.cuda.stream(copy_stream):
                for g_dev, g_host in zip(groups_of(inp), host):
                    for d, h in zip(g_dev, g_host):
                        d.copy_(h, non_blocking=True)
                    e = torch.cuda.Event()
                    e.record(copy_stream)
                    ready.append([e])
            span("copy", copy_stream)
            inp["ready"] = ready

        def e2e_steps(nsteps):
            copy_stream.wait_stream(stream)
            enqueue_copies(0)
            for k in range(nsteps):
                if k + 1 < nsteps:
                    enqueue_copies(k + 1)
                span("step", stream)
                step(False, sets[k % 2])
                span("step", stream)
                done[k % 2].record(stream)
                hloss.copy_(loss_out, non_blocking=True)

        for d in done:
            d.record(stream)
        e2e_steps(1)
        torch.cuda.synchronize()
        barrier(world)
        s2, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        spans["copy"].clear()
        spans["step"].clear()
        s2.record(stream)
        e2e_steps(args.steps)
        e2.record(stream)
        torch.cuda.synchronize()
        et = max_over_ranks(s2.elapsed_time(e2) / 1e3, world)

        def median_ms(evs):
            xs = [a.elapsed_time(b) for a, b in zip(evs[0::2], evs[1::2])]
            return statistics.median(xs) if xs else None

        copy_ms = median_ms(spans["copy"])
        e2e = {"value": total_nnz / et, "unit": unit, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": 16,
               "copy_ms_per_step": copy_ms,
               "h2d_gbs": h2d / copy_ms / 1e6 if copy_ms else None,
               "compute_ms_per_step": median_ms(spans["step"])}
        if slices:
            e2e["inputs"] = ("every mode's slice layout as values, row pointers, fiber ids "
                             "and fiber coordinates (its coordinate arrays are rebuilt on the "
                             "device each step: own mode from row_ptr, other modes from the "
                             "fiber table), and the test set")
            if any(sl.fid is None for sl in slices):
                e2e["inputs"] += ("; a mode without fibers ships its values, row pointers "
                                  "and other modes' coordinates instead")
        del sets[1]

    # end to end from raw COO: every step copies the raw training and test sets
    # from pinned host memory, builds the slice layout and fiber table of
    # every mode on the device (the preprocessing the headline leaves out, as
    # the paper does for B-CSF), runs the epoch and reads the loss back
    e2e_raw = None
    if slices and not args.no_e2e and not args.no_e2e_raw:
        hraw = [t.cpu().pin_memory() for t in list(idx) + [val] + list(tidx) + [tval]]
        draw = [torch.empty_like(t) for t in list(idx) + [val] + list(tidx) + [tval]]
        hloss2 = torch.zeros(2, dtype=torch.float64).pin_memory()
        use_f = [sl.fid is not None for sl in slices]
        use_p = [sl.P is not None for sl in slices]

        def raw_step():
            for dd, hh in zip(draw, hraw):
                dd.copy_(hh, non_blocking=True)
            ridx, rval = draw[:N], draw[N]
            lays = [dec.slices(n, ridx, rval,
                               synth.csf_order(ridx, n) if args.order == "csf" else None)
                    for n in range(N)]
            for n, sl in enumerate(lays):
                sl._scratch = None
                if use_f[n]:
                    sl.build_fibers(dec, core=use_p[n])
            inp = {"slices": lays, "idx": ridx, "val": rval, "tidx": draw[N + 1:2 * N + 1],
                   "tval": draw[2 * N + 1], "ready": None}
            step(False, inp)
            hloss2.copy_(loss_out, non_blocking=True)

        raw_step()
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            raw_step()
        torch.cuda.synchronize()
        rt = max_over_ranks(time.perf_counter() - t0, world)
        e2e_raw = {"value": total_nnz / rt, "unit": unit,
                   "h2d_bytes_per_step": int(sum(t.numel() * t.element_size() for t in hraw)),
                   "d2h_bytes_per_step": 16,
                   "what": "epoch plus, every step, the host-to-device copy of the raw COO "
                           "train and test sets and the device build of every mode's slice "
                           "layout and fiber table (host wall clock over the steps)"}
        del draw, hraw

    # precision block and convergence curves: the same epoch with bfloat16
    # cached products (timed like the headline, from the initial parameters),
    # and the test RMSE after each of `epochs_rmse` epochs from the same
    # initial parameters for both storages of C (untimed)
    conv = None
    if args.epochs_rmse > 0 and rank == 0 and world == 1:
        def fresh(prec_c):
            d = sft.Decomposition(T.A0, T.B0, deterministic=False, max_batch=4096, prec=prec_c)
            if slices:
                d.set_slice_tiling(args.slice_tile, args.slice_max_direct)
                if args.long_slices == "subslices":
                    d.set_long_slices(sft.SFT_LONG_SUBSLICES)
                d.set_blocked_chains(args.blocked_chains == "on")
                if chain_limits:
                    for sl in slices:
                        d.autotune_slices(sl, lr=lr, lam=0.01)
            return d

        other = sft.SFT_BF16 if prec == sft.SFT_FP32 else sft.SFT_FP32
        other_name = "bf16" if other == sft.SFT_BF16 else "fp32"
        lo = torch.zeros(2, dtype=torch.float64, device=dev)
        d_o = fresh(other)
        for _ in range(args.warmup):
            step(False, d=d_o, lout=lo)
        torch.cuda.synchronize()
        ev.clear()
        s3, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s3.record(stream)
        for _ in range(args.steps):
            step(True, d=d_o, lout=lo)
        e3.record(stream)
        torch.cuda.synchronize()
        o_elapsed = s3.elapsed_time(e3) / 1e3
        of_ms, _ = avg_ms("factor", N)
        oc_ms, _ = avg_ms("core", N)
        o_cb = 2 if other == sft.SFT_BF16 else 4
        o_fac, _ = algorithmic_bytes(N, J, R, args.path, rows_per_nnz, o_cb)
        d_o.close()
        del d_o
        curves = {}
        for name, pc in ((args.prec, prec), (other_name, other)):
            d = fresh(pc)
            ys = []
            for _ in range(args.epochs_rmse):
                step(False, d=d, lout=lo)
                sse_e, _ = lo.tolist()
                ys.append((sse_e / ntest) ** 0.5 if ntest else None)
            curves[name] = ys
            d.close()
            del d
        conv = {
            other_name: {"value": nnz * args.steps / o_elapsed, "unit": unit,
                         "ms_per_step": o_elapsed / args.steps * 1e3,
                         "per_launch_ms": {"factor": of_ms, "core": oc_ms},
                         "c_storage": other_name},
            "test_rmse_per_epoch": curves,
            "epochs": args.epochs_rmse,
            "final_rmse_ratio_bf16_over_fp32": (curves["bf16"][-1] / curves["fp32"][-1]
                                                if curves["fp32"][-1] else None),
            "speedup_bf16_over_fp32": (
                (nnz * args.steps / o_elapsed) / value if other == sft.SFT_BF16
                else value / (nnz * args.steps / o_elapsed)),
            "what": "test RMSE after each epoch from the same initial parameters "
                    "(Section 'Real-world accuracy'); the other storage of C timed like "
                    "the headline",
        }

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, dt, S = cpu_oracle_epoch_rate(T, args.cpu_sample, args.order)
        cpu = {"value": rate, "unit": unit, "cores": 1, "kind": "oracle",
               "sample": f"first {S} training nonzeros, one epoch ({dt:.1f} s)"}

    if rank == 0:
        line = {
            "metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "c_storage": args.prec,
            "config": {
                "workload": workload, "train_nnz": nnz, "test_nnz": ntest, "J": J, "R": R,
                "lr": lr, "lambda": 0.01,
                "parallelism": "replicas only" if world > 1 else "single GPU",
                "path": args.path,
                "long_slices": args.long_slices if args.path == "slices" else None,
                "blocked_chains": args.blocked_chains if args.path == "slices" else None,
                "schedule": (("factor: every mode-n slice element by element (Algorithm 4), "
                              + ("in the B-CSF traversal order (each slice sorted by the other "
                                 "modes' coordinates)" if args.order == "csf"
                                 else "in storage order"))
                             if slices else "factor: Hogwild rows (COO)")
                            + f"; core: batch {core_batch} (Algorithm 5 when = nnz); refresh "
                              "after every pass; test loss",
                "layout_build_s": round(layout_s, 3),
                "factor_rows_per_nnz": rows_per_nnz,
                "fibers": fibers,
                "chain_limit_per_mode": chain_limits,
                "l2": "inputs larger than L2 (COO 1.6 GB)", "generation_s": round(gen_s, 2),
                "test_rmse_after": test_rmse,
                "per_launch_ms": {"factor": f_ms, "core": c_ms, "refresh": r_ms, "loss": l_ms},
                "per_mode_ms": {"factor": f_mode, "core": c_mode},
                "per_step_ms": {"factor": f_step, "core": c_step, "refresh": r_step,
                                "loss": l_step},
                "algorithmic_bytes_per_nnz": {"factor": fac_epoch / (N * nnz),
                                              "core": core_epoch / (N * nnz)},
                "achieved_gbs": {k: v[1] for k, v in kernels.items()},
            },
            "roofline": {"bound": "hbm", "kernel": f"{dom} pass", "achieved": ach, "peak": peak,
                         "unit": "GB/s", "frac": ach / peak,
                         # the record covers the default configuration's kernels only
                         "traffic": (measured_traffic(f"{workload}|{args.prec}|{args.path}|{dom}")
                                     if args.long_slices == "maps" and args.order == "storage"
                                     and args.blocked_chains == "on" else None),
                         "peak_source": peak_kind},
            "clocks": clk.summary(),
            "gpu_launches": launches,
            "e2e": e2e,
            "e2e_raw": e2e_raw,
            "precision_and_convergence": conv,
            "cpu_baseline": cpu,
        }
        if print_line:
            print(json.dumps(line))
        return line
    return None


if __name__ == "__main__":
    main()
