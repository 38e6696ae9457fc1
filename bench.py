#!/usr/bin/env python3
"""Benchmark of the FIM black-oil linearisation path on GB300.

Workload: the 100x100x20 three-phase black-oil box (200 000 cells, 3x3
blocks, 1 372 000 stored blocks), seeded synthetic inputs.  One step is one
pass of the whole hot path over it:
    ocp_linearize (properties, accumulation, fluxes, wells, residual and
    block-CSR Jacobian) + 50 x ocp_bsr_spmv (the products a Krylov solve
    iterates on) + 1 x ocp_adjoint_vjp (all four gradients).
Metric: Mcell FIM linearisations/s = cells x steps / time (whole job, all
ranks).  L2 is flushed (a 512 MB write) before every step, outside the step's
CUDA events.  Multi-GPU runs are replicas: every rank runs its own copy of the
workload (weak scaling), no collective on the data path.

``--impl reference`` times the CPU oracle (the plain FP64 numpy checker) on
the host cores on a bounded sample of the same workload, in the same unit.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SPMV = 50
# FP64 peak of GB300 from its unit counts and clock: 152 SMs, 2 DFMA per SM
# per clock (2 flop each), 2.07 GHz maximum SM clock
FP64_NOMINAL_GFLOPS = 2 * 2 * 152 * 2.07


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


# Figures that only an ncu capture gives (DRAM bytes, FP64 instruction
# counts), stored with the SHA-256 (first 16 hex digits) of the sources of
# the kernels they describe; `stored()` returns them only while those files
# still hash to the recorded value, and None (reported null) after any change.
# Captures: profiles/layered_box_lin_vjp_fp64_dram.md (commands there).
#   fp64_inst_per_cell  FP64 thread instructions per cell (per row for the
#                       SpMV), summed over the kernels of the phase
#   fp64_warp_inst_per_cell  FP64 warp instructions per cell: each occupies
#                       the SM's FP64 pipe for 16 cycles whatever its lanes
#   dram_bytes          DRAM read + write bytes of one call on the
#                       100x100x20 workload
STORED = {
    "spmv": {"sources": ["spmv_adjoint.cu", "ocp_internal.cuh"], "sha16": "f3457da1c16ec428",
             "dram_bytes": 104.44e6, "fp64_inst_per_cell": 63.84, "fp64_warp_inst_per_cell": 2.0041},
    # FP64 counts: the three stage kernels' sum (the one-launch ordered kernel
    # executes 372.54 / 12.0007).  DRAM bytes per call by launch mode
    # ("ordered" of the launch shape): 0 with 128/128/256-cell tiles, 1 and 2
    # with 64-cell tiles
    "linearize": {"sources": ["linearize.cu", "ocp_internal.cuh"], "sha16": "630f544f6f1a0b3a",
                  "fp64_inst_per_cell": 370.54, "fp64_warp_inst_per_cell": 11.9382,
                  "dram_bytes": {"0": 326.81e6, "1": 204.19e6, "2": 121.56e6}},
    "vjp": {"sources": ["spmv_adjoint.cu", "ocp_internal.cuh"], "sha16": "f3457da1c16ec428",
            "fp64_inst_per_cell": 177.19, "fp64_warp_inst_per_cell": 5.5739, "dram_bytes": 147.39e6},
}


def sources_sha16(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2406_10862_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def stored(name, key):
    rec = STORED[name]
    if rec.get("sha16") is None or sources_sha16(rec["sources"]) != rec["sha16"]:
        return None
    return rec.get(key)


def spmv_traffic():
    return stored("spmv", "dram_bytes")


def lin_fp64_per_cell():
    return stored("linearize", "fp64_inst_per_cell")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None
        self.window = None

    def mark(self, t0, t1):
        """Wall-clock window (time.time()) of the timed region."""
        self.window = (t0, t1)

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        import datetime
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 10:
                    continue
                try:
                    ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    rows.append((ts, float(f[2]), float(f[3]), [n for n, v in zip(names, f[6:10])
                                                                 if v.lower() == "active"]))
                except ValueError:
                    continue
        os.unlink(self.path)
        inside = rows
        if self.window is not None:
            inside = [r for r in rows if self.window[0] - 0.05 <= r[0] <= self.window[1] + 0.05] or rows
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "samples": len(inside), "reasons": sorted(set(n for r in inside for n in r[3]))}


# --------------------------------------------------------------------- CPU side
def sub_box(g, s, sx, sy, sz):
    """The corner sub-box [0,sx) x [0,sy) x [0,sz) of the workload as a grid of
    its own (same rock, fluid, states and the perforations inside it)."""
    import numpy as np

    from paper_2406_10862_gb300 import workloads as W
    kk, jj, ii = np.meshgrid(np.arange(sz), np.arange(sy), np.arange(sx), indexing="ij")
    cells = (ii + g.nx * (jj + g.ny * kk)).ravel()
    local = {int(c): n for n, c in enumerate(cells)}
    h = W.GridDesc(**{f: getattr(g, f) for f in g.__dataclass_fields__})
    h.nx, h.ny, h.nz = sx, sy, sz
    h.lnk, h.phi = g.lnk[cells], g.phi[cells]
    h.wells = []
    for w in g.wells:
        inside = [local[int(c)] for c in w.cells if int(c) in local]
        if inside:
            h.wells.append(W.Well(kind=w.kind, phase=w.phase, p_bh=w.p_bh, rw=w.rw, skin=w.skin,
                                  cells=np.array(inside, dtype=np.int64)))
    st = W.State(u_new=s.u_new[:, cells], flag_new=s.flag_new[cells], u_old=s.u_old[:, cells],
                 flag_old=s.flag_old[cells], dt=s.dt)
    return h, st


def oracle_sample_step(g, s, sx=20, sy=20, sz=5, seed=9):
    """Times one whole step of the CPU oracle on a bounded sample of the
    workload: the corner sub-box [0,sx) x [0,sy) x [0,sz) (it holds the
    producer column at (4, 4)) linearised once, 50 SpMVs over all of its rows
    (five seeded vectors in turn, as in the GPU step) and one adjoint pass.
    Everything reported is timed; nothing is extrapolated.  Returns (seconds,
    cells of the sample, description)."""
    import numpy as np

    from oracle.linearize import linearize
    from oracle.spmv import bsr_spmv

    h, st = sub_box(g, s, sx, sy, sz)
    nsub = h.N
    rng = np.random.default_rng(seed)
    xs = [rng.normal(size=nsub * 3) for _ in range(5)]
    lam = rng.normal(size=(nsub, 3))
    t0 = time.perf_counter()
    o = linearize(h, st.u_new, st.flag_new, st.u_old, st.flag_old, st.dt)
    for k in range(N_SPMV):
        bsr_spmv(o["row_ptr"], o["col_idx"], o["val"], xs[k % 5])
    linearize(h, st.u_new, st.flag_new, st.u_old, st.flag_old, st.dt, mode="all", lam=lam)
    sec = time.perf_counter() - t0
    desc = ("oracle (numpy, 1 thread) on the %dx%dx%d corner sub-box of the workload (%d cells), one whole "
            "step: one linearisation and one adjoint pass (vectorised numpy with dual numbers) and 50 SpMVs "
            "over all of its rows (the oracle's per-row Python loop, most of the time)" % (sx, sy, sz, nsub))
    return sec, nsub, desc


def _oracle_slab_task(task):
    """One process of the all-cores oracle baseline: the oracle linearisation
    of one slab of the workload (its owned layers plus ghost layers).
    Returns (owned cells, seconds)."""
    rank, world = task
    os.environ["OMP_NUM_THREADS"] = "1"
    from oracle.linearize import linearize
    from paper_2406_10862_gb300 import partition as P
    from paper_2406_10862_gb300 import workloads as W
    g, s = W.layered_box()
    slab = P.slab_of(g.nz, g.nx * g.ny, rank, world)
    if slab.k1 <= slab.k0:
        return 0, 0.0
    h = P.subgrid(g, slab)
    cells = slab.global_cells
    t0 = time.perf_counter()
    linearize(h, s.u_new[:, cells], s.flag_new[cells], s.u_old[:, cells], s.flag_old[cells], s.dt)
    return (slab.k1 - slab.k0) * slab.nxy, time.perf_counter() - t0


def oracle_all_cores():
    """The oracle's linearisation of the whole 200 000-cell workload on every
    host core: the box split into one slab per core (with ghost layers), one
    spawned process per slab, timed from the start of the first to the end of
    the last after the processes have started."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    world = min(cores, 20)                      # at least one layer per slab
    ctx = mp.get_context("spawn")
    with ctx.Pool(world) as pool:
        pool.map(_oracle_slab_task, [(0, 20)] * world)     # warm-up: start-up and imports
        t0 = time.perf_counter()
        res = pool.map(_oracle_slab_task, [(r, world) for r in range(world)])
        wall = time.perf_counter() - t0
    owned = sum(n for n, _ in res)
    return {"value": owned / wall / 1e6, "unit": "Mcell linearisations/s", "cores": world, "kind": "oracle",
            "sample": "oracle linearisation (numpy) of the whole 100x100x20 workload split into %d slabs with "
                      "ghost layers, one spawned process per slab; wall %.1f s" % (world, wall)}


def host_info():
    import platform
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"machine": platform.machine(), "cpus": os.cpu_count(), "model": model}


def run_reference(args, rank, world):
    """The CPU oracle as the reference arm: every step is a bounded sample."""
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from paper_2406_10862_gb300 import workloads as W
    g, s = W.layered_box()
    per = []
    desc = ""
    # the sample shrinks with the number of steps so the run stays within minutes
    n = args.warmup + args.steps
    sx, sy, sz = (20, 20, 5) if n <= 30 else (10, 10, 5)
    nsub = sx * sy * sz
    for k in range(n):
        sec, nsub, desc = oracle_sample_step(g, s, sx, sy, sz, seed=k)
        if k >= args.warmup:
            per.append(sec)
    ms_step = 1e3 * statistics.mean(per)
    value = nsub / (ms_step * 1e-3) / 1e6
    line = {
        "impl": "reference", "metric": "Mcell FIM linearisations/s (FP64 residual+BSR Jacobian), % HBM roofline",
        "value": value, "unit": "Mcell/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "%dx%dx%d corner sub-box (%d cells) of the layered black-oil box 100x100x20 "
                               "(3x3 BSR); the rate per cell is the one quoted for the 200000-cell box"
                               % (sx, sy, sz, nsub),
                   "step": "linearize + 50 SpMV + adjoint VJP of the sub-box, all timed", "global_batch": 1,
                   "parallelism": "cpu"},
        "cpu_baseline": {"value": value, "unit": "Mcell/s", "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "Mcell/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- GPU side
def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2406_10862_gb300 import build as B
    from paper_2406_10862_gb300 import ocp, workloads as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    B.build()
    ocp.load()
    if args.box:
        nx, ny, nz = (int(a) for a in args.box.lower().split("x"))
        g, s = W.layered_box(nx=nx, ny=ny, nz=nz)
    else:
        g, s = W.layered_box()
    grid = ocp.Grid(g, local_rank)
    N, nb, nnzb = grid.N, grid.nb, grid.nnzb
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    un, fn, uo, fo = T(s.u_new.ravel()), T(s.flag_new), T(s.u_old.ravel()), T(s.flag_old)
    r = torch.empty(nb * N, dtype=torch.float64, device=dev)
    v = torch.empty(nnzb * nb * nb, dtype=torch.float64, device=dev)
    ff = torch.empty(3 * nb * N, dtype=torch.float64, device=dev)
    rng = np.random.default_rng(11)
    xs = [T(rng.normal(size=nb * N)) for _ in range(5)]
    y = torch.empty(nb * N, dtype=torch.float64, device=dev)
    lam = T(rng.normal(size=nb * N))
    gout = {k: torch.empty(n, dtype=torch.float64, device=dev)
            for k, n in (("unew", nb * N), ("uold", nb * N), ("lnk", N), ("phi", N))}
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size if hasattr(
        torch.cuda.get_device_properties(dev), "L2_cache_size") else 132 * 2 ** 20
    flush = torch.empty(max(4 * l2, 512 * 2 ** 20) // 8, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    # launch shape of the linearisation: given, or autotuned (ocp_batch_tune
    # on a batch of this one grid, cached in _build/launch_shapes.json), or
    # the grid's default
    shape_src = "default"
    if args.shape:
        grid.set_shape(json.loads(args.shape))
        shape_src = "--shape"
    elif not args.no_tune and not args.profile:
        from paper_2406_10862_gb300 import autotune
        one = ocp.Batch([grid])
        one.set_io([dict(u_new=un, flag_new=fn, u_old=uo, flag_old=fo, residual=r, bsr_val=v, face_flux=ff)])
        tuned, cached = autotune.tuned_shape(one, s.dt)
        one.close()
        grid.set_shape(tuned)
        shape_src = "autotuned (cached)" if cached else "autotuned"
    lin_shape = grid.get_shape()

    def lin():
        grid.linearize(un, fn, uo, fo, s.dt, r, v, ff)

    def spmvs():
        for k in range(N_SPMV):
            grid.spmv(v, xs[k % 5], 1.0, 0.0, y)

    def vjp():
        grid.adjoint_vjp(un, fn, uo, fo, s.dt, v, ff, lam, out=gout)

    phases = [lin, spmvs, vjp]
    if not args.no_graph:
        # each phase captured once as a CUDA graph and replayed: the same
        # kernels on the same buffers, without the Python binding's per-call
        # launch overhead between them
        for f in phases:
            f()
        torch.cuda.synchronize(dev)
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        graphs = []
        with torch.cuda.stream(side):
            for f in phases:
                gr = torch.cuda.CUDAGraph()
                with torch.cuda.graph(gr, stream=side):
                    f()
                graphs.append(gr)
        stream.wait_stream(side)
        torch.cuda.synchronize(dev)
        phases = [gr.replay for gr in graphs]

    def step(ev=None):
        for i, f in enumerate(phases):
            if ev is not None:
                ev[i].record(stream)
            f()
        if ev is not None:
            ev[3].record(stream)

    # attainable FP64 rate, measured now (not under --profile, whose launch list is the workload's)
    fp64_peak = None if args.profile else ocp.probe_fp64(local_rank, reps=3)
    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize(dev)
    if grid.status() != 0:
        raise RuntimeError("device status not OK after warm-up")

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local_rank) as clk:
        time.sleep(0.3)
        w0 = time.time()
        t0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            step(evs[k])
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        clk.mark(w0, time.time())
        time.sleep(0.1)
    if world > 1:
        dist.barrier()
    st = grid.status()
    if args.profile:
        if rank == 0:
            print(json.dumps({"profile_run": True, "steps": args.steps, "device_status": st}))
        return
    lin = [e[0].elapsed_time(e[1]) for e in evs]
    spm = [e[1].elapsed_time(e[2]) / N_SPMV for e in evs]
    vjp = [e[2].elapsed_time(e[3]) for e in evs]
    ms_step = statistics.mean(a + N_SPMV * b + c for a, b, c in zip(lin, spm, vjp))
    if world > 1:
        t = torch.tensor([ms_step], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    # the same step without the L2 flush in between (warm numbers, reported
    # beside the flushed ones; the metric is the flushed step)
    n_warm = min(args.steps, 20)
    evw = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(n_warm)]
    for k in range(n_warm):
        step(evw[k])
    torch.cuda.synchronize(dev)
    warm = {"linearize": statistics.mean(e[0].elapsed_time(e[1]) for e in evw),
            "spmv_each": statistics.mean(e[1].elapsed_time(e[2]) / N_SPMV for e in evw),
            "vjp": statistics.mean(e[2].elapsed_time(e[3]) for e in evw), "steps": n_warm}

    # ---- end to end through the public API, host buffers, copies inside.
    # Serial: every step copies its inputs in, runs the API calls and copies
    # its results out, with a synchronise on both sides.  Pipelined (the
    # reported e2e): two sets of device buffers; step k+1's inputs are copied
    # in on one copy stream and step k's residual, product and gradient are
    # copied out on another while step k computes, its three phases replayed
    # as CUDA graphs captured from the same API calls.  Each step still moves
    # all of its bytes; the step's working set (Jacobian 98.8 MB, scratch
    # 160 MB) is larger than L2, so no flush is inserted.
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a)).pin_memory()
    h_un, h_fn, h_uo, h_fo = pin(s.u_new.ravel()), pin(s.flag_new), pin(s.u_old.ravel()), pin(s.flag_old)
    h_r = [torch.empty(nb * N, dtype=torch.float64).pin_memory() for _ in range(2)]
    h_y = [torch.empty(nb * N, dtype=torch.float64).pin_memory() for _ in range(2)]
    h_g = [torch.empty(N, dtype=torch.float64).pin_memory() for _ in range(2)]
    d_in = [tuple(torch.empty_like(a) for a in (un, fn, uo, fo)) for _ in range(2)]
    d_r = [torch.empty_like(r) for _ in range(2)]
    d_y = [torch.empty_like(y) for _ in range(2)]
    d_g = [{k: torch.empty_like(a) for k, a in gout.items()} for _ in range(2)]
    h2d = sum(t.numel() * t.element_size() for t in (h_un, h_fn, h_uo, h_fo))
    d2h = sum(t[0].numel() * t[0].element_size() for t in (h_r, h_y, h_g))

    def copy_in(b):
        for d, h in zip(d_in[b], (h_un, h_fn, h_uo, h_fo)):
            d.copy_(h, non_blocking=True)

    def e2e_phases(b):
        a, f, o, fo_ = d_in[b]
        return [lambda: grid.linearize(a, f, o, fo_, s.dt, d_r[b], v, ff),
                lambda: [grid.spmv(v, xs[k % 5], 1.0, 0.0, d_y[b]) for k in range(N_SPMV)],
                lambda: grid.adjoint_vjp(a, f, o, fo_, s.dt, v, ff, lam, out=d_g[b])]

    def e2e_serial_step():
        copy_in(0)
        for f in e2e_phases(0):
            f()
        h_r[0].copy_(d_r[0], non_blocking=True)
        h_y[0].copy_(d_y[0], non_blocking=True)
        h_g[0].copy_(d_g[0]["lnk"], non_blocking=True)

    for _ in range(2):
        e2e_serial_step()
    torch.cuda.synchronize(dev)
    ser_ms = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e2e_serial_step()
        torch.cuda.synchronize(dev)
        ser_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_serial_ms = statistics.mean(ser_ms)

    h2d_s, d2h_s = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    if args.no_graph:
        e2e_run = [e2e_phases(b) for b in range(2)]
    else:
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        e2e_graphs = []
        with torch.cuda.stream(side):
            for b in range(2):
                gs = []
                for f in e2e_phases(b):
                    gr = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(gr, stream=side):
                        f()
                    gs.append(gr)
                e2e_graphs.append(gs)
        stream.wait_stream(side)
        e2e_run = [[gr.replay for gr in gs] for gs in e2e_graphs]
    ev = {n: [torch.cuda.Event() for _ in range(2)] for n in ("in", "lin", "spmv", "done", "out")}
    used = [False, False]

    def e2e_step(k):
        b = k % 2
        if used[b]:                      # step k-2 has finished with buffer set b
            h2d_s.wait_event(ev["done"][b])
            stream.wait_event(ev["out"][b])
        with torch.cuda.stream(h2d_s):
            copy_in(b)
            ev["in"][b].record(h2d_s)
        stream.wait_event(ev["in"][b])
        lin_f, spmv_f, vjp_f = e2e_run[b]
        lin_f()
        ev["lin"][b].record(stream)
        spmv_f()
        ev["spmv"][b].record(stream)
        vjp_f()
        ev["done"][b].record(stream)
        with torch.cuda.stream(d2h_s):
            d2h_s.wait_event(ev["lin"][b])
            h_r[b].copy_(d_r[b], non_blocking=True)
            d2h_s.wait_event(ev["spmv"][b])
            h_y[b].copy_(d_y[b], non_blocking=True)
            d2h_s.wait_event(ev["done"][b])
            h_g[b].copy_(d_g[b]["lnk"], non_blocking=True)
            ev["out"][b].record(d2h_s)
        used[b] = True

    for k in range(4):
        e2e_step(k)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for k in range(args.steps):
        e2e_step(k)
    torch.cuda.synchronize(dev)
    e2e_step_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    e2e_ok = all(torch.equal(h_r[b], h_r[0]) and torch.equal(h_g[b], h_g[0]) for b in range(2))
    if world > 1:
        t = torch.tensor([e2e_step_ms, e2e_serial_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_step_ms, e2e_serial_ms = (float(a) for a in t.tolist())

    if rank == 0:
        spmv_ms = statistics.mean(spm)
        flops = 2.0 * nb * nb * nnzb                               # algorithmic FP64 flops per SpMV
        hbm_bytes = 8.0 * nb * nb * nnzb + 4.0 * nnzb + 4.0 * (N + 1) + 8.0 * nb * N * 2
        achieved = flops / (spmv_ms * 1e-3) / 1e9
        pk = peaks()
        hbm_peak = pk.get("hbm_gbs")
        line = {
            "metric": "Mcell FIM linearisations/s (FP64 residual+BSR Jacobian), % HBM roofline",
            "value": world * N / (ms_step * 1e-3) / 1e6, "unit": "Mcell/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "layered black-oil box 100x100x20 (200000 cells, 3x3 BSR, 1372000 blocks)",
                       "step": "linearize + 50 SpMV + adjoint VJP", "global_batch": world,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "flushed before every step (512 MB write outside the step events)",
                       "launch": "per-call launches" if args.no_graph else
                                 "each phase (linearise, 50 SpMV, adjoint) replayed as a CUDA graph"},
            "phases_ms": {"linearize": statistics.mean(lin), "spmv_each": spmv_ms, "vjp": statistics.mean(vjp),
                          "wall_timed_region_ms": wall * 1e3},
            "phases_ms_warm_l2": warm,
            "roofline": {"kernel": "spmv_grid_kernel<3>", "bound": "alu", "achieved": achieved,
                         "peak": FP64_NOMINAL_GFLOPS, "unit": "GFLOP/s", "frac": achieved / FP64_NOMINAL_GFLOPS,
                         "peak_source": "FP64 units x clock: 152 SMs x 2 DFMA/clock x 2 flop x 2.07 GHz",
                         "peak_measured": fp64_peak, "frac_of_measured": achieved / fp64_peak,
                         "peak_measured_source": "FP64 FMA rate measured in this run by ocp_probe_fp64",
                         "traffic": spmv_traffic(),
                         "hbm": {"algorithmic_bytes": hbm_bytes,
                                 "achieved_gbs": hbm_bytes / (spmv_ms * 1e-3) / 1e9,
                                 "peak_gbs": hbm_peak,
                                 "frac": (hbm_bytes / (spmv_ms * 1e-3) / 1e9 / hbm_peak) if hbm_peak else None}},
            "e2e": {"value": world * N / (e2e_step_ms * 1e-3) / 1e6, "unit": "Mcell/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_step_ms,
                    "mode": "pipelined two deep: step k+1's inputs copied in and step k's residual, product and "
                            "gradient copied out on two copy streams while step k computes (its phases replayed "
                            "as CUDA graphs of the same API calls); wall clock over all steps; the Jacobian "
                            "(98.8 MB) stays on the device, where the SpMVs consume it",
                    "l2": "no flush: each step's working set (Jacobian 98.8 MB + 160 MB scratch) exceeds L2",
                    "results_consistent": e2e_ok,
                    "serial": {"value": world * N / (e2e_serial_ms * 1e-3) / 1e6, "ms_per_step": e2e_serial_ms,
                               "mode": "copy in, per-call API launches, copy out, synchronise; L2 flushed "
                                       "before every step"}},
            "linearize": lin_line(N, nnzb, statistics.mean(lin), lin_shape, shape_src, hbm_peak),
            "vjp": vjp_line(N, nnzb, statistics.mean(vjp), hbm_peak),
            "gpu_launches": args.steps * ((3 if lin_shape["ordered"] == 0 else 2 if lin_shape["ordered"] == 1 else 1)
                                          + N_SPMV + 1),
            "clocks": clk.summary(),
            "device_status": st,
        }
        # the side measurements are single-GPU figures: taken at N = 1 only, so
        # that a multi-GPU run does not hold the other GPUs idle meanwhile
        if not args.no_ensemble and world == 1:
            line["ensemble"] = run_ensemble(dev, local_rank, reps=max(5, min(args.steps, 20)))
        if not args.no_extra and world == 1:
            line["small_case"] = run_small_case(dev, local_rank)
            line["oil_water"] = run_oil_water(dev, local_rank)
            line["adjoint"] = run_adjoint(dev, local_rank)
            line["wells"] = run_wells(dev, local_rank)
            line["pn"] = run_pn(dev, local_rank)
            line["impec"] = run_impec(dev, local_rank)
            line["coupling"] = run_coupling(dev, local_rank, with_oracle=(world == 1 and not args.no_cpu_baseline))
        if world == 1 and not args.no_cpu_baseline:
            runs = [oracle_sample_step(g, s, seed=k) for k in range(3)]
            sec = statistics.median(r[0] for r in runs)
            line["cpu_baseline"] = {"value": runs[0][1] / sec / 1e6, "unit": "Mcell/s", "cores": 1,
                                    "kind": "oracle", "sample": runs[0][2] + "; median of 3 steps"}
            line["cpu_baseline_all_cores"] = oracle_all_cores()
            line["host"] = host_info()
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# FP64 thread instructions per second of GB300's FP64 pipes: 152 SMs x 2 per
# clock x 2.07 GHz (a warp instruction occupies an SM's pipe for 16 cycles)
FP64_INST_PEAK_G = 152 * 2 * 2.07


def fp64_part(inst, warp_inst, cells, ms):
    if inst is None:
        return {"inst_per_cell": None, "note": "the kernel sources changed since the ncu count was taken"}
    rate = inst * cells / (ms * 1e-3) / 1e9
    out = {"inst_per_cell": inst, "achieved_ginst_s": rate, "peak_ginst_s": FP64_INST_PEAK_G,
           "frac": rate / FP64_INST_PEAK_G,
           "peak_source": "152 SMs x 2 FP64 lanes per clock x 2.07 GHz"}
    if warp_inst is not None:
        out["pipe_frac"] = 32 * warp_inst * cells / (ms * 1e-3) / 1e9 / FP64_INST_PEAK_G
        out["pipe_frac_meaning"] = "FP64 warp instructions x 16 pipe cycles over the SMs' cycles: the pipe's busy share"
    return out


def lin_line(N, nnzb, ms, shape, shape_src, hbm_peak):
    """The linearisation's own figures: cells per second, algorithmic bytes
    (state in and out, old state, flags, transmissibilities, porosity,
    residual, Jacobian) against the copy rate, and FP64 instructions
    against the FP64 pipe's rate (ncu counts stored with their sources)."""
    alg = 106.0 * N + 72.0 * nnzb
    by_mode = stored("linearize", "dram_bytes") or {}
    traffic = by_mode.get(str(shape["ordered"]))
    return {"mcells": N / (ms * 1e-3) / 1e6, "ms": ms, "launch_shape": shape, "shape_source": shape_src,
            "hbm": {"algorithmic_bytes": alg, "bytes_per_cell": alg / N,
                    "achieved_gbs": alg / (ms * 1e-3) / 1e9, "peak_gbs": hbm_peak,
                    "frac": alg / (ms * 1e-3) / 1e9 / hbm_peak if hbm_peak else None,
                    "traffic": traffic, "traffic_over_algorithmic": traffic / alg if traffic else None,
                    "traffic_by_launch_mode": {m: {"bytes": b, "over_algorithmic": b / alg}
                                               for m, b in sorted(by_mode.items())} or None,
                    "traffic_launch_modes": "0: three launches, 128/128/256-cell tiles; 1: cell launch + ordered "
                                            "face/assembly launch, 64-cell tiles; 2: one ordered launch, 64-cell "
                                            "tiles"},
            "fp64": fp64_part(stored("linearize", "fp64_inst_per_cell"),
                              stored("linearize", "fp64_warp_inst_per_cell"), N, ms),
            "bound": "alu"}


def vjp_line(N, nnzb, ms, hbm_peak):
    """The adjoint product's own figures, as lin_line: algorithmic bytes are
    the Jacobian, multiplier, face fluxes, ln k weights, both states, flags,
    porosity and the four gradients."""
    alg = 72.0 * nnzb + (24 + 72 + 48 + 48 + 2 + 8 + 64) * N
    traffic = stored("vjp", "dram_bytes")
    return {"mcells": N / (ms * 1e-3) / 1e6, "ms": ms,
            "hbm": {"algorithmic_bytes": alg, "bytes_per_cell": alg / N,
                    "achieved_gbs": alg / (ms * 1e-3) / 1e9, "peak_gbs": hbm_peak,
                    "frac": alg / (ms * 1e-3) / 1e9 / hbm_peak if hbm_peak else None,
                    "traffic": traffic, "traffic_over_algorithmic": traffic / alg if traffic else None},
            "fp64": fp64_part(stored("vjp", "fp64_inst_per_cell"), stored("vjp", "fp64_warp_inst_per_cell"),
                              N, ms),
            "bound": "alu"}


def run_ensemble(dev, local_rank, reps=10):
    """The 64-model ensemble (cell counts log-uniform in 2e4..4e5, ~8.1 M cells):
    one batched pass (tuned launch shape, CUDA graph) against 64 separate
    ocp_linearize calls on the same stream; both must give identical bits."""
    import numpy as np
    import torch

    from paper_2406_10862_gb300 import autotune, ocp, workloads as W

    models = W.ensemble()
    grids, ios = [], []
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    for g, s in models:
        grid = ocp.Grid(g, local_rank)
        grids.append(grid)
        ios.append(dict(u_new=T(s.u_new.ravel()), flag_new=T(s.flag_new), u_old=T(s.u_old.ravel()),
                        flag_old=T(s.flag_old),
                        residual=torch.empty(grid.nb * grid.N, dtype=torch.float64, device=dev),
                        bsr_val=torch.empty(grid.nnzb * grid.nb ** 2, dtype=torch.float64, device=dev)))
    dt = models[0][1].dt
    ncell = sum(g.N for g in grids)
    batch = ocp.Batch(grids)
    batch.set_io(ios)
    shape, cached = autotune.tuned_shape(batch, dt)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 2 ** 20 // 8, dtype=torch.float64, device=dev)

    def per_model():
        for grid, io in zip(grids, ios):
            grid.linearize(io["u_new"], io["flag_new"], io["u_old"], io["flag_old"], dt, io["residual"],
                           io["bsr_val"])

    def batched():
        batch.linearize(dt, graph=True)

    # the fairer baseline: each model's three launches captured once as its own
    # CUDA graph, the 64 graphs replayed back to back (no binding overhead)
    per_model()
    torch.cuda.synchronize(dev)
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    model_graphs = []
    with torch.cuda.stream(side):
        for grid, io in zip(grids, ios):
            gr = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gr, stream=side):
                grid.linearize(io["u_new"], io["flag_new"], io["u_old"], io["flag_old"], dt, io["residual"],
                               io["bsr_val"])
            model_graphs.append(gr)
    stream.wait_stream(side)
    torch.cuda.synchronize(dev)

    def per_model_graphs():
        for gr in model_graphs:
            gr.replay()

    def timed(fn):
        for _ in range(2):
            fn()
        ms = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    t_sep = timed(per_model)
    ref = [(io["residual"].clone(), io["bsr_val"].clone()) for io in ios]
    t_gr = timed(per_model_graphs)
    same_gr = all(torch.equal(io["residual"].view(torch.int64), r.view(torch.int64)) and
                  torch.equal(io["bsr_val"].view(torch.int64), v.view(torch.int64)) for io, (r, v) in zip(ios, ref))
    t_bat = timed(batched)
    same = all(torch.equal(io["residual"].view(torch.int64), r.view(torch.int64)) and
               torch.equal(io["bsr_val"].view(torch.int64), v.view(torch.int64)) for io, (r, v) in zip(ios, ref))
    st = batch.status()
    out = {"workload": "64 black-oil boxes, cell counts log-uniform in 2e4..4e5", "models": len(grids),
           "cells": ncell, "per_model_ms": t_sep, "per_model_graphs_ms": t_gr, "batched_graph_ms": t_bat,
           "per_model_mcells": ncell / (t_sep * 1e-3) / 1e6,
           "per_model_graphs_mcells": ncell / (t_gr * 1e-3) / 1e6,
           "batched_mcells": ncell / (t_bat * 1e-3) / 1e6,
           "speedup": t_sep / t_bat, "speedup_vs_per_model_graphs": t_gr / t_bat,
           "bitwise_equal": bool(same and same_gr), "device_status": st,
           "launch_shape": shape, "shape_from_cache": cached, "launches_per_model_path": 3 * len(grids),
           "launches_batched": 3,
           "baselines": "per_model: 64 ocp_linearize calls through the binding on one stream; per_model_graphs: "
                        "each model's three launches captured as its own CUDA graph, 64 replays back to back"}
    fp = lin_fp64_per_cell()
    if fp is not None:
        rate = ncell * fp / (t_bat * 1e-3) / 1e9
        out["fp64"] = {"inst_per_cell": fp, "achieved_ginst_s": rate, "peak_ginst_s": FP64_NOMINAL_GFLOPS / 2,
                       "frac": rate / (FP64_NOMINAL_GFLOPS / 2),
                       "source": "FP64 thread instructions per cell of the three linearisation kernels, ncu "
                                 "capture of the 100x100x10 box (same kernels as the batch)"}
    return out


def _events(stream):
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_small_case(dev, local_rank, reps=200):
    """The 10x10x3 three-phase box (300 cells): launch-latency bound, so its
    figure is microseconds per linearisation, as three stream launches and as
    one CUDA-graph replay (a one-model batch)."""
    import numpy as np
    import torch

    from paper_2406_10862_gb300 import ocp, workloads as W

    g, s = W.spe1_like()
    grid = ocp.Grid(g, local_rank)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    io = dict(u_new=T(s.u_new.ravel()), flag_new=T(s.flag_new), u_old=T(s.u_old.ravel()), flag_old=T(s.flag_old),
              residual=torch.empty(3 * grid.N, dtype=torch.float64, device=dev),
              bsr_val=torch.empty(grid.nnzb * 9, dtype=torch.float64, device=dev))
    batch = ocp.Batch([grid])
    batch.set_io([io])
    stream = torch.cuda.current_stream(dev)
    out = {"default_shape": batch.get_shape()}

    def time_us(fn):
        for _ in range(20):
            fn()
        e0, e1 = _events(stream)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) * 1e3 / reps

    out["stream_us"] = time_us(lambda: grid.linearize(io["u_new"], io["flag_new"], io["u_old"], io["flag_old"],
                                                      s.dt, io["residual"], io["bsr_val"]))
    out["graph_us_default_shape"] = time_us(lambda: batch.linearize(s.dt, graph=True))
    from paper_2406_10862_gb300 import autotune
    shape, cached = autotune.tuned_shape(batch, s.dt)
    out["tuned_shape"] = shape
    out["graph_us_tuned_shape"] = time_us(lambda: batch.linearize(s.dt, graph=True))
    # the tuner times stream launches, whose launch overhead favours fewer
    # launches; under graph replay either shape may win, so both are timed
    best = min(("default_shape", out["graph_us_default_shape"]), ("tuned_shape", out["graph_us_tuned_shape"]),
               key=lambda t: t[1])
    out["graph_us"] = best[1]
    out.update(workload="10x10x3 three-phase box (300 cells)", cells=grid.N, status=batch.status(),
               graph_us_meaning="one CUDA-graph replay of the linearisation, the faster of the default and the "
                                "autotuned launch shape (%s)" % best[0])
    return out


def run_oil_water(dev, local_rank, steps=10):
    """The 60x220x85 channelised oil-water model (1 122 000 cells, 2x2
    blocks): 10 steps of linearise + one SpMV, each step's new state the
    previous one plus a seeded perturbation."""
    import numpy as np
    import torch

    from paper_2406_10862_gb300 import ocp, workloads as W

    g, s = W.channelised_ow()
    grid = ocp.Grid(g, local_rank)
    N, nb = grid.N, grid.nb
    rng = np.random.default_rng(33)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    states = []
    u = s.u_old.copy()
    for k in range(steps + 1):
        states.append(T(u.ravel()))
        u = u.copy()
        u[0] += rng.normal(0.0, 5.0, N)
        u[1] = np.clip(u[1] + rng.uniform(0.0, 0.01, N), 0.0, 1.0)
    r = torch.empty(nb * N, dtype=torch.float64, device=dev)
    v = torch.empty(grid.nnzb * nb * nb, dtype=torch.float64, device=dev)
    x = T(rng.normal(size=nb * N))
    y = torch.empty(nb * N, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    # the linearisation's launch shape autotuned (a one-grid batch), as for the main workload
    from paper_2406_10862_gb300 import autotune
    one = ocp.Batch([grid])
    one.set_io([dict(u_new=states[1], flag_new=None, u_old=states[0], flag_old=None, residual=r, bsr_val=v,
                     face_flux=None)])
    tuned, _ = autotune.tuned_shape(one, 1.0)
    one.close()
    grid.set_shape(tuned)
    for _ in range(2):
        grid.linearize(states[1], None, states[0], None, 1.0, r, v)
        grid.spmv(v, x, 1.0, 0.0, y)
    lin, spm = [], []
    flush = torch.empty(512 * 2 ** 20 // 8, dtype=torch.float64, device=dev)
    for k in range(steps):
        flush.fill_(float(k))
        e0, e1 = _events(stream)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        grid.linearize(states[k + 1], None, states[k], None, 1.0, r, v)
        e1.record(stream)
        grid.spmv(v, x, 1.0, 0.0, y)
        e2.record(stream)
        torch.cuda.synchronize(dev)
        lin.append(e0.elapsed_time(e1))
        spm.append(e1.elapsed_time(e2))
    st = grid.status()
    ms = statistics.mean(a + b for a, b in zip(lin, spm))
    nnzb = grid.nnzb
    return {"workload": "channelised oil-water 60x220x85 (1122000 cells, 2x2 BSR)", "steps": steps,
            "launch_shape": tuned,
            "linearize_ms": statistics.mean(lin), "spmv_ms": statistics.mean(spm), "ms_per_step": ms,
            "mcells_per_s": N / (ms * 1e-3) / 1e6,
            "spmv_gflops": 2.0 * 4 * nnzb / (statistics.mean(spm) * 1e-3) / 1e9, "device_status": st}


def run_wells(dev, local_rank, reps=20):
    """One backward-Euler step of the 200 000-cell box with every well on
    surface-rate control (producers: half their oil rate at 3500 psi, limit
    1000 psi; injector: half its gas rate at 5500 psi, limit 8000 psi), the
    bottom-hole pressures as unknowns: Newton iterations of
    ocp_linearize_wells + ocp_residual_norms + ocp_bicgstab_wells +
    updates.  Also the linearisation with well rows against the plain one."""
    import numpy as np
    import torch

    from paper_2406_10862_gb300 import fim, ocp, workloads as W

    g, s = W.layered_box()
    grid = ocp.Grid(g, local_rank)
    nb, nw = grid.nb, grid.nwell
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    un, fn = T(s.u_old.ravel()), T(s.flag_old)
    q = grid.well_rates(un, fn).view(nw, nb).cpu().numpy()
    ctrl, lim, p0 = [], [], []
    for iw, w in enumerate(g.wells):
        if w.kind == 0:
            ctrl.append((1, 1, 0.5 * -q[iw, 1]))
            lim.append(1000.0)
        else:
            ctrl.append((1, nb - 1, 0.5 * q[iw, nb - 1]))
            lim.append(8000.0)
        p0.append(w.p_bh)
    st = fim.Stepper(grid)
    c = ocp.well_controls(ctrl, lim, dev)
    st.step_wells(un, fn, 1.0, T(p0), c)                       # warm-up
    c = ocp.well_controls(ctrl, lim, dev)
    st.newton_iters = st.linear_iters = 0
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    u, f, p, lins = st.step_wells(un, fn, 1.0, T(p0), c)
    torch.cuda.synchronize(dev)
    step_s = time.perf_counter() - t0
    # the converged well equations: rate targets met
    out = grid.linearize_wells(u, f, un, fn, 1.0, p, c)
    nrm = grid.residual_norms(out["residual"], 1.0, out["well_res"], c).cpu().tolist()
    # linearisation with and without the well rows, same state
    stream = torch.cuda.current_stream(dev)
    r = torch.empty(nb * grid.N, dtype=torch.float64, device=dev)
    v = torch.empty(grid.nnzb * nb * nb, dtype=torch.float64, device=dev)
    times = {}
    for name, fn_ in (("linearize_ms", lambda: grid.linearize(u, f, un, fn, 1.0, r, v)),
                      ("linearize_wells_ms", lambda: grid.linearize_wells(u, f, un, fn, 1.0, p, c, out=out))):
        for _ in range(3):
            fn_()
        e0, e1 = _events(stream)
        e0.record(stream)
        for _ in range(reps):
            fn_()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times[name] = e0.elapsed_time(e1) / reps
    res = {"workload": "layered black-oil box 100x100x20, 5 rate-controlled wells, one step of 1 day",
           "newton_iterations": st.newton_iters, "linearisations": lins, "linear_iterations": st.linear_iters,
           "step_s": step_s, "ms_per_newton_iteration": 1e3 * step_s / max(st.newton_iters, 1),
           "p_bh": p.cpu().tolist(), "controls_after": [list(x) for x in ocp.read_controls(c)],
           "final_norms": nrm, "device_status": grid.status()}
    res.update(times)
    res["well_rows_overhead_ms"] = times["linearize_wells_ms"] - times["linearize_ms"]
    return res


def run_pn(dev, local_rank, reps=20):
    """The 200 000-cell box in the paper's own unknowns, pressure and
    component amounts with the volume balance: one linearisation with the
    volume rows eliminated (3x3 blocks), the same with the full 4x4 system
    written too, and the natural-variable linearisation of the same state;
    then one backward-Euler step of 1 day by Newton in (P, N)."""
    import numpy as np
    import torch

    from paper_2406_10862_gb300 import fim, ocp, workloads as W

    g, s = W.layered_box()
    grid = ocp.Grid(g, local_rank)
    nb, N = grid.nb, grid.N
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    un, fn, uo, fo = T(s.u_new.ravel()), T(s.flag_new), T(s.u_old.ravel()), T(s.flag_old)
    pn_new, pn_old = grid.pn_from_natural(un, fn), grid.pn_from_natural(uo, fo)
    r = torch.empty(nb * N, dtype=torch.float64, device=dev)
    v = torch.empty(grid.nnzb * nb * nb, dtype=torch.float64, device=dev)
    red = grid.linearize_pn(pn_new, pn_old, 1.0)
    full = grid.linearize_pn(pn_new, pn_old, 1.0, full=True)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 2 ** 20 // 8, dtype=torch.float64, device=dev)
    times = {}
    for name, fn_ in (("natural_linearize_ms", lambda: grid.linearize(un, fn, uo, fo, 1.0, r, v)),
                      ("pn_linearize_ms", lambda: grid.linearize_pn(pn_new, pn_old, 1.0, out=red)),
                      ("pn_linearize_full_ms", lambda: grid.linearize_pn(pn_new, pn_old, 1.0, out=full, full=True))):
        for _ in range(3):
            fn_()
        tot = 0.0
        for k in range(reps):
            flush.fill_(float(k))
            e0, e1 = _events(stream)
            e0.record(stream)
            fn_()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            tot += e0.elapsed_time(e1)
        times[name] = tot / reps
    st = fim.Stepper(grid)
    st.step_pn(pn_old, 1.0)                                   # warm-up
    st.newton_iters = st.linear_iters = 0
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    pn, flag, lins = st.step_pn(pn_old, 1.0)
    torch.cuda.synchronize(dev)
    out = {"workload": "layered black-oil box 100x100x20 in (P, N_w, N_o, N_g), volume rows eliminated",
           "cells": N, "mcells_per_s_reduced": N / (times["pn_linearize_ms"] * 1e-3) / 1e6,
           "newton_iterations": st.newton_iters, "linearisations": lins, "linear_iterations": st.linear_iters,
           "step_s": time.perf_counter() - t0, "device_status": grid.status(),
           "l2": "flushed before every timed linearisation"}
    out.update(times)
    return out


def run_impec(dev, local_rank, reps=20):
    """IMPEC on the 200 000-cell box in (P, N): the pressure system
    (ocp_impec_pressure), its Jacobi BiCGSTAB solve and the explicit update,
    one step of 0.1 day from the perturbed state, timed part by part."""
    import numpy as np
    import torch

    from paper_2406_10862_gb300 import fim, ocp, workloads as W

    g, s = W.layered_box()
    grid = ocp.Grid(g, local_rank)
    N = grid.N
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    pn0 = grid.pn_from_natural(T(s.u_new.ravel()), T(s.flag_new))
    dt = 0.1
    work = grid.solver_work()
    val, rhs = grid.impec_pressure(pn0, dt)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 2 ** 20 // 8, dtype=torch.float64, device=dev)
    dp = torch.zeros(N, dtype=torch.float64, device=dev)
    pn1 = grid.empty(4 * N)
    times = {"pressure_system_ms": 0.0, "update_ms": 0.0}
    for k in range(reps + 3):
        flush.fill_(float(k))
        e0, e1 = _events(stream)
        e0.record(stream)
        grid.impec_pressure(pn0, dt, val, rhs)
        e1.record(stream)
        dp.zero_()
        grid.bicgstab_scalar(val, rhs, dp, 1e-12, 4000, work=work)
        flush.fill_(float(k))
        e2, e3 = _events(stream)
        e2.record(stream)
        grid.impec_update(pn0, dp, dt, pn1)
        e3.record(stream)
        torch.cuda.synchronize(dev)
        if k >= 3:
            times["pressure_system_ms"] += e0.elapsed_time(e1) / reps
            times["update_ms"] += e2.elapsed_time(e3) / reps
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    _, dp2, its = fim.impec_step(grid, pn0, dt, rtol=1e-12, work=work)
    torch.cuda.synchronize(dev)
    step_s = time.perf_counter() - t0
    x0, x1 = pn0.view(4, N), pn1.view(4, N)
    out = {"workload": "layered black-oil box 100x100x20 in (P, N), one IMPEC step of 0.1 day", "cells": N,
           "solve_iterations": its, "step_s": step_s, "max_dp_psi": float(dp2.abs().max()),
           "max_dN": [float((x1[e] - x0[e]).abs().max()) for e in range(1, 4)],
           "device_status": grid.status(), "l2": "flushed before each timed kernel sequence"}
    out.update(times)
    return out


def run_coupling(dev, local_rank, reps=20, with_oracle=False):
    """Adaptive subdomain coupling (Sec. 4) on the 4000x4000x1 flood (16
    million cells) split into 40x25 boxes: mark cells whose saturations moved
    by more than 5e-3, couple the boxes, label the connected components.  The
    inputs (S_w, S_g of both states and both flag arrays, 544 MB) exceed L2,
    so consecutive calls re-read them from HBM."""
    import numpy as np
    import torch

    from paper_2406_10862_gb300 import ocp, workloads as W

    g, s = W.addm_2d()
    grid = ocp.Grid(g, local_rank)
    N = grid.N
    px, py, pz = 40, 25, 1
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    un, fn, uo, fo = T(s.u_new.ravel()), T(s.flag_new), T(s.u_old.ravel()), T(s.flag_old)
    labels, work = grid.coupling_components(un, fn, uo, fo, 5e-3, px, py, pz)
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        grid.coupling_components(un, fn, uo, fo, 5e-3, px, py, pz, labels, work)
    e0, e1 = _events(stream)
    e0.record(stream)
    for _ in range(reps):
        grid.coupling_components(un, fn, uo, fo, 5e-3, px, py, pz, labels, work)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    api_ms = e0.elapsed_time(e1) / reps
    # the same call captured once in a CUDA graph: device time without the
    # Python binding's per-call overhead
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            grid.coupling_components(un, fn, uo, fo, 5e-3, px, py, pz, labels, work)
    stream.wait_stream(side)
    for _ in range(3):
        graph.replay()
    e0, e1 = _events(stream)
    e0.record(stream)
    for _ in range(reps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / reps
    S = px * py * pz
    w = work.cpu().numpy()
    lab = labels.cpu().numpy()
    _, cnt = np.unique(lab, return_counts=True)
    nbytes = N * (2 * 2 * 8 + 2)
    hbm_peak = peaks().get("hbm_gbs")
    out = {"workload": "4000x4000x1 three-phase flood, 40x25 subdomains, threshold 5e-3", "cells": N,
           "subdomains": S, "marked_cells": int(w[2 * S]), "coupled_groups": int((cnt > 1).sum()),
           "coupled_subdomains": int(cnt[cnt > 1].sum()), "union_retries": int(w[2 * S + 1]),
           "error_flag": int(w[2 * S + 2]),
           "ms_per_call": ms, "api_ms_per_call": api_ms, "gcells_per_s": N / (ms * 1e-3) / 1e9,
           "launches_per_call": 2, "timing": "CUDA-graph replay of one call; api_ms_per_call through the binding",
           "roofline": {"bound": "hbm", "algorithmic_bytes": nbytes,
                        "achieved": nbytes / (ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                        "frac": (nbytes / (ms * 1e-3) / 1e9 / hbm_peak) if hbm_peak else None,
                        "timed": "whole call (marking, coupling, components)"}}
    if with_oracle:
        from oracle.coupling import coupling_components
        t0 = time.perf_counter()
        ref, _, _ = coupling_components(g, s.u_new, s.flag_new, s.u_old, s.flag_old, 5e-3, px, py, pz)
        out["oracle_s"] = time.perf_counter() - t0
        out["labels_match_oracle"] = bool(np.array_equal(ref, lab.astype(np.int64)))
    grid.close()
    return out


def run_adjoint(dev, local_rank):
    """Gradient of the squared well-rate mismatch with respect to ln k over
    20 FIM steps on the 100x100x10 box (observed rates from the truth field),
    checkpoints every 5 steps: forward and reverse wall time, and the adjoint
    VJP kernel alone on the final state."""
    import numpy as np
    import torch

    from paper_2406_10862_gb300 import fim, ocp, workloads as W

    g, s, lnk_truth, lnk_prior, dt, nsteps = W.history_match()
    grid = ocp.Grid(g, local_rank)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    hm = fim.HistoryMatch(grid, T(s.u_old.ravel()), T(s.flag_old), dt, nsteps, checkpoint=5)
    _, _, rates = hm.run(T(lnk_truth))
    hm.q_obs = torch.stack(rates)
    hm.q_scale = hm.q_obs.abs().amax(dim=(0, 1)) + 1e-30
    # one untimed forward and backward: the first use of torch's own
    # elementwise kernels in the loss and the cotangent bookkeeping can
    # include their just-in-time compilation
    warm = T(lnk_prior).requires_grad_(True)
    fim.HistoryMatchLoss.apply(warm, hm).backward()
    lnk = T(lnk_prior).requires_grad_(True)
    hm.stepper.newton_iters = hm.stepper.linear_iters = 0
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    loss = fim.HistoryMatchLoss.apply(lnk, hm)
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    loss.backward()
    torch.cuda.synchronize(dev)
    t2 = time.perf_counter()
    # the VJP kernel alone, at the last step's state
    st = hm.stepper
    u1, f1 = T(s.u_old.ravel()).clone(), T(s.flag_old).clone()
    u2, f2 = st.step(u1, f1, dt)
    _, val, ff = st.linearize_at(u2, f2, u1, f1, dt)
    lam = T(np.random.default_rng(5).normal(size=3 * grid.N))
    out = {k: torch.empty(n, dtype=torch.float64, device=dev) for k, n in
           (("unew", 3 * grid.N), ("uold", 3 * grid.N), ("lnk", grid.N), ("phi", grid.N))}
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        grid.adjoint_vjp(u2, f2, u1, f1, dt, val, ff, lam, out=out)
    e0, e1 = _events(stream)
    e0.record(stream)
    for _ in range(20):
        grid.adjoint_vjp(u2, f2, u1, f1, dt, val, ff, lam, out=out)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    vjp_ms = e0.elapsed_time(e1) / 20
    vjp_bytes = grid.nnzb * 9 * 8 + 4 * grid.nnzb * 3 + 8 * grid.N * (3 + 9 + 6 + 6 + 1 + 8)
    return {"workload": "history match 100x100x10 (100000 cells), 20 steps of 1 day, checkpoints every 5",
            "loss": float(loss.detach()), "forward_s": t1 - t0, "gradient_s": t2 - t1,
            "newton_iterations": st.newton_iters, "linear_iterations": st.linear_iters,
            "grad_norm": float(lnk.grad.norm()), "vjp_ms": vjp_ms,
            "vjp_gbs_algorithmic": vjp_bytes / (vjp_ms * 1e-3) / 1e9, "device_status": grid.status()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the 64-model batched-ensemble measurement")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the 300-cell, oil-water and history-match measurements")
    ap.add_argument("--only", choices=["coupling", "wells", "pn", "impec", "small_case", "oil_water", "adjoint", "ensemble"],
                    help="only that side measurement, printed as one JSON line")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the step's kernels one call at a time instead of replaying per-phase CUDA graphs")
    ap.add_argument("--profile", action="store_true",
                    help="warm-up + timed steps only (no e2e, no CPU baseline): the command profiled by ncu")
    ap.add_argument("--source-hashes", action="store_true",
                    help="print the hashes of the kernel sources that the stored ncu figures are keyed to")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default launch shape of the workload's grid instead of the autotuned one")
    ap.add_argument("--shape", metavar="JSON",
                    help="launch shape of the workload's linearisation (the dict of ocp.Grid.set_shape)")
    ap.add_argument("--box", metavar="NXxNYxNZ",
                    help="with --profile: run the step on a layered box of this shape instead of 100x100x20 "
                         "(the small case of an ncu capture)")
    args = ap.parse_args()
    if args.box and not args.profile:
        ap.error("--box is only for --profile runs: the benchmark's workload is the 100x100x20 box")
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local_rank = env_int("RANK", 0), env_int("WORLD_SIZE", 1), env_int("LOCAL_RANK", 0)
    if args.source_hashes:
        print(json.dumps({k: sources_sha16(v["sources"]) for k, v in STORED.items()}))
        return
    if args.only:
        import torch
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        part = {"coupling": lambda: run_coupling(dev, local_rank, with_oracle=not args.no_cpu_baseline),
                "wells": lambda: run_wells(dev, local_rank),
                "pn": lambda: run_pn(dev, local_rank),
                "impec": lambda: run_impec(dev, local_rank),
                "small_case": lambda: run_small_case(dev, local_rank),
                "oil_water": lambda: run_oil_water(dev, local_rank),
                "adjoint": lambda: run_adjoint(dev, local_rank),
                "ensemble": lambda: run_ensemble(dev, local_rank)}[args.only]
        print(json.dumps({args.only: part()}))
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
