#!/usr/bin/env python
"""Benchmark of the APM solve (Passy & Bryan, arXiv:1410.0010) on GB300.

One step = one full APM solve over the workload's hierarchy: per level the
drift + TSC deposit (+ baryons), the FFT convolution with the Green's table,
the FD accelerations with the parent carry, then the TSC interpolation to all
particles.  Default workload: periodic 512^3 root + 2 levels of 64 subgrids of
128^3, 16,777,216 Zel'dovich particles (the largest single-GPU configuration).

Prints ONE JSON line (rank 0): the step's throughput and per-kernel bandwidth,
the dominant kernel's roofline (with its ncu DRAM traffic when the sources
match the capture), the end-to-end step through StepPipeline, the FP64 path,
the plain per-grid path (the same kernels launched grid by grid, FP64 and
FP32) and the batched FP32 step's speed-up over it, the FFT passes' combined
fraction of HBM peak, the other gradient operators, one evolution timestep and
the kick-drift, the cuFFT comparison, and the CPU oracle on a sample together
with each GPU path's error against it.  `--impl reference` times the
FP64 CPU oracle on a bounded sample of the same workload instead;
`--write-traffic CSV` writes profiles/traffic.json from an ncu capture.
Run: python bench.py [--gpus N --steps K --warmup W] [--workload c5|c4|c3|c2|c1]
     [--gradient fd2|fd4|spectral]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

FALLBACK_HBM_GBS = 6800.0
METRIC = "APM level-solve Mcells/s + particles/s, FP32 vs FP64 GPU at stated err; HBM GB/s"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def workload(name):
    import apm_inputs as W
    return W.CONFIGS[name]()


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) == 7:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        smax = max(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------
# algorithmic bytes of each kernel (compulsory HBM traffic of its inputs/outputs)
# ----------------------------------------------------------------------------
def interp_field_bytes(w, levels, parts, half_dt, rsz, chunk=1 << 22):
    """Acceleration-field bytes the interpolation reads at least once: each
    particle reads the 27 cells around its drifted position on its owner grid
    (the finest solved grid whose interior holds it), three components of rsz
    bytes; a cell read by several particles counts once.  Computed on the
    device from the particle arrays (FP64 drift; a particle on a cell edge may
    land one cell over, which changes the count negligibly)."""
    import torch
    N0 = w.grids[0].dims[0]
    x = [parts[k] + parts["v" + k] * half_dt for k in ("x", "y", "z")]
    if w.periodic:
        x = [torch.remainder(v, 1.0) for v in x]
    n = x[0].numel()
    dev = x[0].device
    owner = torch.full((n,), -1, dtype=torch.int32, device=dev)
    order = sorted((g.level, gi) for gi, g in enumerate(w.grids) if g.level in levels)
    for lev, gi in order:                      # coarse to fine: a finer grid overrides
        g = w.grids[gi]
        scale = N0 * 2 ** lev
        inside = torch.ones(n, dtype=torch.bool, device=dev)
        for j in range(3):
            c = torch.floor(x[j] * scale).to(torch.int64)
            inside &= (c >= g.start[j]) & (c < g.start[j] + g.dims[j])
        owner[inside] = gi
    offs = torch.stack(torch.meshgrid(*(torch.arange(-1, 2, device=dev),) * 3, indexing="ij"), -1).reshape(27, 3)
    total = 0
    for lev, gi in order:
        g = w.grids[gi]
        E = [d + 2 for d in g.dims]
        mark = torch.zeros(E[0] * E[1] * E[2], dtype=torch.bool, device=dev)
        ids = torch.nonzero(owner == gi).flatten()
        scale = N0 * 2 ** lev
        for a in range(0, ids.numel(), chunk):
            sel = ids[a:a + chunk]
            c = torch.stack([torch.floor(x[j][sel] * scale).to(torch.int64) - g.start[j] + 1 for j in range(3)], -1)
            cl = (c[:, None, :] + offs[None, :, :]).reshape(-1, 3)
            ok = ((cl >= 0) & (cl < torch.tensor(E, device=dev))).all(-1)
            cl = cl[ok]
            mark[cl[:, 0] + E[0] * (cl[:, 1] + E[1] * cl[:, 2])] = True
        total += int(mark.sum()) * 3 * rsz
    return total


def algorithmic_bytes(solver, w, levels, csz, rsz, batched, interp_fields=None):
    """Bytes per step per kernel, summed over the solved levels.

    csz / rsz: bytes of one complex / real value of the precision; batched:
    the deposit and the interpolation read the particles once for all levels.
    The spectral gradient runs the z, y-inverse and x-inverse passes once per
    component (phi, A_x, A_y, A_z), each reading its input again; its
    acceleration kernel reads phi and the three components on the output
    cells instead of differencing.  interp_fields: the acceleration-field
    bytes the interpolation reads (interp_field_bytes); None counts every
    grid's whole field."""
    out = {k: 0 for k in ("gas_init", "tsc_deposit", "fft_x_fwd", "fft_y_fwd", "fft_z_green",
                          "fft_y_inv", "fft_x_inv", "accel_carry", "tsc_interp", "particle_order")}
    n = w.n_particles
    # the particle order: positions and velocities read (48 B), bin and rank
    # written and read back (16 B), the permutation written (4 B)
    out["particle_order"] = 68 * n if getattr(solver, "order_capacity", 0) else 0
    for lev in levels:
        kinds = solver.pass_kernels(lev)
        for j, gi in enumerate(solver.level_grids[lev]):
            inf = solver.info[gi]
            G, M, Wd, F = inf["gmf"], inf["fft"], inf["phi_short"], inf["field"]
            Hx = M[0] // 2 + 1
            cg = G[0] * G[1] * G[2]
            gas_b = 8 * int(np.prod(w.grids[gi].dims)) if (w.gas is not None and w.gas[gi] is not None) else 0
            out["gas_init"] += 8 * cg + gas_b
            out["tsc_deposit"] += 8 * cg                      # the accumulated field
            if kinds[0][j] == 2:                       # fused x + y forward: GMF in, y spectrum out
                out["fft_x_fwd"] += 8 * cg + csz * G[2] * M[1] * Hx
            else:
                out["fft_x_fwd"] += 8 * cg + csz * G[1] * G[2] * Hx
                out["fft_y_fwd"] += csz * G[1] * G[2] * Hx + csz * G[2] * M[1] * Hx
            comps = inf.get("comps", 1)
            out["fft_z_green"] += comps * (csz * G[2] * M[1] * Hx + csz * Wd[2] * M[1] * Hx
                                           + rsz * Hx * (M[1] // 2 + 1) * (M[2] // 2 + 1))
            if kinds[4][j] == 2:                       # fused y + x inverse: z output in, window out
                out["fft_x_inv"] += comps * (csz * Wd[2] * M[1] * Hx + rsz * Wd[0] * Wd[1] * Wd[2])
            else:
                out["fft_y_inv"] += comps * (csz * Wd[2] * M[1] * Hx + csz * Wd[2] * Wd[1] * Hx)
                out["fft_x_inv"] += comps * (csz * Wd[2] * Wd[1] * Hx + rsz * Wd[0] * Wd[1] * Wd[2])
            ec = F[0] * F[1] * F[2]
            if comps > 1:
                out["accel_carry"] += 4 * rsz * ec + 4 * rsz * ec
            else:
                out["accel_carry"] += rsz * Wd[0] * Wd[1] * Wd[2] + 4 * rsz * ec
            if interp_fields is None:
                out["tsc_interp"] += 3 * rsz * ec
        if not batched:
            out["tsc_deposit"] += 56 * n      # x, y, z, vx, vy, vz, m per level
            out["tsc_interp"] += 48 * n       # positions and velocities per level
    if batched:                               # one pass over the particles for all levels
        out["tsc_deposit"] += 56 * n
        out["tsc_interp"] += 48 * n
    out["tsc_interp"] += 3 * rsz * n      # accelerations written once
    if interp_fields is not None:
        out["tsc_interp"] += interp_fields
    return out


def cufft_convolution_ms(solver, levels, dev, steps, timed):
    """The same convolutions done with cuFFT (torch.fft), for comparison: per
    level, every grid's FP32 field on its M grid (batched by M shape),
    forward R2C, multiplied by a real half-spectrum table, inverse C2R.  No
    zero-padding pruning or windowing; the table is a stand-in of the right
    shape.  Returns {"ms_per_step": ..., "batches": [...]}."""
    import torch
    groups = {}
    for lev in levels:
        for gi in solver.level_grids[lev]:
            M = tuple(solver.info[gi]["fft"])
            groups[M] = groups.get(M, 0) + 1
    bufs = []
    for M, cnt in groups.items():
        x = torch.rand((cnt, M[2], M[1], M[0]), dtype=torch.float32, device=dev)
        t = torch.rand((M[2], M[1], M[0] // 2 + 1), dtype=torch.float32, device=dev)
        bufs.append((x, t))

    def conv():
        for x, t in bufs:
            y = torch.fft.irfftn(torch.fft.rfftn(x, dim=(1, 2, 3)) * t, s=x.shape[1:], dim=(1, 2, 3))
            del y

    for _ in range(2):
        conv()
    ms = timed(conv, max(steps, 1))
    out = {"ms_per_step": ms, "batches": [{"M": list(M), "grids": c} for M, c in groups.items()],
           "library": "cuFFT via torch.fft (R2C, multiply, C2R; full M grids)"}
    del bufs
    torch.cuda.empty_cache()
    return out


def kernel_source_hash():
    """sha256 over the CUDA sources of the library (file names and contents, in
    name order): identifies the kernels a DRAM-traffic capture was taken on."""
    import hashlib
    d = os.path.join(ROOT, "paper_1410_0010_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h")):
            h.update(name.encode())
            with open(os.path.join(d, name), "rb") as f:
                h.update(f.read())
    return h.hexdigest()


def ncu_label(name):
    """bench.py's kernel label of an ncu kernel name, or None.  The column passes
    (runtime k_col<T, axis, mode, threads> and compile-time-planned
    k_col_fast<plan, axis, mode, lines, threads>) by their axis and mode; the
    fused plane kernels by the x pass they stand in for."""
    import re
    # anonymous-namespace markers: "ns::<unnamed>::" (demangled) or
    # "unnamed>::" (ncu's CSV)
    name = name.replace("::<unnamed>::", "::").replace("unnamed>::", "")
    m = re.search(r"\bk_([a-z_]+)[<(]", name)
    if not m:
        return None
    base = m.group(1)
    if base in ("col", "col_fast"):
        rest = re.sub(r"FastPlan<[^>]*>", "P", name[m.end():])
        a = [t.strip() for t in rest.split(">")[0].split(",")]
        return {("1", "0"): "fft_y_fwd", ("2", "1"): "fft_z_green", ("1", "2"): "fft_y_inv",
                ("2", "3"): "fft_z_green"}.get((a[1], a[2])) if len(a) >= 3 else None
    return {"gas_init": "gas_init", "deposit_levels": "tsc_deposit", "deposit": "tsc_deposit",
            "xf": "fft_x_fwd", "xf_fast": "fft_x_fwd", "xy_fast": "fft_x_fwd",
            "xi": "fft_x_inv", "xi_fast": "fft_x_inv", "yx_fast": "fft_x_inv",
            "accel": "accel_carry", "accel_var": "accel_carry", "interp_levels": "tsc_interp",
            "interp": "tsc_interp"}.get(base)


def write_traffic(csv_paths, small="c5s", full="c5", scale=8):
    """profiles/traffic.json from ncu --csv captures (one or more files, comma
    separated) of the `small` workload: dram__bytes_read.sum +
    dram__bytes_write.sum per launch, mean over the captured launches of each
    kernel label, with the per-launch figures scaled by `scale` for the `full`
    workload and the sha256 of the current sources."""
    import csv
    unit = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    per = {}
    for fi, csv_path in enumerate(csv_paths.split(",")):
        rows = list(csv.reader(open(csv_path)))
        hdr = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
        H = rows[hdr]
        ki, mi, vi, ui, ii = (H.index(c) for c in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit", "ID"))
        for r in rows[hdr + 1:]:
            if len(r) <= vi or not r[mi].startswith("dram__bytes_"):
                continue
            label = ncu_label(r[ki])
            if label is None:
                continue
            d = per.setdefault(label, {})
            key = (fi, int(r[ii]))
            d[key] = d.get(key, 0.0) + float(r[vi].replace(",", "")) * unit.get(r[ui], 1)
    import apm_inputs as W
    ws, wf = W.NAMES[small], W.NAMES[full]
    out = {}
    for label, launches in sorted(per.items()):
        mean = sum(launches.values()) / len(launches)
        out[f"{ws}:{label}"] = int(round(mean))
        out[f"{wf}:{label}"] = int(round(mean * scale))
    doc = {"source_sha256": kernel_source_hash(),
           "note": ("dram__bytes_read.sum + dram__bytes_write.sum per launch (mean over the captured launches "
                    f"of each kernel label), captured on {ws} and scaled x{scale} to {wf} ({scale}x the cells, "
                    f"grids and particles per launch); the {ws} values are kept as measured"),
           "per_launch_bytes": out}
    path = os.path.join(ROOT, "profiles", "traffic.json")
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
    return path


# ----------------------------------------------------------------------------
# oracle sample (CPU baseline and the reference arm)
# ----------------------------------------------------------------------------
def sample_grids(w, n_grids=2):
    """The grids the oracle sample solves: the first n_grids refined grids of the
    solved levels, or the root when no refined level is solved."""
    ids = [i for i, g in enumerate(w.grids)
           if g.level >= 1 and (w.solve_levels is None or g.level in w.solve_levels)][:n_grids]
    return ids or [0]


def oracle_sample(w, n_grids=2, outputs=None):
    """The sampled grids of the workload (sample_grids) solved by the FP64 CPU
    oracle: TSC deposit of every particle touching each GMF (with the grid's
    gas and, on its border, the parent's), naive-DFT convolution on its M
    grid, FD accelerations (the parent carry is omitted: zero parent fields).  Returns (interior cells, seconds,
    description); with outputs={} it also fills outputs[gi] = (phi_short, acc)."""
    import oracle
    cfg = oracle.Config(periodic=w.periodic, mass_frac_bits=w.mass_frac_bits)
    grids = [oracle.Grid(*g) for g in w.grids]
    ids = sample_grids(w, n_grids)
    oracle.lib()
    t0 = time.perf_counter()
    for gi in ids:
        gas = None if w.gas is None else w.gas[gi]
        par = w.grids[gi].parent
        pgas = None if (w.gas is None or par < 0) else w.gas[par]   # the border's baryons (Sec. 2)
        gmf, _ = oracle.deposit(cfg, grids, gi, w.particles, w.half_dt, gas=gas, parent_gas=pgas)
        phis = oracle.solve(cfg, grids, gi, gmf)
        _, acc = oracle.accel(cfg, grids, gi, phis)
        if outputs is not None:
            outputs[gi] = (phis, acc)
    dt = time.perf_counter() - t0
    cells = int(sum(np.prod(w.grids[gi].dims) for gi in ids))
    plans = [oracle.plan_grid(cfg, grids, gi).M for gi in ids]
    desc = (f"oracle solve of {len(ids)} grid(s) {[tuple(w.grids[gi].dims) for gi in ids]} "
            f"(M={plans}): deposit of all {w.n_particles} particles, naive-DFT convolution, "
            f"FD accelerations")
    return cells, dt, desc


def cpu_cores():
    n = os.environ.get("APM_ORACLE_THREADS")
    return int(n) if n and int(n) > 0 else (os.cpu_count() or 1)


# ----------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Ranks:
    """The process group around the timed region: a barrier, and the maximum or
    sum of a number over ranks (NCCL for GPU ranks; any backend whose tensors
    live on `device`).  With one rank every call is the identity."""

    def __init__(self, world, device):
        self.world = world
        self.device = device

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def _reduce(self, x, op):
        if self.world == 1:
            return x
        import torch
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        import torch.distributed as dist
        return self._reduce(x, dist.ReduceOp.MAX)

    def sum(self, x):
        import torch.distributed as dist
        return self._reduce(x, dist.ReduceOp.SUM)


def job_rate(ranks, units, ms):
    """Whole-job throughput in millions of units per second: the units all ranks
    processed over the slowest rank's time (ms, the max over ranks)."""
    return ranks.sum(units) / (ms / 1e3) / 1e6


def snapshot(solver, bufs, ids):
    """Host copies of the sampled grids' phi_short and accelerations."""
    out = {}
    for gi in ids:
        lev, k = solver.info[gi]["level"], solver.info[gi]["level_index"]
        out[gi] = (bufs[lev]["phis"][k].double().cpu().numpy(), bufs[lev]["acc"][k].double().cpu().numpy())
    return out


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def errors_vs_oracle(snap, ref, carried):
    """Relative L2 of the GPU outputs against the oracle's on the sampled grids:
    phi_short always; the accelerations only on grids whose step added no
    parent carry (the oracle sample omits it)."""
    e_phi = max(rel_l2(snap[gi][0], ref[gi][0]) for gi in ref)
    acc = [rel_l2(snap[gi][1], ref[gi][1]) for gi in ref if not carried(gi)]
    return {"phi_short": e_phi, "acc": max(acc) if acc else None}


def fft_pass_summary(prof, ab, steps, hbm):
    """The five FFT passes together: algorithmic bytes over their summed device
    time per step, and that bandwidth as a fraction of the HBM peak."""
    names = ("fft_x_fwd", "fft_y_fwd", "fft_z_green", "fft_y_inv", "fft_x_inv")
    ms = sum(prof[k][1] for k in names if k in prof) / max(steps, 1)
    byts = sum(ab[k] for k in names)
    gbs = byts / (ms * 1e-3) / 1e9 if ms > 0 else None
    return {"ms_per_step": ms, "bytes_per_step": byts, "GBps": gbs, "frac": gbs / hbm if gbs else None}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = workload(args.workload)
    times, cells = [], 0
    for i in range(args.warmup + args.steps):
        c, dt, desc = oracle_sample(w)
        if i >= args.warmup:
            times.append(dt)
            cells = c
    t = sum(times) / len(times)
    value = cells / t / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mcells/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "sample": desc},
            "cpu_baseline": {"value": value, "unit": "Mcells/s", "cores": cpu_cores(),
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "Mcells/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_apm(args):
    import torch
    import torch.distributed as dist

    from paper_1410_0010_gb300.solver import Particles, Solver, StepPipeline

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    w = workload(args.workload)
    levels = list(range(1 + max(g.level for g in w.grids))) if w.solve_levels is None else w.solve_levels

    # auto: measured below (with and without the order, after tuning); the
    # other legs follow the choice
    use_order = args.order in ("on", "tiles") or (args.order == "auto" and not w.spatial_order)
    use_tiles = args.order == "tiles"
    order_note = args.order

    def make(precision, gradient=args.gradient, order=None):
        s = Solver(w.grids, periodic=w.periodic, precision=precision,
                   mass_frac_bits=w.mass_frac_bits, device=local, gradient=gradient)
        if use_order if order is None else order:   # the particle processing order, recomputed every step
            s.reserve_order(w.n_particles)
            s.set_deposit_tiles(use_tiles)          # ... and the deposit through shared-memory tiles
        return s, s.alloc_all()

    host = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in w.particles.items()}
    dparts = {k: v.to(dev) for k, v in host.items()}
    P = Particles(dparts)
    gas = None
    if w.gas is not None:
        gas = [None if g is None else torch.from_numpy(np.ascontiguousarray(g)).to(dev) for g in w.gas]
    n = w.n_particles
    cells = w.interior_cells(levels)

    ranks = Ranks(world, dev)

    def timed(fn, steps):
        ranks.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ranks.barrier()
        return ranks.max(e0.elapsed_time(e1) / steps)

    # ---------------- FP32 (the product configuration)
    s32, b32 = make("fp32")
    pacc = torch.zeros((3, n), dtype=torch.float32, device=dev)

    def step32():
        s32.step(P, w.half_dt, b32, pacc, gas=gas, levels=levels)

    # FFT pass launch shapes from the library's autotuner (one tuned solve per level)
    shapes32 = s32.autotune(P, w.half_dt, b32, gas=gas, levels=levels) if not args.no_tune else None
    for _ in range(args.warmup):
        step32()
    s32.sync_status()
    if args.order == "auto" and not w.spatial_order:
        # the order costs a sort per step and pays in the particle kernels only
        # where the caller's order is incoherent: five eager steps each way
        def t_order(on, tiles):
            s32.reserve_order(n if on else 0)
            s32.set_deposit_tiles(tiles)
            for _ in range(2):
                step32()
            return timed(step32, 5)
        t = {"off": t_order(False, False), "on": t_order(True, False), "tiles": t_order(True, True)}
        pick = min(t, key=t.get)
        use_order, use_tiles = pick != "off", pick == "tiles"
        s32.reserve_order(n if use_order else 0)
        s32.set_deposit_tiles(use_tiles)
        order_note = ("auto: ms per eager step " +
                      ", ".join(f"{k} {v:.3f}" for k, v in t.items()) + f"; chose {pick}")
        for _ in range(2):
            step32()
        s32.sync_status()
    graph = None
    try:   # the step as a library-owned CUDA graph (apm_graph_begin / apm_graph_end)
        graph = s32.capture(step32)
        graph.replay()
        torch.cuda.synchronize()
        s32.sync_status()
    except Exception as exc:  # capture is an optimisation; eager launches are the fallback
        print(f"# graph capture failed ({exc}); timing eager launches", file=sys.stderr)
        graph = None
    run = graph.replay if graph is not None else step32
    used_graph = graph is not None

    clocks = Clocks(local)
    clocks.start()
    ms = timed(run, args.steps)
    clk = clocks.stop()
    s32.sync_status()
    ids = sample_grids(w)
    snap32 = snapshot(s32, b32, ids)

    # per-kernel device times (tracing on, eager, same workload)
    s32.profile(True)
    for _ in range(args.steps):
        step32()
    prof = s32.profile_read()
    s32.profile(False)
    launches_per_step = sum(v[0] for v in prof.values()) / max(args.steps, 1)

    # end to end: host inputs copied in, particle accelerations copied out, every
    # step.  Serial: copy in, solve, copy out on one stream.  Pipelined
    # (StepPipeline, the library's end-to-end driver): two device buffer sets,
    # step k+1's upload and step k-1's download overlap step k's solve.
    hout = torch.empty((3, n), dtype=torch.float32).pin_memory()

    def e2e_step():
        for k in dparts:
            dparts[k].copy_(host[k], non_blocking=True)
        run()                     # the captured step (same launches as step32)
        hout.copy_(pacc, non_blocking=True)

    e2e_serial_ms = timed(e2e_step, args.steps)
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = hout.numel() * hout.element_size()
    pipe = StepPipeline(s32, b32, host, w.half_dt, gas=gas, levels=levels)
    pipe.run(args.warmup)
    e2e_ms = timed(lambda: pipe.run(args.steps), 1) / args.steps
    s32.sync_status()
    del pipe

    # ---------------- FP64 GPU path (same kernels in double), and the FP32 error against it
    fp64 = None
    if not args.no_fp64:
        phi32 = [t.clone() for t in b32[-1]["phi"]]
        pacc32 = pacc.clone()
        graph = None
        run = None
        s64, b64 = make("fp64")
        pacc64 = torch.zeros((3, n), dtype=torch.float64, device=dev)

        def step64():
            s64.step(P, w.half_dt, b64, pacc64, gas=gas, levels=levels)

        if not args.no_tune:
            s64.autotune(P, w.half_dt, b64, gas=gas, levels=levels)
        for _ in range(max(1, args.warmup // 2)):
            step64()
        s64.sync_status()
        ms64 = timed(step64, max(1, args.steps // 2))
        own = pacc64.abs().sum(0) > 0
        e_pacc = float(torch.linalg.vector_norm((pacc32.double() - pacc64)[:, own]) /
                       torch.linalg.vector_norm(pacc64[:, own]))
        e_phi = float(max(torch.linalg.vector_norm(a.double() - b) / torch.linalg.vector_norm(b)
                          for a, b in zip(phi32, b64[-1]["phi"])))
        fp64 = {"value": job_rate(ranks, cells, ms64), "ms_per_step": ms64,
                "fp32_speedup": ms64 / ms, "fp32_rel_l2_vs_fp64": {"phi_finest": e_phi, "pacc": e_pacc}}
        snap64 = snapshot(s64, b64, ids)
        s64.close()
        del b64, pacc64

    # ---------------- the plain per-grid path: the same kernels launched grid
    # by grid (apm_set_grid_batching(0)) for the level solve and the
    # accelerations, FP64 and FP32, graph-captured like the main step;
    # the batched FP32 step's speed-up over it at the accuracy reported
    per_grid = None
    if not args.no_per_grid:
        per_grid = {"launch": "one launch sequence per grid for apm_solve_level and apm_accel; "
                              "deposit and interpolation one pass over the particles for all levels, "
                              "in the particles' own order"}
        for prec in ("fp64", "fp32"):
            sp, bp = make(prec, order=False)
            sp.set_grid_batching(False)
            pp = torch.zeros((3, n), dtype=sp.dtype, device=dev)

            def stepp():
                sp.step(P, w.half_dt, bp, pp, gas=gas, levels=levels)

            # the main solver's shapes and plans (its own tuning for FP64), so the
            # FP32 per-grid step runs the same kernels grid by grid
            if prec == "fp32" and shapes32:
                for lev, sh in shapes32.items():
                    sp.set_fft_shapes(lev, sh)
            elif not args.no_tune:
                sp.autotune(P, w.half_dt, bp, gas=gas, levels=levels)
            stepp()
            sp.sync_status()
            gp = sp.capture(stepp)
            gp.replay()
            torch.cuda.synchronize()
            sp.sync_status()
            msp = timed(gp.replay, max(1, args.steps // 2))
            ms_eager = timed(stepp, 1)
            ref = pacc if prec == "fp32" else None
            per_grid[prec] = {"ms_per_step": msp, "value": job_rate(ranks, cells, msp),
                              "eager_ms_per_step": ms_eager,
                              "launches_per_step": None,
                              "equal_to_batched": bool(torch.equal(pp, ref)) if ref is not None else None}
            sp.profile(True)
            stepp()
            lp = sp.profile_read()
            sp.profile(False)
            per_grid[prec]["launches_per_step"] = sum(v[0] for v in lp.values())
            del gp
            sp.close()
            del bp, pp
        per_grid["batched_fp32_speedup_vs_per_grid_fp64"] = per_grid["fp64"]["ms_per_step"] / ms
        per_grid["batched_fp32_speedup_vs_per_grid_fp32"] = per_grid["fp32"]["ms_per_step"] / ms

    # ---------------- one evolution timestep (solve at half_dt = dt/2, then the
    # kick-drift), graph-captured, on a copy of the particles (the kick moves
    # them); the kick-drift alone against its algorithmic bytes: six FP64
    # arrays read and written and the accelerations read, per particle
    evolution = None
    if not args.no_evolution:
        Pe = Particles({k: v.clone() for k, v in dparts.items()})
        dt = 2.0 * w.half_dt
        pe = torch.zeros((3, n), dtype=torch.float32, device=dev)
        s32.step(Pe, w.half_dt, b32, pe, gas=gas, levels=levels)
        s32.kick_drift(Pe, pe, dt)
        def evo():
            s32.step(Pe, w.half_dt, b32, pe, gas=gas, levels=levels)
            s32.kick_drift(Pe, pe, dt)

        ge = s32.capture(evo)
        ge.replay()
        torch.cuda.synchronize()
        s32.sync_status()
        ms_evo = timed(ge.replay, args.steps)
        ms_kick = timed(lambda: s32.kick_drift(Pe, pe, dt), max(args.steps, 10))
        s32.sync_status()
        kick_bytes = (12 * 8 + 3 * 4) * n
        evolution = {"ms_per_step": ms_evo, "steps_per_s": 1e3 / ms_evo,
                     "kick_drift": {"ms_per_launch": ms_kick, "bytes_per_launch": kick_bytes,
                                    "GBps": kick_bytes / (ms_kick * 1e-3) / 1e9,
                                    "frac": kick_bytes / (ms_kick * 1e-3) / 1e9 / peaks()[0]}}
        del ge, Pe, pe

    # ---------------- the other gradient operators (Sec. 2.2), FP32, same workload
    gradients = None
    if not args.no_gradients:
        gradients = {}
        from paper_1410_0010_gb300._lib import ApmError
        for grad in [g for g in ("fd2", "fd4", "spectral") if g != args.gradient]:
            try:
                sv, bv = make("fp32", grad)
            except ApmError as exc:      # e.g. the four-point root limit (N0 <= 511, isolated)
                gradients[grad] = {"unsupported": str(exc)}
                continue
            pv = torch.zeros((3, n), dtype=torch.float32, device=dev)

            def stepv():
                sv.step(P, w.half_dt, bv, pv, gas=gas, levels=levels)

            if not args.no_tune:
                sv.autotune(P, w.half_dt, bv, gas=gas, levels=levels)
            for _ in range(args.warmup):
                stepv()
            sv.sync_status()
            gv = sv.capture(stepv)
            gv.replay()
            torch.cuda.synchronize()
            sv.sync_status()
            msv = timed(gv.replay, args.steps)
            sv.profile(True)
            for _ in range(args.steps):
                stepv()
            pv_prof = sv.profile_read()
            sv.profile(False)
            sv.sync_status()
            gradients[grad] = {
                "value": job_rate(ranks, cells, msv), "ms_per_step": msv, "time_vs_main": msv / ms,
                "kernel_ms_per_step": {k: v[1] / args.steps for k, v in pv_prof.items() if v[0]},
                "launches_per_step": sum(v[0] for v in pv_prof.values()) / args.steps}
            del gv
            sv.close()
            del bv, pv

    # ---------------- cuFFT comparison (context only: cuFFT is not on the product path)
    cufft = None
    if not args.no_cufft and args.gradient == "fd2":     # cuFFT does one convolution, like the two-point path
        cufft = cufft_convolution_ms(s32, levels, dev, args.steps, timed)
        ours = sum(prof[k][1] for k in ("fft_x_fwd", "fft_y_fwd", "fft_z_green", "fft_y_inv", "fft_x_inv")
                   if k in prof) / max(args.steps, 1)
        cufft["ours_ms_per_step"] = ours

    # ---------------- roofline of the dominant kernel
    hbm, peak_src = peaks()
    batched = levels == list(range(s32.n_levels))
    ab = algorithmic_bytes(s32, w, levels, 8, 4, batched,
                           interp_fields=interp_field_bytes(w, levels, dparts, w.half_dt, 4))
    kernels = {}
    for name, (cnt, tot) in prof.items():
        if cnt == 0:
            continue
        per_launch_ms = tot / cnt
        bytes_per_launch = ab[name] / (cnt / args.steps)
        kernels[name] = {"launches_per_step": cnt / args.steps, "ms_per_launch": per_launch_ms,
                         "share": tot / sum(v[1] for v in prof.values()),
                         "GBps": bytes_per_launch / (per_launch_ms * 1e-3) / 1e9}
    fft_passes = fft_pass_summary(prof, ab, args.steps, hbm)
    top = max(kernels, key=lambda k: kernels[k]["share"])
    ach = kernels[top]["GBps"]
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tj = json.load(f)
        # counters taken on other kernel sources (or on the two-point path when
        # another operator runs) do not describe these kernels
        if tj.get("source_sha256") == kernel_source_hash() and args.gradient == "fd2":
            traffic = tj.get("per_launch_bytes", {}).get(f"{w.name}:{top}")
    roofline = {"bound": "hbm", "kernel": top, "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "peak_source": peak_src, "traffic": traffic}

    # ---------------- CPU baseline: the oracle on a bounded sample (rank 0, N = 1)
    cpu = None
    err_oracle = None
    if rank == 0 and world == 1 and not args.no_cpu:
        ref = {}
        c, dt, desc = oracle_sample(w, outputs=ref)
        cpu = {"value": c / dt / 1e6, "unit": "Mcells/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": desc, "seconds": dt}

        def carried(gi):
            lev = s32.info[gi]["level"]
            return lev > 0 and (lev - 1) in levels

        err_oracle = {"grids": ids, "fp32": errors_vs_oracle(snap32, ref, carried),
                      "fp64": errors_vs_oracle(snap64, ref, carried) if fp64 is not None else None,
                      "tolerance": {"fp32": {"phi_short": 2e-5, "acc": 1e-4}, "fp64": 1e-12}}

    value = job_rate(ranks, cells, ms)
    line = {
        "metric": METRIC, "value": value, "unit": "Mcells/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "levels": levels, "grids": len(w.grids),
                   "interior_cells": cells, "particles": n, "periodic": w.periodic,
                   "l2": "inputs larger than L2 (no flush)", "cuda_graph": used_graph,
                   "parallelism": f"replicas x{world}", "gradient": args.gradient,
                   "particle_order": ("tiles" if use_tiles else "on") if use_order else "off",
                   "particle_order_choice": order_note,
                   "fft_shapes": shapes32},
        "particles_per_s": job_rate(ranks, n, ms) * 1e6,
        "roofline": roofline,
        "kernels": kernels,
        "cpu_baseline": cpu,
        "e2e": {"value": job_rate(ranks, cells, e2e_ms), "unit": "Mcells/s",
                "ms_per_step": e2e_ms, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "pipelined": True, "serial_ms_per_step": e2e_serial_ms},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "fp64": fp64,
        "per_grid": per_grid,
        "fft_passes": fft_passes,
        "rel_l2_vs_oracle": err_oracle,
        "gradients": gradients,
        "evolution": evolution,
        "cufft_compare": cufft,
        "clocks": clk,
    }
    s32.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def probe_peaks():
    """Builds and runs the compute-peak probe (csrc/peak_probe.cu) and writes
    profiles/compute_peaks.json: measured FP32/FP64 FMA, INT32 multiply-add,
    warp-issue and 64-bit reduction rates of this GPU, the denominators of the
    kernels that are bound by instruction issue rather than HBM."""
    from paper_1410_0010_gb300 import buildlib
    exe = buildlib.build_probe()
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    doc = json.loads(out.strip().splitlines()[-1])
    doc["command"] = "python bench.py --probe-peaks"
    doc["when"] = time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())
    path = os.path.join(ROOT, "profiles", "compute_peaks.json")
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
    return path


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["apm", "reference"], default="apm")
    ap.add_argument("--workload", choices=["c1", "c2", "c3", "c4", "c5", "c5s"], default="c5")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--order", choices=["auto", "on", "off", "tiles"], default="auto",
                    help="sort the particles by root-level bin every step before the particle kernels "
                         "(apm_order_particles; results are bit-identical either way); tiles: also deposit "
                         "through shared-memory tiles (apm_set_deposit_tiles); auto: off when the workload "
                         "stores its particles in spatial order (the Zel'dovich lattice), otherwise the fastest "
                         "of five eager steps each way")
    ap.add_argument("--no-per-grid", action="store_true",
                    help="skip timing the plain per-grid launch path (FP64 and FP32)")
    ap.add_argument("--no-tune", action="store_true", help="default FFT pass shapes, no autotuner")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT convolution comparison")
    ap.add_argument("--write-traffic", metavar="CSV[,CSV...]",
                    help="write profiles/traffic.json from ncu --csv captures of c5s launches, then exit")
    ap.add_argument("--no-evolution", action="store_true", help="skip timing the evolution timestep")
    ap.add_argument("--gradient", choices=["fd2", "fd4", "spectral"], default="fd2",
                    help="the gradient operator of the measured solve (default: the two-point difference)")
    ap.add_argument("--no-gradients", action="store_true",
                    help="skip timing the other gradient operators")
    ap.add_argument("--probe-peaks", action="store_true",
                    help="measure this GPU's FP32/FP64/INT32, issue and reduction rates into "
                         "profiles/compute_peaks.json, then exit")
    args = ap.parse_args()
    if args.probe_peaks:
        print(probe_peaks())
        return 0
    if args.write_traffic:
        print(write_traffic(args.write_traffic))
        return 0
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_apm(args)


if __name__ == "__main__":
    sys.exit(main())
