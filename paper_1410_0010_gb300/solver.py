"""Python face of libapm: the four C-ABI calls with torch tensors as device
memory and torch streams.  Every step of the solve runs in the library's CUDA
kernels; this module only marshals pointers and allocates output buffers.
"""
import ctypes
import json
import os

import torch

from . import _lib
from ._lib import ApmConfig, ApmFftShapes, ApmGrid, ApmGridInfo, ApmParticles, check, lib, ptr_array

PARTICLE_KEYS = ("x", "y", "z", "vx", "vy", "vz", "m")


def _stream_handle(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else t.data_ptr()


def check_field(t, shape, dtype, device, name):
    """The C ABI sees only a pointer: a tensor handed to it must have this
    exact shape and dtype, be contiguous and live on the context's device."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if t.dtype != dtype:
        raise ValueError(f"{name} has dtype {t.dtype}, expected {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, the context on {device}")


class Particles:
    """Device particle arrays (float64, contiguous) and their C view."""

    def __init__(self, arrays):
        self.t = {}
        n = None
        for k in PARTICLE_KEYS:
            a = arrays[k]
            if not a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous():
                raise ValueError(f"particle array {k} must be a contiguous float64 CUDA tensor")
            n = a.numel() if n is None else n
            if a.numel() != n:
                raise ValueError("particle arrays differ in length")
            self.t[k] = a
        self.n = int(n)
        self.c = ApmParticles(self.n, *[self.t[k].data_ptr() for k in PARTICLE_KEYS])


class Solver:
    """One APM context on one GPU with a static grid hierarchy.

    grids: sequence of (level, parent, start(3), dims(3)); grid 0 is the root.
    gradient: "fd2" (two-point difference), "fd4" (four-point) or "spectral"
    (D = -ik), the operator the accelerations and the influence function use.
    """

    def __init__(self, grids, periodic=False, precision="fp32", mass_frac_bits=52,
                 root_correction=True, a_over_dx=3.4, pad_factor=0.65, box=1.0, device=None,
                 gradient="fd2"):
        L = lib()
        cfg = ApmConfig()
        L.apm_config_default(ctypes.byref(cfg))
        cfg.box = box
        cfg.a_over_dx = a_over_dx
        cfg.pad_factor = pad_factor
        cfg.root_bc = _lib.APM_BC_PERIODIC if periodic else _lib.APM_BC_ISOLATED
        cfg.precision = _lib.APM_FP64 if precision == "fp64" else _lib.APM_FP32
        cfg.mass_frac_bits = int(mass_frac_bits)
        cfg.root_correction = 1 if root_correction else 0
        cfg.gradient = _lib.GRADIENTS[gradient]
        self.gradient = gradient
        dev = torch.cuda.current_device() if device is None else int(device)
        cfg.device = dev
        self.device = torch.device("cuda", dev)
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.precision = precision
        self._ctx = ctypes.c_void_p()
        check(L.apm_create(ctypes.byref(cfg), ctypes.byref(self._ctx)), "apm_create")
        self.grids = [tuple(g) for g in grids]
        arr = (ApmGrid * len(self.grids))()
        for i, (lev, par, start, dims) in enumerate(self.grids):
            arr[i].level = int(lev)
            arr[i].parent = int(par)
            for j in range(3):
                arr[i].start[j] = int(start[j])
                arr[i].dims[j] = int(dims[j])
        try:
            check(L.apm_set_hierarchy(self._ctx, arr, len(self.grids)), "apm_set_hierarchy")
        except Exception:
            L.apm_destroy(self._ctx)
            self._ctx = None
            raise
        self.n_levels = L.apm_num_levels(self._ctx)
        self.info = []
        for i in range(len(self.grids)):
            gi = ApmGridInfo()
            check(L.apm_get_grid_info(self._ctx, i, ctypes.byref(gi)), "apm_get_grid_info")
            self.info.append(dict(level=gi.level, border=gi.border, gmf=tuple(gi.gmf),
                                  fft=tuple(gi.fft), phi_short=tuple(gi.phi_short),
                                  field=tuple(gi.field), level_index=gi.level_index,
                                  delta=gi.delta, comps=gi.phi_short_comps))
        self.level_grids = [[i for i, g in enumerate(self.grids) if g[0] == lev]
                            for lev in range(self.n_levels)]

    def close(self):
        if getattr(self, "_ctx", None):
            lib().apm_destroy(self._ctx)
            self._ctx = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ buffers
    def alloc_level(self, level):
        """Output buffers of one level: gmf (int64), phi_short ([4, ...] with the
        spectral gradient), phi, acc ([3, ...])."""
        out = dict(gmf=[], phis=[], phi=[], acc=[])
        for gi in self.level_grids[level]:
            inf = self.info[gi]
            out["gmf"].append(torch.empty(inf["gmf"][::-1], dtype=torch.int64, device=self.device))
            shape = inf["phi_short"][::-1]
            if inf["comps"] > 1:
                shape = (inf["comps"],) + shape
            out["phis"].append(torch.empty(shape, dtype=self.dtype, device=self.device))
            out["phi"].append(torch.empty(inf["field"][::-1], dtype=self.dtype, device=self.device))
            out["acc"].append(torch.empty((3,) + inf["field"][::-1], dtype=self.dtype, device=self.device))
        return out

    def alloc_all(self):
        return [self.alloc_level(lev) for lev in range(self.n_levels)]

    # ------------------------------------------------------------------ C-ABI calls
    def deposit(self, level, particles, half_dt, gmf, gas=None, parent_gas=None, stream=None):
        P = particles if isinstance(particles, Particles) else Particles(particles)
        g = ptr_array([_ptr(t) for t in gmf])
        ga = None if gas is None else ptr_array([_ptr(t) for t in gas])
        pg = None if parent_gas is None else ptr_array([_ptr(t) for t in parent_gas])
        check(lib().apm_deposit(self._ctx, level, ctypes.byref(P.c), float(half_dt), ga, pg, g,
                                _stream_handle(stream)), "apm_deposit")

    def deposit_all(self, particles, half_dt, gmf, gas=None, stream=None):
        """apm_deposit_all: gmf / gas are lists over the hierarchy's grids."""
        P = particles if isinstance(particles, Particles) else Particles(particles)
        ga = None if gas is None else ptr_array([_ptr(t) for t in gas])
        check(lib().apm_deposit_all(self._ctx, ctypes.byref(P.c), float(half_dt), ga,
                                    ptr_array([_ptr(t) for t in gmf]), _stream_handle(stream)),
              "apm_deposit_all")

    def interp_all(self, acc, particles, half_dt, out, stream=None):
        """apm_interp_all: acc is a list over the hierarchy's grids."""
        P = particles if isinstance(particles, Particles) else Particles(particles)
        check_field(out, (3, P.n), self.dtype, self.device, "particle accelerations")
        check(lib().apm_interp_all(self._ctx, ptr_array([_ptr(t) for t in acc]), ctypes.byref(P.c),
                                   float(half_dt), out.data_ptr(), _stream_handle(stream)),
              "apm_interp_all")

    def _per_grid(self, bufs, key):
        """One buffer per grid in hierarchy order from the per-level lists of alloc_all()."""
        out = [None] * len(self.grids)
        for lev, ids in enumerate(self.level_grids):
            for k, gi in enumerate(ids):
                out[gi] = bufs[lev][key][k]
        return out

    def solve_level(self, level, gmf, phis, stream=None):
        check(lib().apm_solve_level(self._ctx, level, ptr_array([_ptr(t) for t in gmf]),
                                    ptr_array([_ptr(t) for t in phis]), _stream_handle(stream)),
              "apm_solve_level")

    def autotune_level(self, level, gmf, phis, stream=None):
        """apm_solve_level that also picks the fastest launch shape of each FFT pass."""
        check(lib().apm_autotune_level(self._ctx, level, ptr_array([_ptr(t) for t in gmf]),
                                       ptr_array([_ptr(t) for t in phis]), _stream_handle(stream)),
              "apm_autotune_level")

    def reserve_order(self, n_max):
        """Workspace for the particle processing order of up to n_max
        particles (0 frees it); while reserved, step() orders the particles
        (apm_order_particles) and the interpolation visits them in that
        order; results are bit-identical either way."""
        check(lib().apm_reserve_order(self._ctx, int(n_max)), "apm_reserve_order")
        self.order_capacity = int(n_max)

    def order_particles(self, particles, half_dt, stream=None):
        P = particles if isinstance(particles, Particles) else Particles(particles)
        check(lib().apm_order_particles(self._ctx, ctypes.byref(P.c), float(half_dt), _stream_handle(stream)),
              "apm_order_particles")

    def capture(self, fn):
        """Records the work fn() issues (typically step() and kick_drift()) as a
        CUDA graph owned by the library (apm_graph_begin / apm_graph_end), on a
        side stream ordered after the current one, and returns a Graph whose
        replay() launches it on the current stream.  Run fn() once before
        capturing it."""
        side = torch.cuda.Stream(device=self.device)
        cur = torch.cuda.current_stream(self.device)
        side.wait_stream(cur)
        with torch.cuda.stream(side):
            h = _stream_handle(side)
            check(lib().apm_graph_begin(self._ctx, h), "apm_graph_begin")
            try:
                fn()
            finally:
                gid = ctypes.c_int32(-1)
                rc = lib().apm_graph_end(self._ctx, h, ctypes.byref(gid))
            check(rc, "apm_graph_end")
        cur.wait_stream(side)
        return Graph(self, int(gid.value))

    def set_grid_batching(self, batched):
        """True (default): one launch per FFT pass (and for the accelerations)
        over all grids of a level; False: one launch sequence per grid, the
        plain per-grid baseline.  Results are bit-identical."""
        check(lib().apm_set_grid_batching(self._ctx, 1 if batched else 0), "apm_set_grid_batching")

    def set_deposit_tiles(self, on):
        """True: while a particle order is current, the deposits visit the
        particles in it and gather each CTA's charges in shared-memory tiles
        (bit-identical; pays where many particles share cells).  Default off."""
        check(lib().apm_set_deposit_tiles(self._ctx, 1 if on else 0), "apm_set_deposit_tiles")

    def fft_shapes(self, level):
        sh = ApmFftShapes()
        check(lib().apm_get_fft_shapes(self._ctx, level, ctypes.byref(sh)), "apm_get_fft_shapes")
        return {"budget": list(sh.budget), "threads": list(sh.threads), "plan": list(sh.plan),
                "max_radix": int(sh.max_radix), "packing": int(sh.packing)}

    def set_fft_shapes(self, level, shapes):
        """Sets a level's shapes; keys missing from `shapes` keep their current
        values (plan, max_radix and packing may be left out)."""
        cur = self.fft_shapes(level)
        sh = ApmFftShapes()
        for i in range(5):
            sh.budget[i] = int(shapes["budget"][i])
            sh.threads[i] = int(shapes["threads"][i])
            sh.plan[i] = int(shapes.get("plan", cur["plan"])[i])
        sh.max_radix = int(shapes.get("max_radix", cur["max_radix"]))
        sh.packing = int(shapes.get("packing", cur["packing"]))
        check(lib().apm_set_fft_shapes(self._ctx, level, ctypes.byref(sh)), "apm_set_fft_shapes")

    def pass_kernels(self, level):
        """Per FFT pass (x fwd, y fwd, z, y inv, x inv), the kernel each grid of
        the level runs (in level_grids[level] order): 0 runtime plan, 1
        compile-time plan, 2 fused plane kernel (x and y passes together), 3
        none (done by the fused kernel)."""
        n = len(self.level_grids[level])
        out = []
        for q in range(5):
            kinds = (ctypes.c_int32 * n)()
            check(lib().apm_get_pass_kernels(self._ctx, level, q, kinds, n), "apm_get_pass_kernels")
            out.append(list(kinds))
        return out

    def shape_key(self, level):
        """Autotuner cache key of a level: GPU name, precision and every grid's
        FFT lengths, GMF box and window (what the pass shapes depend on)."""
        grids = sorted((tuple(self.info[i]["fft"]), tuple(self.info[i]["gmf"]),
                        tuple(self.info[i]["phi_short"])) for i in self.level_grids[level])
        return json.dumps([torch.cuda.get_device_name(self.device), self.precision, grids])

    def autotune(self, particles, half_dt, bufs, gas=None, levels=None, cache=None, stream=None):
        """Picks the FFT pass shapes of every level: from the JSON file `cache`
        (default: the APM_TUNE_CACHE environment variable, if set) when it holds
        this GPU, precision and level shape; otherwise by one step whose solves
        run the library's autotuner (apm_autotune_level), after which the file
        is updated.  Returns {level: shapes}."""
        if cache is None:
            cache = os.environ.get("APM_TUNE_CACHE") or None
        levs = list(range(self.n_levels) if levels is None else levels)
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
        keys = {lev: self.shape_key(lev) for lev in levs}
        if all(k in table for k in keys.values()):
            for lev in levs:
                self.set_fft_shapes(lev, table[keys[lev]])
        else:
            self.step(particles, half_dt, bufs, None, gas=gas, levels=levels, stream=stream, tune=True)
            for lev in levs:
                table[keys[lev]] = self.fft_shapes(lev)
            if cache:
                tmp = cache + ".tmp"
                with open(tmp, "w") as f:
                    json.dump(table, f, indent=1)
                os.replace(tmp, cache)
        return {lev: self.fft_shapes(lev) for lev in levs}

    def accel(self, level, phis, phi, acc, parent_phi=None, parent_acc=None, stream=None):
        pp = None if parent_phi is None else ptr_array([_ptr(t) for t in parent_phi])
        pa = None if parent_acc is None else ptr_array([_ptr(t) for t in parent_acc])
        check(lib().apm_accel(self._ctx, level, ptr_array([_ptr(t) for t in phis]), pp, pa,
                              ptr_array([_ptr(t) for t in phi]), ptr_array([_ptr(t) for t in acc]),
                              _stream_handle(stream)), "apm_accel")

    def interp(self, level, acc, particles, half_dt, out, stream=None):
        P = particles if isinstance(particles, Particles) else Particles(particles)
        check(lib().apm_interp(self._ctx, level, ptr_array([_ptr(t) for t in acc]),
                               ctypes.byref(P.c), float(half_dt), out.data_ptr(),
                               _stream_handle(stream)), "apm_interp")

    def kick_drift(self, particles, acc, dt, stream=None):
        """apm_kick_drift: one leapfrog step in place, acc (3, n) evaluated at
        the half-step drifted positions (step with half_dt = dt / 2)."""
        P = particles if isinstance(particles, Particles) else Particles(particles)
        check_field(acc, (3, P.n), self.dtype, self.device, "accelerations")
        for k in ("x", "y", "z", "vx", "vy", "vz"):
            check_field(P.t[k], (P.n,), torch.float64, self.device, f"particle array {k}")
        t = P.t
        check(lib().apm_kick_drift(self._ctx, P.n, t["x"].data_ptr(), t["y"].data_ptr(), t["z"].data_ptr(),
                                   t["vx"].data_ptr(), t["vy"].data_ptr(), t["vz"].data_ptr(),
                                   acc.data_ptr(), float(dt), _stream_handle(stream)), "apm_kick_drift")

    def evolve(self, particles, dt, steps, bufs, pacc, gas=None, callback=None, stream=None,
               graph=False):
        """`steps` timesteps without subcycling: each solves the hierarchy at
        the half-step drifted positions (half_dt = dt / 2) and applies
        apm_kick_drift.  callback(k, particles, pacc), if given, runs after
        step k (k = 1 .. steps).  graph: after the first step (eager), one
        step is captured as a CUDA graph and replayed for the others, which
        removes the per-launch host cost (the same launches, the same
        results)."""
        P = particles if isinstance(particles, Particles) else Particles(particles)
        g = None
        for k in range(1, steps + 1):
            if g is not None:
                g.replay()
            else:
                self.step(P, 0.5 * dt, bufs, pacc, gas=gas, stream=stream)
                self.kick_drift(P, pacc, dt, stream)
                if graph and k < steps:
                    def one():
                        self.step(P, 0.5 * dt, bufs, pacc, gas=gas)
                        self.kick_drift(P, pacc, dt)
                    g = self.capture(one)
            if callback is not None:
                callback(k, P, pacc)

    def profile(self, on, capacity=65536):
        """Turns kernel tracing on (event pool of `capacity` launches) or off."""
        check(lib().apm_profile_enable(self._ctx, 1 if on else 0, int(capacity)), "apm_profile_enable")

    def profile_read(self):
        """{kernel name: (launches, total device ms)} since tracing was enabled."""
        L = lib()
        out = {}
        for k in range(L.apm_kernel_count()):
            n = ctypes.c_int64()
            ms = ctypes.c_double()
            check(L.apm_profile_read(self._ctx, k, ctypes.byref(n), ctypes.byref(ms)), "apm_profile_read")
            out[L.apm_kernel_name(k).decode()] = (int(n.value), float(ms.value))
        return out

    def sync_status(self, stream=None):
        check(lib().apm_sync_status(self._ctx, _stream_handle(stream)), "apm_sync_status")

    # ------------------------------------------------------------------ one solve
    def step(self, particles, half_dt, bufs, pacc, gas=None, levels=None, stream=None, tune=False,
             batched=True):
        """One APM solve over the hierarchy (Sec. 2, 2.2), levels top-down:
        deposit -> solve -> accel per level, then interpolation on every level.
        bufs: from alloc_all(); pacc: (3, n) tensor of the context precision, or
        None to stop after the cell accelerations; gas: None or a list with one
        device density tensor (or None) per grid; tune: solve through the
        autotuner; batched: deposit and interpolate every level in one call each
        (apm_deposit_all / apm_interp_all, bit-identical to the per-level calls)
        when all levels are stepped."""
        P = particles if isinstance(particles, Particles) else Particles(particles)
        if pacc is not None:
            check_field(pacc, (3, P.n), self.dtype, self.device, "particle accelerations")
        if gas is not None:
            if len(gas) != len(self.grids):
                raise ValueError(f"gas has {len(gas)} entries, the hierarchy {len(self.grids)} grids")
            for gi, g in enumerate(gas):
                if g is not None:
                    check_field(g, tuple(self.grids[gi][3])[::-1], torch.float64, self.device, f"gas of grid {gi}")
        levs = range(self.n_levels) if levels is None else levels
        whole = batched and (levels is None or list(levels) == list(range(self.n_levels)))
        if 0 < P.n <= getattr(self, "order_capacity", 0):
            self.order_particles(P, half_dt, stream)
        if whole:   # every level: one pass over the particles (apm_deposit_all)
            self.deposit_all(P, half_dt, self._per_grid(bufs, "gmf"), gas, stream)
        for lev in levs:
            b = bufs[lev]
            ids = self.level_grids[lev]
            if not whole:
                g = None if gas is None else [gas[i] for i in ids]
                pg = None
                if gas is not None and lev > 0:
                    pg = [gas[i] for i in self.level_grids[lev - 1]]
                    if all(t is None for t in pg):
                        pg = None
                if g is not None and all(t is None for t in g):
                    g = None
                self.deposit(lev, P, half_dt, b["gmf"], g, pg, stream)
            if tune:
                self.autotune_level(lev, b["gmf"], b["phis"], stream)
            else:
                self.solve_level(lev, b["gmf"], b["phis"], stream)
            if lev > 0 and (levels is None or (lev - 1) in levs):
                self.accel(lev, b["phis"], b["phi"], b["acc"], bufs[lev - 1]["phi"],
                           bufs[lev - 1]["acc"], stream)
            else:
                self.accel(lev, b["phis"], b["phi"], b["acc"], stream=stream)
        if pacc is None:
            return
        if whole:
            self.interp_all(self._per_grid(bufs, "acc"), P, half_dt, pacc, stream)
            return
        for lev in levs:
            self.interp(lev, bufs[lev]["acc"], P, half_dt, pacc, stream)


class Graph:
    """A library-owned CUDA graph of a Solver (Solver.capture)."""

    def __init__(self, solver, gid):
        self.s = solver
        self.gid = gid

    def replay(self, stream=None):
        check(lib().apm_graph_launch(self.s._ctx, self.gid, _stream_handle(stream)), "apm_graph_launch")

    def destroy(self):
        if self.gid >= 0 and getattr(self.s, "_ctx", None):
            check(lib().apm_graph_destroy(self.s._ctx, self.gid), "apm_graph_destroy")
        self.gid = -1


class StepPipeline:
    """End-to-end solves from pinned host particles to host accelerations, with
    the copies overlapped: two device particle/acceleration buffer sets, each
    with its own captured solve (a library-owned CUDA graph), an upload stream
    that copies step k+1's particles in while step k solves, and a download
    stream that copies step k's accelerations out once it has solved (one
    stream per direction, so that a full-duplex host link runs both at once).
    Every step still copies all of its inputs in and its result out.

    solver, bufs: a Solver and its alloc_all() buffers (shared by both sets);
    host: dict of pinned float64 host arrays (PARTICLE_KEYS); the rest as for
    Solver.step.  run(steps, inputs=None, outputs=None): inputs(k) -> host dict
    of step k (default: `host` every step); outputs(k) -> pinned host (3, n)
    tensor of the solver's precision that receives step k's accelerations
    (default: two alternating buffers)."""

    def __init__(self, solver, bufs, host, half_dt, gas=None, levels=None):
        self.s = solver
        self.host = host
        dev = solver.device
        self.n = int(host["x"].numel())
        self.sets = []
        for _ in range(2):
            P = Particles({k: torch.empty_like(host[k], device=dev) for k in PARTICLE_KEYS})
            pacc = torch.zeros((3, self.n), dtype=solver.dtype, device=dev)
            self.sets.append((P, pacc))
        self.hout = [torch.empty((3, self.n), dtype=solver.dtype).pin_memory() for _ in range(2)]
        self.copy = torch.cuda.Stream(device=dev)
        self.copy_out = torch.cuda.Stream(device=dev)
        self.graphs = []
        for P, pacc in self.sets:
            for k in PARTICLE_KEYS:
                P.t[k].copy_(host[k])
            solver.step(P, half_dt, bufs, pacc, gas=gas, levels=levels)     # warm, outside capture
            self.graphs.append(solver.capture(
                lambda P=P, pacc=pacc: solver.step(P, half_dt, bufs, pacc, gas=gas, levels=levels)))
        torch.cuda.synchronize(dev)
        solver.sync_status()

    def bytes_per_step(self):
        h2d = sum(self.host[k].numel() * self.host[k].element_size() for k in PARTICLE_KEYS)
        return h2d, self.hout[0].numel() * self.hout[0].element_size()

    def run(self, steps, inputs=None, outputs=None):
        comp = torch.cuda.current_stream(self.s.device)
        cp = self.copy
        ev_in = [torch.cuda.Event(), torch.cuda.Event()]
        ev_done = [torch.cuda.Event(), torch.cuda.Event()]
        ev_out = [torch.cuda.Event(), torch.cuda.Event()]

        def upload(k):
            P = self.sets[k % 2][0]
            src = self.host if inputs is None else inputs(k)
            with torch.cuda.stream(cp):
                for key in PARTICLE_KEYS:
                    P.t[key].copy_(src[key], non_blocking=True)
                ev_in[k % 2].record(cp)

        dn = self.copy_out
        cp.wait_stream(comp)
        dn.wait_stream(comp)
        if steps > 0:
            upload(0)
        for k in range(steps):
            b = k % 2
            comp.wait_event(ev_in[b])
            if k >= 2:
                comp.wait_event(ev_out[b])         # step k-2's download of this set is done
            self.graphs[b].replay()
            ev_done[b].record(comp)
            if k + 1 < steps:
                if k >= 1:
                    cp.wait_event(ev_done[1 - b])      # set 1-b is free once step k-1 has solved
                upload(k + 1)
            with torch.cuda.stream(dn):
                dn.wait_event(ev_done[b])
                dst = self.hout[b] if outputs is None else outputs(k)
                dst.copy_(self.sets[b][1], non_blocking=True)
                ev_out[b].record(dn)
        comp.wait_stream(cp)
        comp.wait_stream(dn)
