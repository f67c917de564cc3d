"""Accuracy studies of the APM solve, run on the GPU through the library:

* padding: the refined level's accelerations against border factors around the
  paper's 0.65 R a / delta extra cells (Sec. 2.2);
* softening: the mesh force against the S2 reference force for a / delta
  around the paper's 3.4 (Sec. 2.2, after HE);
* the isolated root's k-space optimal correction on and off, and the three
  gradient operators (Sec. 2.2), by the same measure;
* the force decomposition of Sec. 2.2 Fig. 2: the radial short-range force each
  level adds around a particle at the centre of the Fig. 1 hierarchy (32^3
  root), against the analytical 1/r^2.

`python -m paper_1410_0010_gb300.accuracy` prints every table (FP64).  The
reference force is this module's own quadrature of the pair force of two S2
spheres from Eq. S2k: F(r) = (2/pi) int S^2(k a/2) [sin(kr)/(kr^2) - cos(kr)/r] dk.
"""
import argparse
import json
import math

import numpy as np
import torch
from scipy import integrate

from .solver import Particles, Solver

FIG1_BOUNDS = [(0.1875, 0.8125), (0.3125, 0.6875), (0.40625, 0.59375)]


def s_hat(eta):
    """Eq. S2k: 12/eta^4 (2 - 2 cos eta - eta sin eta), its series below 0.1."""
    if eta < 0.1:
        e2 = eta * eta
        return 1.0 - e2 / 15.0 + e2 * e2 / 560.0
    return 12.0 / eta ** 4 * (2.0 - 2.0 * math.cos(eta) - eta * math.sin(eta))


def s2_pair_force(r, a):
    """Attraction between two unit S2 spheres of diameter a at distance r (G = 1);
    exactly 1/r^2 once the spheres no longer overlap (r >= a)."""
    if r >= a:
        return 1.0 / (r * r)
    f = lambda k: s_hat(k * a / 2) ** 2 * (math.sin(k * r) / (k * r * r) - math.cos(k * r) / r)
    kmax = 400.0 / a
    val, _ = integrate.quad(f, 1e-12, kmax, limit=2000)
    return 2.0 / math.pi * val


def _grids_from_bounds(root, bounds):
    out = [(0, -1, (0, 0, 0), (root,) * 3)]
    for lev, (lo, hi) in enumerate(bounds, start=1):
        n = root * 2 ** lev
        s, e = int(round(lo * n)), int(round(hi * n))
        out.append((lev, lev - 1, (s,) * 3, (e - s,) * 3))
    return out


def _particles(pos, m, device):
    n = pos.shape[1]
    z = np.zeros(n)
    arrs = dict(x=pos[0], y=pos[1], z=pos[2], vx=z, vy=z, vz=z, m=np.asarray(m, float))
    return Particles({k: torch.as_tensor(np.ascontiguousarray(v, dtype=np.float64), device=device)
                      for k, v in arrs.items()})


def _solve(grids, P, n, device, precision="fp64", **cfg):
    s = Solver(grids, precision=precision, device=device, **cfg)
    bufs = s.alloc_all()
    pacc = torch.zeros((3, n), dtype=s.dtype, device=torch.device("cuda", device))
    s.step(P, 0.0, bufs, pacc)
    s.sync_status()
    return s, bufs, pacc


def padding_sweep(pads=(0.15, 0.3, 0.45, 0.65, 0.8, 1.0), ref_pad=1.3, device=0, seed=3):
    """Relative L2 difference of a refined grid's accelerations (16^3 level-1
    grid at the centre of a 32^3 isolated root, 3000 particles over the level
    and its surroundings) from those with a generous border (ref_pad)."""
    rng = np.random.default_rng(seed)
    grids = [(0, -1, (0, 0, 0), (32, 32, 32)), (1, 0, (24, 24, 24), (16, 16, 16))]
    n = 3000
    P = _particles(0.3 + 0.4 * rng.random((3, n)), np.full(n, 1.0 / n), torch.device("cuda", device))
    acc = {}
    info = {}
    for pad in tuple(pads) + (ref_pad,):
        s, bufs, _ = _solve(grids, P, n, device, pad_factor=pad)
        acc[pad] = bufs[1]["acc"][0][:, 1:-1, 1:-1, 1:-1].double().cpu().numpy()
        info[pad] = (s.info[1]["border"], s.info[1]["fft"][0])
        s.close()
    ref = acc[ref_pad]
    return [{"pad_factor": p, "border": info[p][0], "fft": info[p][1],
             "rel_l2": float(np.linalg.norm(acc[p] - ref) / np.linalg.norm(ref))} for p in pads]


def force_errors(root=32, device=0, seed=5, centres=8, per_centre=400, precision="fp64", **cfg):
    """Radial and tangential force of a unit mass on massless particles at
    r in [0.5, 10] root cells (log-uniform, random directions) around `centres`
    random sub-cell positions of an isolated root, against the S2 reference
    force: mean and rms of the relative radial error inside (r < 2a) and
    outside the softening, and the rms tangential force relative to it."""
    rng = np.random.default_rng(seed)
    d = 1.0 / root
    a = cfg.get("a_over_dx", 3.4) * d
    grids = [(0, -1, (0, 0, 0), (root,) * 3)]
    rows = {"near": [], "far": []}
    dev = torch.device("cuda", device)
    ref_cache = {}
    for _ in range(centres):
        c = 0.5 + rng.random(3) * d
        r = d * 10 ** rng.uniform(math.log10(0.5), 1.0, per_centre)
        u = rng.normal(size=(3, per_centre))
        u /= np.linalg.norm(u, axis=0)
        pos = np.concatenate([c[:, None], c[:, None] + r * u], axis=1)
        m = np.r_[1.0, np.zeros(per_centre)]
        s, _, pacc = _solve(grids, _particles(pos, m, dev), per_centre + 1, device, precision, **cfg)
        s.close()
        acc = pacc[:, 1:].double().cpu().numpy()
        fr = -(acc * u).sum(0)
        ft = np.linalg.norm(acc + fr[None, :] * u, axis=0)
        for k in range(per_centre):
            key = round(float(r[k]), 12)
            if key not in ref_cache:
                ref_cache[key] = s2_pair_force(float(r[k]), a)
            f0 = ref_cache[key]
            rows["near" if r[k] < 2 * a else "far"].append(((fr[k] - f0) / f0, ft[k] / f0))
    out = {}
    for key, v in rows.items():
        if not v:       # no sample on this side of 2a (large a)
            out[key] = {"mean": None, "rms": None, "tangential_rms": None, "n": 0}
            continue
        v = np.array(v)
        out[key] = {"mean": float(v[:, 0].mean()), "rms": float(np.sqrt((v[:, 0] ** 2).mean())),
                    "tangential_rms": float(np.sqrt((v[:, 1] ** 2).mean())), "n": int(len(v))}
    return out


def softening_sweep(values=(2.0, 2.5, 3.0, 3.4, 4.0, 5.0), device=0):
    return [{"a_over_dx": v, **force_errors(device=device, a_over_dx=v)} for v in values]


def correction_and_gradients(device=0):
    rows = []
    for corr in (True, False):
        for grad in ("fd2", "fd4", "spectral"):
            rows.append({"root_correction": corr, "gradient": grad,
                         **force_errors(device=device, root_correction=corr, gradient=grad)})
    return rows


def force_decomposition(root=32, bins=16, device=0, precision="fp64"):
    """Sec. 2.2 Fig. 2: a unit mass at the centre of the Fig. 1 hierarchy; for
    each level the radial short-range acceleration its own solve adds (its
    potential differenced without the parent carry), averaged in log-r bins
    over that level's interior cells, and the total (from the finest level
    holding the cell) as its ratio to 1/r^2 averaged over the bin's cells."""
    dev = torch.device("cuda", device)
    grids = _grids_from_bounds(root, FIG1_BOUNDS)
    x0 = 0.5 + 0.3 / (root * 8)           # inside the finest level, off the cell centres
    P = _particles(np.array([[x0], [x0], [x0]]), [1.0], dev)
    s, bufs, _ = _solve(grids, P, 1, device, precision)
    edges = np.logspace(math.log10(0.5 / (root * 8)), math.log10(0.5), bins + 1)
    table = {"r": np.sqrt(edges[:-1] * edges[1:]).tolist(), "newton": [], "total_ratio": [], "levels": [],
             "a": [], "delta": []}
    total_sum = np.zeros(bins)
    total_cnt = np.zeros(bins)
    for lev in range(s.n_levels):
        g = s.grids[s.level_grids[lev][0]]
        b = bufs[lev]
        phi = [torch.empty_like(t) for t in b["phi"]]
        acc = [torch.empty_like(t) for t in b["acc"]]
        s.accel(lev, b["phis"], phi, acc)         # no parent term: this level's own part
        torch.cuda.synchronize()
        own = acc[0][:, 1:-1, 1:-1, 1:-1].double().cpu().numpy()
        full = b["acc"][0][:, 1:-1, 1:-1, 1:-1].double().cpu().numpy()
        d = s.info[s.level_grids[lev][0]]["delta"]
        idx = [(np.arange(g[3][j]) + g[2][j] + 0.5) * d for j in range(3)]
        zz, yy, xx = np.meshgrid(idx[2], idx[1], idx[0], indexing="ij")
        rv = np.stack([xx - x0, yy - x0, zz - x0])
        r = np.linalg.norm(rv, axis=0)
        fr_own = -(own * rv).sum(0) / np.maximum(r, 1e-300)
        fr_full = -(full * rv).sum(0) / np.maximum(r, 1e-300)
        # the finest level covering a cell gives the total there
        mask = np.ones_like(r, dtype=bool)
        if lev + 1 < s.n_levels:
            gn = s.grids[s.level_grids[lev + 1][0]]
            lo = np.array(gn[2]) * (d / 2)
            hi = lo + np.array(gn[3]) * (d / 2)
            inside = ((xx >= lo[0]) & (xx < hi[0]) & (yy >= lo[1]) & (yy < hi[1]) &
                      (zz >= lo[2]) & (zz < hi[2]))
            mask &= ~inside
        which = np.digitize(r, edges) - 1
        mean_own = []
        for k in range(bins):
            sel = which == k
            mean_own.append(float(fr_own[sel].mean()) if sel.any() else None)
            selt = sel & mask
            total_sum[k] += (fr_full[selt] * r[selt] ** 2).sum()
            total_cnt[k] += selt.sum()
        table["levels"].append(mean_own)
        table["a"].append(3.4 * float(d))
        table["delta"].append(float(d))
    s.close()
    table["total_ratio"] = [float(total_sum[k] / total_cnt[k]) if total_cnt[k] else None for k in range(bins)]
    table["newton"] = [1.0 / rr ** 2 for rr in table["r"]]
    return table


def _fmt(v, f="{:.3e}"):
    return "-" if v is None else f.format(v)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--json", help="also write every table to this file")
    args = ap.parse_args(argv)
    out = {"padding": padding_sweep(device=args.device),
           "softening": softening_sweep(device=args.device),
           "correction_and_gradients": correction_and_gradients(device=args.device),
           "decomposition": force_decomposition(device=args.device)}
    print("## Padding (level-1 accelerations vs pad 1.3)\n")
    print("| pad factor | B | M | rel L2 |\n|---|---|---|---|")
    for r in out["padding"]:
        print(f"| {r['pad_factor']} | {r['border']} | {r['fft']} | {r['rel_l2']:.2e} |")
    print("\n## Softening (radial error vs the S2 reference force; r < 2a and r >= 2a)\n")
    print("| a/delta | near mean | near rms | near tangential | far mean | far rms | far tangential |")
    print("|---|---|---|---|---|---|---|")
    for r in out["softening"]:
        n, f = r["near"], r["far"]
        print(f"| {r['a_over_dx']} | {_fmt(n['mean'], '{:+.4f}')} | {_fmt(n['rms'], '{:.4f}')} | "
              f"{_fmt(n['tangential_rms'], '{:.4f}')} | {_fmt(f['mean'], '{:+.4f}')} | "
              f"{_fmt(f['rms'], '{:.4f}')} | {_fmt(f['tangential_rms'], '{:.4f}')} |")
    print("\n## Root correction and gradient operator (a/delta = 3.4)\n")
    print("| correction | gradient | near mean | near rms | far mean | far rms | far tangential |")
    print("|---|---|---|---|---|---|---|")
    for r in out["correction_and_gradients"]:
        n, f = r["near"], r["far"]
        print(f"| {'on' if r['root_correction'] else 'off'} | {r['gradient']} | {n['mean']:+.4f} | "
              f"{n['rms']:.4f} | {f['mean']:+.4f} | {f['rms']:.4f} | {f['tangential_rms']:.4f} |")
    t = out["decomposition"]
    print("\n## Force decomposition (Fig. 2): mean radial force each level adds, 1/r^2, total / (1/r^2)\n")
    head = " | ".join(f"level {k} (a = {a:.4f})" for k, a in enumerate(t["a"]))
    print(f"| r | {head} | 1/r^2 | total ratio |\n|---|" + "---|" * (len(t["levels"]) + 2))
    for k, r in enumerate(t["r"]):
        cols = " | ".join(_fmt(lv[k]) for lv in t["levels"])
        print(f"| {r:.4f} | {cols} | {t['newton'][k]:.3e} | {_fmt(t['total_ratio'][k], '{:.3f}')} |")
    if args.json:
        with open(args.json, "w") as f:
            json.dump(out, f, indent=1)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
