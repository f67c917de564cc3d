"""bench.py's DRAM-traffic file from an ncu --csv capture (host logic): kernel
names map to the bench's labels (the column passes by their template
arguments), bytes are summed per launch over read and write, averaged per
kernel, scaled to the full workload, and stamped with the sources' hash."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_kernel_names_map_to_labels():
    b = _bench()
    col = "void unnamed>::k_col<float, {}, {}, 256>(const GridDev *, const Chunk *, int)"
    assert b.ncu_label(col.format(1, 0)) == "fft_y_fwd"
    assert b.ncu_label(col.format(2, 1)) == "fft_z_green"
    assert b.ncu_label(col.format(1, 2)) == "fft_y_inv"
    assert b.ncu_label("void unnamed>::k_xf<float, 128>(const GridDev *)") == "fft_x_fwd"
    assert b.ncu_label("void unnamed>::k_xi<double, 256>(const GridDev *)") == "fft_x_inv"
    assert b.ncu_label("unnamed>::k_gas_init(LevelDev, const GridDev *)") == "gas_init"
    assert b.ncu_label("unnamed>::k_deposit_levels(const LevelDev *, int)") == "tsc_deposit"
    assert b.ncu_label("void unnamed>::k_accel<float>(LevelDev, const GridDev *)") == "accel_carry"
    assert b.ncu_label("void unnamed>::k_interp_levels<float>(const LevelDev *, int)") == "tsc_interp"
    assert b.ncu_label("void at::native::vectorized_elementwise_kernel<4>(int)") is None
    fast = "void apm::<unnamed>::k_col_fast<apm::<unnamed>::FastPlan<15, 10, 1>, {}, {}, 16, 80>(const GridDev *)"
    assert b.ncu_label(fast.format(1, 0)) == "fft_y_fwd"
    assert b.ncu_label(fast.format(2, 1)) == "fft_z_green"
    assert b.ncu_label(fast.format(1, 2)) == "fft_y_inv"
    plan = "apm::<unnamed>::FastPlan<8, 8, 8>, "
    assert b.ncu_label(f"void apm::<unnamed>::k_xf_fast<{plan}16, 256>(const GridDev *)") == "fft_x_fwd"
    assert b.ncu_label(f"void apm::<unnamed>::k_xi_fast<{plan}16, 256>(const GridDev *)") == "fft_x_inv"
    assert b.ncu_label(f"void apm::<unnamed>::k_xy_fast<{plan}384>(const GridDev *)") == "fft_x_fwd"
    assert b.ncu_label(f"void apm::<unnamed>::k_yx_fast<{plan}384>(const GridDev *)") == "fft_x_inv"
    assert b.ncu_label("apm::<unnamed>::k_order_bins(LevelDev, Particles)") is None
    # ncu's CSV writes the anonymous namespace as "unnamed>::"
    assert b.ncu_label("void unnamed>::k_xf_fast<unnamed>::FastPlan<16, 16, 1>, 16, 256>(const GridDev *)") \
        == "fft_x_fwd"
    assert b.ncu_label("void unnamed>::k_col_fast<unnamed>::FastPlan<15, 10, 1>, 2, 1, 16, 80>(int)") \
        == "fft_z_green"


def test_write_traffic_averages_scales_and_stamps(tmp_path, monkeypatch):
    b = _bench()
    head = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
            '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"')
    rows = []

    def add(i, name, metric, unit, value):
        rows.append(f'"{i}","1","python","h","{name}","1","7","(256, 1, 1)","(8, 1, 1)","0","10.3","m",'
                    f'"{metric}","{unit}","{value}"')
    acc = "void unnamed>::k_accel<float>(LevelDev, const GridDev *)"
    add(0, acc, "dram__bytes_read.sum", "Mbyte", "100")
    add(0, acc, "dram__bytes_write.sum", "Mbyte", "200")
    add(0, acc, "gpu__time_duration.sum", "usecond", "50")
    add(1, acc, "dram__bytes_read.sum", "Mbyte", "120")
    add(1, acc, "dram__bytes_write.sum", "Kbyte", "180,000")
    add(2, "unnamed>::k_gas_init(LevelDev)", "dram__bytes_write.sum", "byte", "1000")
    csv_path = tmp_path / "t.csv"
    csv_path.write_text("==PROF== noise\n" + head + "\n" + "\n".join(rows) + "\n")
    written = {}

    real_open = open

    def fake_open(path, mode="r", *a, **k):
        if str(path).endswith(os.path.join("profiles", "traffic.json")) and "w" in mode:
            class W:
                def __enter__(self_):
                    return self_

                def __exit__(self_, *e):
                    return False

                def write(self_, s):
                    written.setdefault("s", "")
                    written["s"] += s
            return W()
        return real_open(path, mode, *a, **k)

    monkeypatch.setattr("builtins.open", fake_open)
    b.write_traffic(str(csv_path))
    doc = json.loads(written["s"])
    import apm_inputs as W
    small, full = W.NAMES["c5s"], W.NAMES["c5"]
    assert W.config_isolated_root32().name == W.NAMES["c1"]
    per = doc["per_launch_bytes"]
    assert per[f"{small}:accel_carry"] == 300_000_000          # (300 MB + 300 MB) / 2 launches
    assert per[f"{full}:accel_carry"] == 8 * 300_000_000
    assert per[f"{small}:gas_init"] == 1000
    assert doc["source_sha256"] == b.kernel_source_hash()


def test_algorithmic_bytes_per_operator():
    """bench.py's algorithmic bytes for one refined grid: the spectral path
    counts its z, y-inverse and x-inverse passes four times and reads four
    windows in the acceleration kernel; the four-point one differences a
    wider window."""
    import types

    import numpy as np
    b = _bench()
    N, B = 8, 5
    G = (N + 2 * B,) * 3
    M = (30, 30, 30)
    E = (N + 2,) * 3

    def solver(h, comps, fused=False):
        W = (N + 2 * h,) * 3
        info = [dict(gmf=G, fft=M, phi_short=W, field=E, comps=comps)]
        kinds = [[2], [3], [1], [3], [2]] if fused else [[1]] * 5
        return types.SimpleNamespace(level_grids=[[0]], info=info, n_levels=1,
                                     pass_kernels=lambda lev: kinds), W
    w = types.SimpleNamespace(n_particles=0, gas=None, grids=[types.SimpleNamespace(dims=(N, N, N))])
    csz, rsz = 8, 4
    Hx = M[0] // 2 + 1
    s2, W2 = solver(2, 1)
    s4, W4 = solver(3, 1)
    ss, Ws = solver(2, 4)
    a2 = b.algorithmic_bytes(s2, w, [0], csz, rsz, True)
    a4 = b.algorithmic_bytes(s4, w, [0], csz, rsz, True)
    asp = b.algorithmic_bytes(ss, w, [0], csz, rsz, True)
    ec = int(np.prod(E))
    assert a2["accel_carry"] == rsz * int(np.prod(W2)) + 4 * rsz * ec
    assert a4["accel_carry"] == rsz * int(np.prod(W4)) + 4 * rsz * ec
    assert asp["accel_carry"] == 8 * rsz * ec
    for k in ("fft_z_green", "fft_y_inv", "fft_x_inv"):
        assert asp[k] == 4 * a2[k], k
    for k in ("gas_init", "tsc_deposit", "fft_x_fwd", "fft_y_fwd"):
        assert asp[k] == a2[k] == a4[k], k
    assert a2["fft_x_fwd"] == 8 * int(np.prod(G)) + csz * G[1] * G[2] * Hx
    # the fused plane kernels: the x spectrum between the x and y passes (and
    # the y inverse's output between the y and x inverse) never reaches HBM
    sf, Wf = solver(2, 1, fused=True)
    af = b.algorithmic_bytes(sf, w, [0], csz, rsz, True)
    assert af["fft_y_fwd"] == af["fft_y_inv"] == 0
    assert af["fft_x_fwd"] == 8 * int(np.prod(G)) + csz * G[2] * M[1] * Hx
    assert af["fft_x_inv"] == csz * Wf[2] * M[1] * Hx + rsz * int(np.prod(Wf))
    assert af["fft_z_green"] == a2["fft_z_green"]
    assert af["fft_x_fwd"] + af["fft_y_fwd"] < a2["fft_x_fwd"] + a2["fft_y_fwd"]


def test_interp_field_bytes_counts_each_read_cell_once():
    """The interpolation's field bytes: 27 cells per particle on its owner grid
    (the finest solved grid holding it), each cell once, three components."""
    import types

    import numpy as np
    import torch
    b = _bench()
    from apm_inputs import GridDesc
    grids = [GridDesc(0, -1, (0, 0, 0), (8, 8, 8)), GridDesc(1, 0, (4, 4, 4), (6, 6, 6))]
    w = types.SimpleNamespace(grids=grids, periodic=False)

    def parts(pos):
        pos = np.asarray(pos, dtype=np.float64).T
        d = {k: torch.tensor(pos[j]) for j, k in enumerate("xyz")}
        d.update({"v" + k: torch.zeros(pos.shape[1], dtype=torch.float64) for k in "xyz"})
        return d
    one = (0.1, 0.1, 0.1)                        # root cell 0: its cloud reaches cell -1 of the window
    same = (0.11, 0.12, 0.1)                     # the same root cell: no new cells
    near = (0.26, 0.1, 0.1)                      # root cell 2: its cloud shares x = 1 with the first
    child = (0.45, 0.45, 0.45)                   # level-1 cell 7, inside the child: owned by it
    assert b.interp_field_bytes(w, [0, 1], parts([one]), 0.0, 4) == 27 * 12
    assert b.interp_field_bytes(w, [0, 1], parts([one, same]), 0.0, 4) == 27 * 12
    assert b.interp_field_bytes(w, [0, 1], parts([one, near]), 0.0, 4) == (27 + 18) * 12
    assert b.interp_field_bytes(w, [0, 1], parts([one, child]), 0.0, 4) == 2 * 27 * 12
    # a drift of one root cell moves the cloud
    d = parts([one])
    d["vx"][:] = 1.0
    assert b.interp_field_bytes(w, [0, 1], d, 0.125, 4) == 27 * 12
    # only the solved levels own particles
    assert b.interp_field_bytes(w, [1], parts([one, child]), 0.0, 4) == 27 * 12
