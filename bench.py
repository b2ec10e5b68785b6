"""Throughput of the CAC-LB wetting step on B300: MLUPS and fraction of the
HBM roofline.

Workload (one GPU): the static-droplet case of the paper's Sect. 3.1 at
256^3 -- walls at z = 0 and z = 255, periodic in x and y, a cap of radius 40
centred on the bottom wall, theta = 60 deg, equal densities and viscosities
(nu = 0.04), sigma = 0.02, W = 4, D = 0.02; synthetic seeded input. A step
is one full pass of the method: ghost update, collide-stream, phi update,
volume correction.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line. With N > 1 (torchrun) each rank runs an independent
replica of the workload on its own GPU (the step needs no exchange between
replicas); value is the total over ranks, timed by the slowest rank.
--impl reference times the FP64 CPU oracle on this host's cores instead.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

GRID = 256
THETA = 60.0
METRIC = "MLUPS (CAC-LB step, 256^3)"
STORE_BYTES = {"f32": 4, "f16": 2, "bf16": 2, "moments": 4}
# values stored per node for the populations: 27 populations, or the 17
# coefficients of the moment form
STORE_COMPS = {"f32": 27, "f16": 27, "bf16": 27, "moments": 17}
LB_BYTES_SOLID = 1


def lb_bytes_fluid(storage="f32"):
    """Algorithmic bytes of the collide-stream per fluid node: 27 populations
    (17 coefficients in moment form) read + written, phi read, u written
    (3 x FP32), flags read."""
    return STORE_COMPS[storage] * STORE_BYTES[storage] * 2 + 4 + 12 + 1


def step_bytes(storage="f32"):
    """Algorithmic bytes of one whole step per node: collide-stream, phi
    update (phi read, u read, phi* written, flags) 21, correction 9."""
    return lb_bytes_fluid(storage) + (4 + 12 + 4 + 1) + (4 + 4 + 1)


LB_BYTES_FLUID = lb_bytes_fluid()
STEP_BYTES = step_bytes()
L2_BYTES = 126 * 1024 * 1024


def workload(grid=GRID, theta=THETA):
    from paper_2607_25444_b300 import inputs as I
    n = grid
    p = I.base_params(n, n, n, sigma=0.02, theta_deg=theta)
    solid = I.walls_z(n, n, n)
    phi = I.droplet(n, n, n, (n / 2, n / 2, 0.5), 40.0 * grid / 256, p["width"])
    return p, solid, phi


def kernel_traffic(fluid_nodes):
    """DRAM bytes per collide-stream launch from the committed ncu summary
    (a full-size capture, in bytes per fluid node); None when the kernel
    source changed since the capture (its hash no longer matches)."""
    import hashlib
    import re
    prof = os.path.join(ROOT, "profiles", "lb_collide_pair32_static_droplet_256cube.md")
    if not os.path.exists(prof):
        return None
    text = open(prof).read()
    per = re.search(r"traffic_bytes_per_fluid_node:\s*([0-9.eE+-]+)", text)
    sha = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    if not per or not sha:
        return None
    h = hashlib.sha256()
    for f in ("lb.cu", "cacl_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2607_25444_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != sha.group(1):
        return None
    return float(per.group(1)) * fluid_nodes


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_oracle_run(steps, max_seconds=30.0):
    """FP64 oracle on the host cores, on the lower 64 layers of the same
    workload (the cap is 40 high). Returns MLUPS, cores and the sample."""
    from oracle import oracle as O
    from paper_2607_25444_b300 import inputs as I
    n, nz = GRID, 64
    p = I.base_params(n, n, nz, sigma=0.02, theta_deg=THETA)
    solid = I.walls_z(n, n, nz)
    phi = I.droplet(n, n, nz, (n / 2, n / 2, 0.5), 40.0, p["width"])
    o = O.Oracle(p)
    o.set_geometry(solid)
    o.set_fields(phi.astype(np.float64))
    done, t0 = 0, time.perf_counter()
    while done < steps:
        o.step(1)
        done += 1
        if time.perf_counter() - t0 > max_seconds:
            break
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0))
    threads = int(os.environ.get("OMP_NUM_THREADS", cores))
    return (n * n * nz * done / dt / 1e6, threads,
            f"{done} step(s) of the 256x256x64 lower slab of the 256^3 "
            f"static-droplet workload (walls z=0 and z=63), FP64, "
            f"{dt:.1f} s")


def cpu_case_time(kind, steps):
    """Seconds and node updates of the FP64 oracle on one of the paper-shaped
    cases: "c1" the 2D static droplet (128 x 64, D2Q9), "c2" the 128^3
    spreading case, "slab" the headline's 256 x 256 x 64 lower slab."""
    from oracle import oracle as O
    from paper_2607_25444_b300 import inputs as I
    if kind == "c1":
        p, solid, phi = I.static_droplet_2d(60.0)
    elif kind == "c2":
        p, solid, phi = I.spreading_128(60.0)
    else:
        n, nz = GRID, 64
        p = I.base_params(n, n, nz, sigma=0.02, theta_deg=THETA)
        solid = I.walls_z(n, n, nz)
        phi = I.droplet(n, n, nz, (n / 2, n / 2, 0.5), 40.0, p["width"])
    o = O.Oracle(p)
    o.set_geometry(solid)
    o.set_fields(phi.astype(np.float64))
    t0 = time.perf_counter()
    o.step(steps)
    return time.perf_counter() - t0, phi.size * steps


def run_cpu_extended(args):
    """The oracle on the host cores beyond the bench's bounded sample: the
    headline slab on one thread and on all threads, the 2D c1 case at its
    full length (2000 steps) and a 10-step sample of c2, each in a child
    process with its OpenMP thread count set."""
    import subprocess
    cores = len(os.sched_getaffinity(0))
    cases = [("slab", 1, 1), ("slab", 1, cores), ("c1", 2000, cores),
             ("c1", 2000, 1), ("c2", 10, cores)]
    out = []
    for kind, steps, threads in cases:
        env = dict(os.environ, OMP_NUM_THREADS=str(threads))
        code = ("import json, sys; sys.path.insert(0, %r); import bench; "
                "t, n = bench.cpu_case_time(%r, %d); print(json.dumps([t, n]))"
                % (ROOT, kind, steps))
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True,
                           text=True, check=True)
        t, n = json.loads(r.stdout.strip().splitlines()[-1])
        out.append({"case": kind, "steps": steps, "threads": threads, "seconds": t,
                    "mlups": n / t / 1e6})
    print(json.dumps({"metric": "FP64 oracle MLUPS on the host cores", "cores": cores,
                      "runs": out}), flush=True)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    steps = max(1, args.steps // 100)
    total = 0.0
    vals = []
    for _ in range(max(1, min(args.warmup, 1))):
        cpu_oracle_run(1, max_seconds=60.0)
    for _ in range(1):
        v, cores, sample = cpu_oracle_run(steps, max_seconds=60.0)
        vals.append(v)
        total += v
    v = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "static droplet 256^3 (lower 64-layer slab on "
                               "the CPU)", "grid": [GRID, GRID, GRID]},
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_lb_kernel(solver, torch, reps):
    """Average duration of one collide-stream launch: reps launches enqueued
    back to back between two CUDA events on the library's stream (torch's
    current stream)."""
    stream = torch.cuda.current_stream()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    solver.lb_collide()
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(reps):
        solver.lb_collide()
    end.record(stream)
    torch.cuda.synchronize()
    return start.elapsed_time(end) / reps / 1e3


def impact_sweep_cases(ncases=48, storage="f16", pick=None):
    """Batched impact sweep shaped like the paper's Sect. 3.3: 48 cubes with
    edges drawn from [64, 160], a drop of radius 0.2 n resting on the bottom
    wall with a downward speed set by a Weber number drawn from [1, 80],
    contact angle drawn from [120, 160] deg, density ratio 100, FP16
    storage; seeded draws (pick: indices of the draws to build)."""
    import math as _m

    from paper_2607_25444_b300 import inputs as I
    out = []
    draws = I.impact_sweep(ncases)
    for d in (draws if pick is None else [draws[i] for i in pick]):
        n = d["n"]
        p = I.base_params(n, n, n, sigma=0.003, rho_l=1.0, rho_g=0.01,
                          nu_l=0.03, nu_g=0.03, theta_deg=d["theta_deg"],
                          storage=storage)
        R = d["radius"]
        solid = I.walls_z(n, n, n)
        phi = I.droplet(n, n, n, (n / 2, n / 2, 0.5 + R + 1.0), R, p["width"])
        u = np.zeros((3,) + phi.shape, np.float32)
        u[2] = np.where(phi > 0.5, -d["u0"], 0.0)
        out.append((p, solid, phi, u))
        assert _m.isfinite(d["u0"])
    return out


def median_steps_time(solver, torch, stream, steps, repeats):
    """Median over `repeats` of the CUDA-event time of `steps` steps."""
    times = []
    for _ in range(repeats):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    return float(np.median(times))


def paper_workloads(args, torch, cacl, stream):
    """Throughput on the paper-shaped workloads other than the headline: the
    spreading case of Sect. 3.2 (128^3, cap R = 24, theta = 60 deg, density
    ratio 10, equal kinematic viscosities, sigma = 0.005) with FP32 and the
    16-bit population storage, and the orifice passage of Sect. 3.4
    (128 x 128 x 256, plate 8 thick at z = 128 with a square hole of side
    24, drop R = 20 above it, density ratio 50, Bond number 1, theta =
    60 deg) in FP32. Synthetic seeded inputs."""
    from paper_2607_25444_b300 import inputs as I
    out = {}
    steps = max(20, min(args.steps, 100))
    cases = [("spreading_128cube", I.spreading_128(60.0), ("f32", "f16", "bf16")),
             ("orifice_128x128x256", I.orifice_128x128x256(24, 60.0, 1.0), ("f32",))]
    for name, (p, solid, phi), storages in cases:
        rec = {"grid": [p["nx"], p["ny"], p["nz"]],
               "fluid_nodes": int((solid == 0).sum())}
        N = phi.size
        for st in storages:
            sv = cacl.Solver(dict(p, storage=st))
            sv.set_geometry(solid)
            sv.set_fields(phi)
            sv.step(5)
            dtv = median_steps_time(sv, torch, stream, steps, 3)
            sv.check_finite()
            sv.close()
            rec[st] = {"value": N * steps / dtv / 1e6, "unit": "MLUPS",
                       "ms_per_step": dtv / steps * 1e3,
                       "step_frac": N * step_bytes(st) * steps / dtv / 1e9
                                    / measured_peaks()[0]}
        if "f16" in rec:
            rec["f16"]["speedup_vs_f32"] = rec["f16"]["value"] / rec["f32"]["value"]
            rec["bf16"]["speedup_vs_f32"] = rec["bf16"]["value"] / rec["f32"]["value"]
        rec["steps"] = steps
        out[name] = rec
    return out


def run_batched(args, torch, cacl, stream):
    cases = impact_sweep_cases()
    nodes = sum(c[2].size for c in cases)
    b = cacl.Batch([c[0] for c in cases])
    for view, (p, solid, phi, u) in zip(b.cases, cases):
        view.set_geometry(solid)
        view.set_fields(phi, u)
    del cases
    if args.batch_variant:
        lv, pv = (int(v) for v in args.batch_variant.split(","))
        b.set_option(lv, pv)
        best = {"lb_variant": lv, "phase_variant": pv, "set": "--batch-variant"}
    else:
        best = b.autotune(steps=2)
    k = max(4, args.steps // 20)
    b.step(2)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    # the same cases one after another, each as its own graph
    e0.record(stream)
    for view in b.cases:
        view.step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    t_single = e0.elapsed_time(e1) / 1e3
    finite = True
    for view in b.cases:
        try:
            view.check_finite()
        except cacl.CaclError:
            finite = False
    b.close()
    return {"workload": "impact sweep, 48 cubes 64..160 (seeded), R = 0.2 n, "
                        "theta 120..160 deg, We 1..80, density ratio 100, f16 storage",
            "cases": 48, "nodes": nodes, "steps": k,
            "value": nodes * k / t_batch / 1e6, "unit": "MLUPS",
            "one_case_at_a_time": nodes * k / t_single / 1e6,
            "speedup": t_single / t_batch, "autotuned": best,
            "finite": finite}


def run_adjoint(args, torch, cacl, stream):
    """Adjoint/forward cost on a wettability-inference case shaped like the
    workload of the adjoint: n^3 (96 by default), flat walls, theta in 8 x 8
    patches drawn from [45, 135] deg (seeded), droplet R = n / 6, sigma =
    0.01, nu = 0.1."""
    from paper_2607_25444_b300 import inputs as I
    n = args.adjoint_grid
    p = I.base_params(n, n, n, sigma=0.01, nu_l=0.1, nu_g=0.1, theta_deg=90.0)
    solid = I.walls_z(n, n, n)
    phi = I.droplet(n, n, n, (n / 2, n / 2, 0.5), n / 6.0, p["width"])
    s = cacl.Solver(p)
    s.set_geometry(solid)
    idx = s.wall_list()["idx"]
    x, y = idx % n, (idx // n) % n
    patches = I.SplitMix64(7).array(64, 45.0, 135.0)
    theta_w = patches[(y * 8 // n) * 8 + (x * 8 // n)].astype(np.float32)
    steps, every = args.adjoint_steps, args.adjoint_every
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    s.set_fields(phi)
    s.set_wall_angles(theta_w)
    s.step(10)  # warm-up
    s.set_fields(phi)
    ev[0].record(stream)
    s.step(steps)
    ev[1].record(stream)
    s.set_fields(phi)
    ev[2].record(stream)
    s.adjoint_forward(steps, every, args.adjoint_outer)
    ev[3].record(stream)
    torch.cuda.synchronize()
    free_b, total_b = torch.cuda.mem_get_info()
    g = torch.zeros(n * n * n, dtype=torch.float32, device="cuda")
    g.view(n, n, n)[1] = 1.0  # dL/dphi of the footprint layer sum
    dth = torch.zeros(idx.size, dtype=torch.float64, device="cuda")
    dsg = torch.zeros(1, dtype=torch.float64, device="cuda")
    ev[4].record(stream)
    s.adjoint_backward(g, dth, dsg)
    ev[5].record(stream)
    torch.cuda.synchronize()
    t_bwd_first = ev[4].elapsed_time(ev[5])
    # the steady state of an optimisation loop: the backward again (the
    # segment graphs captured by the first call are replayed)
    ev[4].record(stream)
    s.adjoint_backward(g, dth, dsg)
    ev[5].record(stream)
    torch.cuda.synchronize()
    t_plain = ev[0].elapsed_time(ev[1])
    t_fwd = ev[2].elapsed_time(ev[3])
    t_bwd = ev[4].elapsed_time(ev[5])
    t_rec, _ = s.adjoint_timing()
    s.close()
    return {"workload": f"{n}^3 flat walls, theta in 8x8 patches U[45,135] deg, "
                        f"R={n / 6.0:g}",
            "device_gb_in_use_after_forward": (total_b - free_b) / 1e9,
            "dl_dsigma": float(dsg.item()),
            "dl_dtheta_abs_max": float(dth.abs().max().item()),
            "steps": steps, "ckpt_every": every, "outer_every": args.adjoint_outer,
            "forward_ms_per_step": t_plain / steps,
            "checkpointed_forward_ms_per_step": t_fwd / steps,
            "backward_ms_per_step": t_bwd / steps,
            "first_backward_ms_per_step": t_bwd_first / steps,
            "backward_over_forward": t_bwd / t_plain,
            "recompute_ms_per_step": t_rec / steps,
            "adjoint_over_forward_excluding_recompute": (t_bwd - t_rec) / t_plain,
            "note": "backward (second call, as in an optimisation loop; the first "
                    "call also captures the segment graphs) includes the recompute of "
                    "every segment with its tape; the second ratio leaves that "
                    "recompute out"}


def run_theta_recovery(args):
    """Static-droplet contact-angle recovery at 256^3 (Sect. 3.1 setup):
    for each imposed angle, run to (near) equilibrium and fit the circle of
    the phi = 1/2 crossings on the central xz plane; also the mass drift."""
    import torch

    from paper_2607_25444_b300 import cacl
    from paper_2607_25444_b300 import diagnostics as Dg
    torch.cuda.set_device(0)
    torch.cuda.set_stream(torch.cuda.Stream())
    out = []
    for th in args.angles:
        p, solid, phi = workload(GRID, th)
        s = cacl.Solver(p)
        s.set_geometry(solid)
        s.set_fields(phi)
        rec = {"theta": th, "measured": []}
        done = 0
        for target in args.checkpoints:
            s.step(target - done)
            done = target
            f = s.fields()[0]
            rec["measured"].append([target, Dg.contact_angle(f, 0.5, z_min=1.0),
                                    Dg.contact_angle(f, 0.5, z_min=4.5)])
        s.check_finite()
        m = s.mass()
        f = s.fields()[0].astype(np.float64)
        rec["mass_drift_rel"] = abs(f[solid == 0].sum() - m["m_ref"]) / m["m_ref"]
        # sensitivity of the measured angle to the unstated wall position
        # z_w and to the fit (crossings on z >= 1 against the band of nodes
        # with |phi - 1/2| < 0.1 and 0.2)
        rec["z_wall"] = {str(zw): Dg.contact_angle(f, zw, z_min=1.0)
                         for zw in (0.0, 0.5, 1.0)}
        rec["band_fit"] = {str(e): Dg.contact_angle_band(f, e, 0.5, z_min=1.0)
                           for e in (0.1, 0.2)}
        out.append(rec)
        s.close()
        print(json.dumps(rec), flush=True)
    print(json.dumps({"metric": "static contact angle recovery, 256^3",
                      "results": out}), flush=True)


def run_curved_wall(args):
    """Contact angle on a curved wall next to a flat one, on 2D slabs (the
    D3Q27 lattice one node thick): a drop of radius 30 relaxes for
    args.cw_steps steps (a) on a flat wall (256 x 128, walls at y = 0 and
    127) and (b) on a solid disc of radius 40 (256 x 256, periodic); sigma =
    0.01, W = 4, equal densities and viscosities. The angle comes from the
    circle fitted to the phi = 1/2 crossings farther than 3.5 from the wall
    surface (taken halfway between the solid and the fluid nodes)."""
    import torch

    from paper_2607_25444_b300 import cacl
    from paper_2607_25444_b300 import diagnostics as Dg
    from paper_2607_25444_b300 import inputs as I
    torch.cuda.set_device(0)
    torch.cuda.set_stream(torch.cuda.Stream())
    steps = args.cw_steps
    out = []
    for th in args.angles:
        nx, ny = 256, 128
        p = I.base_params(nx, ny, 1, dim=2, periodic=(1, 0, 1), sigma=0.01,
                          theta_deg=th)
        s = cacl.Solver(p)
        s.set_geometry(I.walls_y(nx, ny, 1))
        s.set_fields(I.droplet(nx, ny, 1, (nx / 2, 0.5, 0.0), 30.0, p["width"]))
        s.step(steps)
        s.check_finite()
        f = s.fields()[0][0]
        flat = Dg.contact_angle(f[:, None, :], z_wall=0.5, y=0, z_min=4.0)
        s.close()
        n, rc, cx, cy = 256, 40.0, 128.0, 100.0
        p = I.base_params(n, n, 1, dim=2, periodic=(1, 1, 1), sigma=0.01,
                          theta_deg=th)
        s = cacl.Solver(p)
        s.set_geometry(I.cylinder_solid(n, n, 1, (cx, cy), rc))
        s.set_fields(I.droplet(n, n, 1, (cx, cy + rc + 0.5, 0.0), 30.0, p["width"]))
        s.step(steps)
        s.check_finite()
        f = s.fields()[0][0]
        disc = Dg.contact_angle_on_disc(f, (cx, cy), rc + 0.5, min_gap=3.5)
        s.close()
        rec = {"theta": th, "flat": flat, "disc": disc, "steps": steps}
        out.append(rec)
        print(json.dumps(rec), flush=True)
    print(json.dumps({"metric": "contact angle on a flat wall and on a disc "
                                "of radius 40 (2D slab, drop radius 30)",
                      "results": out}), flush=True)


def run_inference(args):
    """Wettability inference shaped like the paper's footprint analysis
    (contact angle from the droplet's wetted footprint): 96^3 between flat
    walls, the bottom wall's contact angle in 8 x 8 patches of 12 x 12 nodes
    drawn from U[45, 135] deg (seeded), the top wall at 90 deg, a drop of
    radius 16 resting on the bottom wall, sigma = 0.01, nu = 0.1. The target
    is the footprint phi(x, y, z = 1) after a rollout of --inf-steps steps
    (2000) with the true angles; the angles are recovered from a uniform
    90 deg start by Adam on the 64 patch angles with dL/dtheta from the
    hand-written adjoint (checkpoints every --inf-every steps, FP32 forward,
    FP64 accumulation of the gradients), L = sum over z = 1 of
    (phi - phi_target)^2. Prints one JSON line."""
    import torch

    from paper_2607_25444_b300 import cacl
    from paper_2607_25444_b300 import inputs as I
    torch.cuda.set_device(0)
    torch.cuda.set_stream(torch.cuda.Stream())
    stream = torch.cuda.current_stream()
    n = 96
    p = I.base_params(n, n, n, sigma=0.01, nu_l=0.1, nu_g=0.1, theta_deg=90.0)
    solid = I.walls_z(n, n, n)
    phi0 = I.droplet(n, n, n, (n / 2, n / 2, 0.5), 16.0, p["width"])
    s = cacl.Solver(p)
    s.set_geometry(solid)
    idx = s.wall_list()["idx"]
    x, y, z = idx % n, (idx // n) % n, idx // (n * n)
    bottom = z == 0
    patch = (y // 12) * 8 + (x // 12)
    truth = I.SplitMix64(2025).array(64, 45.0, 135.0)
    steps, every = args.inf_steps, args.inf_every

    def angles(theta_patch):
        th = np.full(idx.size, 90.0, np.float32)
        th[bottom] = np.asarray(theta_patch, np.float64)[patch[bottom]]
        return th

    # target footprint
    s.set_fields(phi0)
    s.set_wall_angles(angles(truth))
    s.step(steps)
    target = s.fields()[0][1].copy()
    # forward cost at this size (plain steps)
    s.set_fields(phi0)
    s.step(10)
    torch.cuda.synchronize()
    t_fwd = median_steps_time(s, torch, stream, 200, 3) / 200
    tgt = torch.from_numpy(target).cuda()
    theta = np.full(64, 90.0)
    m = np.zeros(64)
    v = np.zeros(64)
    lr, b1, b2 = 3.0, 0.9, 0.999
    hist = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2 = torch.cuda.Event(enable_timing=True)
    t_bwd = []
    touched = None
    for it in range(args.inf_iters):
        s.set_fields(phi0)
        s.set_wall_angles(angles(theta))
        e0.record(stream)
        s.adjoint_forward(steps, every)
        e1.record(stream)
        phi = torch.empty(n ** 3, dtype=torch.float32, device="cuda")
        s.fields_device(phi=phi)
        ph1 = phi.view(n, n, n)[1]
        loss = float(((ph1 - tgt) ** 2).sum().item())
        g = torch.zeros(n ** 3, dtype=torch.float32, device="cuda")
        g.view(n, n, n)[1] = 2.0 * (ph1 - tgt)
        dth = torch.zeros(idx.size, dtype=torch.float64, device="cuda")
        dsg = torch.zeros(1, dtype=torch.float64, device="cuda")
        s.adjoint_backward(g, dth, dsg)
        e2.record(stream)
        torch.cuda.synchronize()
        t_bwd.append(e1.elapsed_time(e2) / 1e3 / steps)
        gw = dth.cpu().numpy()
        gp = np.bincount(patch[bottom], weights=gw[bottom], minlength=64)
        if touched is None:
            touched = np.abs(gp) > 1e-6 * np.abs(gp).max()
        hist.append(loss)
        m = b1 * m + (1 - b1) * gp
        v = b2 * v + (1 - b2) * gp * gp
        mh = m / (1 - b1 ** (it + 1))
        vh = v / (1 - b2 ** (it + 1))
        theta = np.clip(theta - lr * mh / (np.sqrt(vh) + 1e-12), 20.0, 160.0)
    free_b, total_b = torch.cuda.mem_get_info()
    s.close()
    err = np.abs(theta - truth)
    line = {
        "metric": "wettability inference from the footprint (adjoint)",
        "workload": f"{n}^3 flat walls, bottom-wall theta in 8x8 patches "
                    "U[45,135] deg (seeded), R=16, sigma=0.01, nu=0.1",
        "steps": steps, "ckpt_every": every, "iterations": args.inf_iters,
        "loss_first": hist[0], "loss_last": hist[-1],
        "loss_reduction": hist[0] / max(hist[-1], 1e-300),
        "patches_touched": int(touched.sum()),
        "theta_err_touched_mean_deg": float(err[touched].mean()),
        "theta_err_touched_max_deg": float(err[touched].max()),
        "theta_err_start_touched_mean_deg": float(np.abs(90.0 - truth)[touched].mean()),
        "theta_err_all_mean_deg": float(err.mean()),
        "forward_ms_per_step": t_fwd * 1e3,
        "backward_ms_per_step": float(np.median(t_bwd)) * 1e3,
        "backward_over_forward": float(np.median(t_bwd)) / t_fwd,
        "device_gb_in_use": (total_b - free_b) / 1e9,
        "loss_history": [round(h, 6) for h in hist],
    }
    print(json.dumps(line), flush=True)


def run_c2_accuracy(args):
    """Storage-mode error on the spreading workload at its configured size
    (128^3, Sect. 3.2 shape, theta = 60 deg): FP32, FP16 and BF16 population
    storage against the FP64 oracle after --c2-steps steps (the horizon the
    oracle runs on this host's cores in a few minutes): the spreading radius
    r = sqrt(A / pi) of the wetted area {phi > 1/2} on the first fluid layer,
    and the largest phi difference. Prints one JSON line."""
    import torch

    from oracle import oracle as O
    from paper_2607_25444_b300 import cacl
    from paper_2607_25444_b300 import inputs as I
    torch.cuda.set_device(0)
    torch.cuda.set_stream(torch.cuda.Stream())
    p, solid, phi = I.spreading_128(60.0)
    steps = args.c2_steps
    o = O.Oracle(p)
    o.set_geometry(solid)
    o.set_fields(phi.astype(np.float64))
    t0 = time.perf_counter()
    o.step(steps)
    t_cpu = time.perf_counter() - t0
    ref = o.fields()[0]

    def radius(f):
        return float(np.sqrt((f[1] > 0.5).sum() / np.pi))

    r_ref = radius(ref)
    out = {"metric": "spreading radius error vs the FP64 oracle, 128^3",
           "steps": steps, "oracle_seconds": t_cpu, "r_oracle": r_ref}
    for st in ("f32", "f16", "bf16"):
        sv = cacl.Solver(dict(p, storage=st))
        sv.set_geometry(solid)
        sv.set_fields(phi)
        sv.step(steps)
        f = sv.fields()[0]
        sv.close()
        out[st] = {"r": radius(f), "r_err": abs(radius(f) - r_ref),
                   "phi_max_err": float(np.abs(f - ref).max())}
    print(json.dumps(out), flush=True)


def run_cuda(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2607_25444_b300 import cacl

    # a dedicated stream: the library and the CUDA events share it
    torch.cuda.set_stream(torch.cuda.Stream())
    p, solid, phi = workload(args.grid)
    p["storage"] = args.storage
    N = phi.size
    fluid = int((solid == 0).sum())
    s = cacl.Solver(p)
    s.set_geometry(solid)
    s.set_fields(phi)
    if args.phase_tile is not None:
        s.set_option(cacl.OPT_PHASE_TILE, args.phase_tile)
    if args.phase_pipe is not None:
        s.set_option(cacl.OPT_PHASE_PIPE, args.phase_pipe)
    if args.lb_pipe is not None:
        s.set_option(cacl.OPT_LB_PIPE, args.lb_pipe)
    W = s.info()["wall_count"]
    # collide-stream, phi update (its last block forms lambda), correction,
    # and the two ghost passes when there are walls
    kernels_per_step = 3 + (2 if W > 0 else 0)

    # warm-up, then REPEATS x K timed steps, each bracketed by barrier +
    # synchronize; the median repeat is the measurement
    s.step(args.warmup)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    times = []
    with ClockSampler(local) as clk:
        for _ in range(args.repeats):
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            s.step(args.steps)
            ev1.record(stream)
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            times.append(ev0.elapsed_time(ev1) / 1e3)
    dt = float(np.median(times))
    s.check_finite()
    mass = s.mass()
    phi_now = s.fields()[0]
    m_now = float(phi_now.astype(np.float64)[solid == 0].sum())
    drift = abs(m_now - mass["m_ref"]) / mass["m_ref"]

    t = torch.tensor([dt], device="cuda")
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    dt_max = float(t.item())
    value = world * N * args.steps / dt_max / 1e6

    # dominant kernel: the collide-stream, timed alone
    reps = max(5, min(50, args.steps))
    lb_s = time_lb_kernel(s, torch, reps)
    lb_bytes = fluid * lb_bytes_fluid(args.storage) + (N - fluid) * LB_BYTES_SOLID
    peak, peak_kind = measured_peaks()
    achieved = lb_bytes / lb_s / 1e9
    step_gbs = N * step_bytes(args.storage) * args.steps / dt / 1e9

    # end to end through the C ABI with pinned host buffers
    ph_host = torch.empty(N, dtype=torch.float32, pin_memory=True).numpy()
    u_host = torch.zeros(3 * N, dtype=torch.float32, pin_memory=True).numpy()
    out_phi = torch.empty(N, dtype=torch.float32, pin_memory=True).numpy()
    out_u = torch.empty(3 * N, dtype=torch.float32, pin_memory=True).numpy()
    ph_host[:] = phi.reshape(-1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.set_fields(ph_host, u_host)
    s.step(args.steps)
    s.L.cacl_get_fields(s.h, cacl._ptr(out_phi), cacl._ptr(out_u), None, 0)
    torch.cuda.synchronize()
    e2e_dt = time.perf_counter() - t0
    e2e = N * args.steps / e2e_dt / 1e6 * world
    h2d = (ph_host.nbytes + u_host.nbytes) / args.steps
    d2h = (out_phi.nbytes + out_u.nbytes) / args.steps
    s.close()

    # the same workload with 16-bit population storage (FP32 arithmetic)
    mixed = {}
    if args.storage == "f32" and not args.no_variants:
        for st in ("f16", "bf16", "moments"):
            pv = dict(p, storage=st)
            sv = cacl.Solver(pv)
            sv.set_geometry(solid)
            sv.set_fields(phi)
            sv.step(args.warmup)
            torch.cuda.synchronize()
            dtv = median_steps_time(sv, torch, stream, args.steps, args.repeats)
            lbv = time_lb_kernel(sv, torch, reps)
            lbytes = fluid * lb_bytes_fluid(st) + (N - fluid) * LB_BYTES_SOLID
            sv.check_finite()
            mixed[st] = {"value": N * args.steps / dtv / 1e6 * world,
                         "ms_per_step": dtv / args.steps * 1e3,
                         "speedup_vs_f32": dt / dtv,
                         "lb_launch_ms": lbv * 1e3,
                         "lb_frac": lbytes / lbv / 1e9 / peak,
                         "step_frac": N * step_bytes(st) * args.steps / dtv / 1e9 / peak}
            sv.close()

    workloads = None
    if not args.no_variants and world == 1:
        workloads = paper_workloads(args, torch, cacl, stream)
    batched = None
    if not args.no_batch and world == 1:
        batched = run_batched(args, torch, cacl, stream)
    adj = None
    if not args.no_adjoint and world == 1:
        adj = run_adjoint(args, torch, cacl, stream)

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu:
        v, cores, sample = cpu_oracle_run(2, max_seconds=30.0)
        cpu = {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": sample}
    options = {k: v for k, v in (("phase_tile", args.phase_tile),
                                 ("phase_pipe", args.phase_pipe),
                                 ("lb_pipe", args.lb_pipe)) if v is not None}
    if args.lb_pipe in (1, 2, 3):
        lb_kernel = {1: "lb_collide_staged", 2: "lb_collide", 3: "lb_collide_tma"}[args.lb_pipe]
    else:
        lb_kernel = {"f32": "lb_collide_pair32", "f16": "lb_collide_quad",
                     "bf16": "lb_collide_quad", "moments": "lb_collide_moments"}[args.storage]
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "repeats": args.repeats,
        "repeat_ms": [round(x * 1e3, 4) for x in times],
        "ms_per_step": dt_max / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "storage": args.storage,
        "data": "synthetic",
        "config": {"workload": f"static droplet on a flat wall, "
                               f"{args.grid}^3, R0={40 * args.grid // 256}, "
                               "theta=60 deg, equal densities, nu=0.04, "
                               "sigma=0.02, W=4, D=0.02",
                   "grid": [args.grid] * 3, "storage": args.storage,
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (populations 2 x 1.8 GB)",
                   "wall_nodes": W, "fluid_nodes": fluid,
                   **({"options": options} if options else {})},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak,
                     "traffic": (kernel_traffic(fluid)
                                 if lb_kernel == "lb_collide_pair32" else None),
                     "kernel": lb_kernel,
                     "peak_source": peak_kind,
                     "algorithmic_bytes_per_launch": lb_bytes,
                     "kernel_bytes_per_fluid_node": lb_bytes_fluid(args.storage) + 12,
                     "launch_ms": lb_s * 1e3},
        "step_roofline": {"bytes_per_node": step_bytes(args.storage),
                          "achieved": step_gbs, "frac": step_gbs / peak,
                          "ideal_mlups": peak * 1e9 / step_bytes(args.storage) / 1e6},
        "e2e": {"value": e2e, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": kernels_per_step * args.steps * args.repeats,
        "clocks": clk.summary(),
        "checks": {"mass_drift_rel": drift, "lambda": mass["lam"]},
        "cpu_baseline": cpu,
        "mixed": mixed or None,
        "workloads": workloads,
        "batched": batched,
        "adjoint": adj,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--repeats", type=int, default=5,
                    help="timed repeats of --steps steps; the median is reported")
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--grid", type=int, default=GRID,
                    help="cube edge (the benchmark is 256; smaller edges are "
                         "for profiling captures)")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16", "moments"],
                    help="population storage of the headline line")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the adjoint/forward cost measurement")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched impact-sweep timing")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the 16-bit storage timings")
    ap.add_argument("--no-cpu", action="store_true",
                    help="skip the CPU-oracle baseline leg")
    ap.add_argument("--theta-recovery", action="store_true",
                    help="measure the static contact angle at 256^3 instead")
    ap.add_argument("--angles", type=float, nargs="*",
                    default=[30.0, 60.0, 90.0, 120.0, 150.0])
    ap.add_argument("--checkpoints", type=int, nargs="*",
                    default=[10000, 20000, 30000, 40000])
    ap.add_argument("--adjoint-steps", type=int, default=200,
                    help="rollout length of the adjoint/forward cost measurement")
    ap.add_argument("--adjoint-every", type=int, default=50,
                    help="checkpoint interval of that measurement")
    ap.add_argument("--curved-wall", action="store_true",
                    help="contact angle of a 2D drop on a flat wall and on a "
                         "disc, for each of --angles")
    ap.add_argument("--cw-steps", type=int, default=40000,
                    help="relaxation steps of --curved-wall")
    ap.add_argument("--adjoint-grid", type=int, default=96,
                    help="cube edge of the adjoint cost measurement")
    ap.add_argument("--adjoint-outer", type=int, default=0,
                    help="outer checkpoint interval (two-level checkpointing; "
                         "0 = one level)")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="run only the adjoint/forward cost measurement and "
                         "print its JSON (for profiling the adjoint kernels)")
    ap.add_argument("--inference", action="store_true",
                    help="run the wettability inference (96^3, 8x8 patches) instead")
    ap.add_argument("--inf-steps", type=int, default=2000)
    ap.add_argument("--inf-every", type=int, default=100)
    ap.add_argument("--inf-iters", type=int, default=30)
    ap.add_argument("--c2-accuracy", action="store_true",
                    help="storage-mode error on the 128^3 spreading case "
                         "against the FP64 oracle instead")
    ap.add_argument("--c2-steps", type=int, default=60)
    ap.add_argument("--cpu-extended", action="store_true",
                    help="time the FP64 oracle on the host: headline slab on 1 and all "
                         "threads, c1 at 2000 steps, 10 steps of c2")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the batched impact sweep and print its JSON")
    ap.add_argument("--phase-tile", type=int, default=None,
                    help="CACL_OPT_PHASE_TILE of the headline solver")
    ap.add_argument("--phase-pipe", type=int, default=None,
                    help="CACL_OPT_PHASE_PIPE of the headline solver")
    ap.add_argument("--lb-pipe", type=int, default=None,
                    help="CACL_OPT_LB_PIPE of the headline solver")
    ap.add_argument("--batch-variant", default="",
                    help="LB,PHASE launch shapes of the batch instead of autotuning")
    args = ap.parse_args()
    if args.inference:
        run_inference(args)
        return
    if args.c2_accuracy:
        run_c2_accuracy(args)
        return
    if args.cpu_extended:
        run_cpu_extended(args)
        return
    if args.batch_only:
        import torch

        from paper_2607_25444_b300 import cacl
        torch.cuda.set_device(0)
        torch.cuda.set_stream(torch.cuda.Stream())
        print(json.dumps(run_batched(args, torch, cacl, torch.cuda.current_stream())),
              flush=True)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.theta_recovery:
        run_theta_recovery(args)
        return
    if args.curved_wall:
        run_curved_wall(args)
        return
    if args.adjoint_only:
        import torch

        from paper_2607_25444_b300 import cacl
        torch.cuda.set_device(0)
        torch.cuda.set_stream(torch.cuda.Stream())
        print(json.dumps(run_adjoint(args, torch, cacl, torch.cuda.current_stream())),
              flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_cuda(args)


if __name__ == "__main__":
    main()
