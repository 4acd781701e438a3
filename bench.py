"""Throughput benchmark of the batched generalized-FDTD engine on GB300.

Workload (default): the batched moving bilayer crystal -- 4096 instances,
Nz log-uniform in [2^12, 2^18] (2.5e8 cells), v uniform in [-0.8, 0.8]c,
64 periods of eps 1/4 layers, FP32 fields, seeded synthetic data.  One bench
"step" is one gfdtd_step call advancing the whole batch by --time-steps
leapfrog steps (all of: moving material, E*, B, H*, D, source injection, DFT
probes); the default 10 steps x 2000 time steps is the full 20000-step run.

Prints one JSON line: Gcell-updates/s (value, device-resident inputs), the
end-to-end number through the C ABI with host buffers (e2e), the plain
one-step-per-launch kernel and the batched/plain ratio, the roofline of the
batched kernel, the FP64 oracle timed on host cores (cpu_baseline) and the
SM clocks seen during the timed region.  --impl reference times the oracle
alone on the same workload.  Under torchrun every rank runs its own
instance batch (weak scaling, no collective on the data path).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOPS_PER_CELL_UPDATE = 20        # FP32 operations of one B and D update (E*, B, H*, D)
SM_COUNT, FP32_LANES_PER_SM, SM_MAX_MHZ = 152, 128, 2070.0


KERNEL_SOURCES = ("gfdtd_block.cuh", "gfdtd_internal.cuh", "gfdtd_block_f32.cu", "gfdtd_block_f32w.cu")


def kernel_source_hash():
    """sha256 over the sources the FP32 fast kernel is compiled from."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2304_06586_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(tile):
    """DRAM bytes per cell-update of the fast kernel in tile shape `tile`
    (cells per lane, time block, blocks per SM) from the committed ncu summary,
    if it was taken on the kernel sources as they are now and on that shape
    (else None)."""
    path = os.path.join(ROOT, "profiles", "fast_kernel_crystal.md")
    if not os.path.exists(path):
        return None
    fields = {}
    with open(path) as f:
        for line in f:
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                fields[k.strip()] = v.strip().strip("`")
    try:
        if fields.get("kernel source sha256") != kernel_source_hash():
            return None
        return float(fields["dram bytes per cell-update, tile %d,%d,%d" % tuple(tile)])
    except (KeyError, ValueError):
        return None


def roofline_of(kt, tile):
    """FP32-pipe roofline of the fast kernel (tile shape `tile`) from per-launch
    CUDA-event times."""
    fast = kt["fast"]
    if fast["launches"] == 0:
        return None
    launch_ms = fast["ms"] / fast["launches"]
    cu_per_launch = fast["cell_updates"] / fast["launches"]
    achieved = FLOPS_PER_CELL_UPDATE * cu_per_launch / (launch_ms / 1e3) / 1e12
    peak = 2 * FP32_LANES_PER_SM * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12
    bpc = measured_traffic(tile)
    total_ms = sum(v["ms"] for v in kt.values())
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "traffic": None if bpc is None else bpc * cu_per_launch,
            "kernel": "fast_kernel", "launch_ms": launch_ms, "cell_updates_per_launch": cu_per_launch,
            "share_of_batched_time": fast["ms"] / total_ms if total_ms > 0 else None,
            "note": "FP32 pipe: %d flops per cell-update (algorithmic), peak = 2 x 128 lanes x 152 SMs x "
                    "2070 MHz (derived); launch time from CUDA events around each fast_kernel launch; "
                    "traffic = ncu DRAM bytes per cell-update x cell-updates per launch"
                    % FLOPS_PER_CELL_UPDATE}


FP64_PEAK_TFLOPS = 2 * 2 * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12   # 2 FP64 FMA per SM per cycle
STAB_FLOPS_PER_SAMPLE = 110      # FP64 operations of one amplification matrix and its eigenvalues
TMM_FLOPS_PER_LAYER = 67         # FP64 operations of one interface + propagation matrix product


def sweep_measurements(torch, gb, stream, reps=3):
    """Throughput of the two batched FP64 sweep kernels (stability map, star TMM)
    on seeded synthetic parameter sets, CUDA events on the launching stream."""
    rng = np.random.default_rng(20230413 + 9)
    out = {}
    n, n_theta = 1 << 20, 1024
    P = [torch.as_tensor(v).to("cuda") for v in (rng.uniform(0.1, 1.0, n), rng.uniform(-0.9, 0.9, n),
                                                   rng.uniform(1.0, 9.0, n), rng.uniform(1.0, 2.0, n))]
    K = torch.as_tensor(rng.integers(0, 2, n), dtype=torch.int32).to("cuda")
    res = torch.empty(n, dtype=torch.float64, device="cuda")
    lib = gb.load()

    def stab():
        rc = lib.gfdtd_stability_map(n, *[t.data_ptr() for t in P], K.data_ptr(), n_theta, res.data_ptr(),
                                     stream.cuda_stream)
        assert rc == 0, rc

    n_s, n_l, n_f = 1 << 16, 16, 64
    off = torch.arange(0, (n_s + 1) * n_l, n_l, dtype=torch.int64).to("cuda")
    eps = torch.as_tensor(rng.uniform(1.0, 6.0, n_s * n_l)).to("cuda")
    mu = torch.ones(n_s * n_l, dtype=torch.float64, device="cuda")
    th = torch.as_tensor(rng.uniform(5.0, 80.0, n_s * n_l)).to("cuda")
    beta = torch.as_tensor(rng.uniform(-0.3, 0.3, n_s)).to("cuda")
    om = torch.linspace(0.05, 0.6, n_f, dtype=torch.float64, device="cuda")
    T = torch.empty(2 * n_s * n_f, dtype=torch.float64, device="cuda")
    G = torch.empty_like(T)

    def tmm():
        rc = lib.gfdtd_star_tmm(n_s, off.data_ptr(), eps.data_ptr(), mu.data_ptr(), th.data_ptr(), beta.data_ptr(),
                                n_f, om.data_ptr(), T.data_ptr(), G.data_ptr(), stream.cuda_stream)
        assert rc == 0, rc

    for name, fn, units, flops_per_unit, unit_name in (
            ("stability_map", stab, n * n_theta, STAB_FLOPS_PER_SAMPLE, "G samples/s"),
            ("star_tmm", tmm, n_s * n_f * (n_l - 1), TMM_FLOPS_PER_LAYER, "G layer-frequencies/s")):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3 / reps
        achieved = flops_per_unit * units / sec / 1e12
        out[name] = {"value": units / sec / 1e9, "unit": unit_name, "ms_per_launch": sec * 1e3,
                     "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                                  "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                                  "note": "FP64 pipe: %d flops per unit (algorithmic, sin/cos not counted), "
                                          "peak = 2 FMA x 152 SMs x 2070 MHz (derived)" % flops_per_unit}}
    out["stability_map"]["config"] = "%d points x %d kz samples, kinds mixed" % (n, n_theta)
    out["star_tmm"]["config"] = "%d stacks x %d layers x %d frequencies" % (n_s, n_l, n_f)
    return out


def adjoint_measurement(gb):
    """The adjoint workload (256 x 2^14 piecewise-linear profiles, 16000 steps):
    wall time of gfdtd_adjoint (forward, sqrt(T) checkpoints, reverse sweep and
    FP64 gradients, host results) against gfdtd_step over the same steps."""
    import torch
    from paper_2304_06586_gb300 import workloads as w
    wl = w.config5()
    T = wl.n_steps
    cells = sum(i.nz for i in wl.instances)

    def make():
        sim = gb.Simulation([i.nz for i in wl.instances], wl.S, gb.F32)
        configure(sim, wl, gb)
        return sim

    f = make()
    f.step(64)                      # tiling, graphs
    f.synchronize()
    t0 = time.perf_counter()
    f.step(T)
    f.synchronize()
    tf = time.perf_counter() - t0
    f.close()
    a = make()
    nv = [len(i.eps) for i in wl.instances]
    a.adjoint(64, 0, 0, 16, nv)     # warm-up
    t0 = time.perf_counter()
    loss, _ = a.adjoint(T, 0, 0, 16, nv)
    ta = time.perf_counter() - t0
    a.close()
    torch.cuda.synchronize()
    return {"value": cells * T / ta / 1e9, "unit": "Gcell-updates/s (forward steps covered per second)",
            "seconds": ta, "forward_seconds": tf, "adjoint_over_forward": ta / tf,
            "config": wl.description, "loss_finite": bool(np.all(np.isfinite(loss)))}


def example_measurements(gb, torch):
    """Throughput of the paper's other example workloads through gfdtd_step
    (inputs resident, one warm-up call for tiling and graphs, then one timed
    call): the moving interface in FP64, the moving-matter slab in FP32, and
    the moving gradient (stable eps 1 -> 2 ramp, 2^20 cells) in every
    precision tier.  Step counts are cut to keep each timing near 0.1-0.5 s."""
    from paper_2304_06586_gb300 import workloads as w
    cases = [("interface FP64 (4000 cells, v=0.3c)", w.config1(), gb.F64, 8000),
             ("moving-matter slab FP32 (5 x 2^16 cells, v in +-0.5c)", w.config2(), gb.F32, 8000)]
    for name, prec in (("F32", gb.F32), ("F32_KAHAN", gb.F32_KAHAN), ("BF16", gb.BF16),
                       ("F16", gb.F16), ("F64", gb.F64)):
        cases.append((f"gradient {name} (2^20 cells, ramp eps 1->2, v=0.7c)", w.config4("stable"), prec,
                      2000 if prec == gb.F64 else 8000))
    out = {}
    for name, wl, prec, steps in cases:
        sim = gb.Simulation([i.nz for i in wl.instances], wl.S, prec)
        configure(sim, wl, gb)
        sim.step(256)
        sim.synchronize()
        t0 = time.perf_counter()
        sim.step(steps)
        sim.synchronize()
        dt = time.perf_counter() - t0
        cells = sum(i.nz for i in wl.instances)
        st = sim.stats()
        out[name] = {"value": cells * steps / dt / 1e9, "unit": "Gcell-updates/s", "steps": steps,
                     "seconds": dt, "tile": [st["cells_per_lane"], st["time_block"], st["blocks_per_sm"]],
                     "uniform_split": bool(st["uniform_split"])}
        sim.close()
    torch.cuda.synchronize()
    return out


def gradient_as_written(gb, window=4000):
    """The moving-gradient workload as written: linear eps ramp 1 -> 6 over 2^18
    of 2^20 cells, v = 0.7c, 2 x 10^5 steps, FP32, from rest with its source.
    Beyond eps = 1/0.49 the ramp has n|v| > 1, where the scheme is unstable
    (Sec. 5); the watchdog's largest |B|, |D| over each `window` steps gives the
    measured growth per step, compared with the von Neumann max|zeta| of the
    ramp's densest medium (App. A).  The watchdog reads (one synchronisation
    per window) are inside the timed run."""
    from paper_2304_06586_gb300 import workloads as w
    wl = w.config4("as_written")
    T = wl.n_steps
    sim = gb.Simulation([i.nz for i in wl.instances], wl.S, gb.F32)
    configure(sim, wl, gb)
    sim.step(256)
    sim.watchdog(reset=True)
    amax, first_flag = [], None
    t0 = time.perf_counter()
    for k in range(T // window):
        sim.step(window)
        flags, a = sim.watchdog(limit=1e30, reset=True)
        amax.append(float(a[0]))
        if flags[0] and first_flag is None:
            first_flag = (k + 1) * window + 256
    dt = time.perf_counter() - t0
    sim.close()
    rates = [(b / a) ** (1.0 / window) for a, b in zip(amax, amax[1:])
             if 0 < a < float("inf") and 0 < b < float("inf")]
    zeta = gb.stability(wl.S, 0.7, 6.0, 1.0, gb.PERTURBATION)
    return {"value": wl.cells * (T // window) * window / dt / 1e9, "unit": "Gcell-updates/s",
            "steps": (T // window) * window, "seconds": dt, "config": wl.description,
            "growth_per_step_max": max(rates) if rates else None,
            "growth_per_step_last": rates[-1] if rates else None,
            "von_neumann_max_abs_zeta_eps6": zeta,
            "flagged_at_step": first_flag, "largest_field_per_window": amax[::5]}


FLOPS_PER_CELL_UPDATE_2D = 19    # FP32 operations of one 2D TE update (E', B_x, B_z, H'x, H'z, D)


def te2d_measurement(gb, torch, n_steps=2000):
    """The 2D TE scheme: 32 periodic columns (dx = 2) x 2^20 cells along the
    motion, slanted moving layers (eps 1 / 4, 20-120 cells, slope 0.3,
    v = 0.3c), an oblique line source and a probe, FP32, tile 8 x 16; CUDA
    events on the context's stream around gfdtd2d_step after a warm-up call."""
    rng = np.random.default_rng(20230413 + 11)
    nx, nz, dx = 32, 1 << 20, 2.0
    widths = rng.integers(20, 121, size=4000)
    z = nz / 8 + np.cumsum(widths)
    z = z[z < 7 * nz / 8]
    eps = np.array([1.0] + [4.0 if i % 2 == 0 else 1.0 for i in range(len(z))])
    stream = torch.cuda.Stream()
    sim = gb.Simulation2D(nx, nz, dx, 0.5, gb.F32, stream=stream.cuda_stream)
    sim.set_medium(0.3, 0.3, z, eps, np.ones(len(eps)))
    w0 = 2 * np.pi / 40.0
    tau = 10 * 40.0 / (2 * np.sqrt(np.log(2)))
    sim.add_source(nz // 16, w0 * 0.5, w0, tau, 4 * tau)
    sim.add_probe(0, nz * 15 // 16, np.linspace(0.75, 1.25, 16) * w0)
    sim.set_tuning(8, 16)
    sim.step(64)
    sim.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(n_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    sim.close()
    cu = nx * nz * n_steps
    achieved = FLOPS_PER_CELL_UPDATE_2D * cu / sec / 1e12
    peak = 2 * FP32_LANES_PER_SM * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12
    return {"value": cu / sec / 1e9, "unit": "Gcell-updates/s", "steps": n_steps, "seconds": sec,
            "config": "%d columns x 2^20 cells, slanted moving layers (slope 0.3, v = 0.3c), FP32, tile 8x16"
                      % nx,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "note": "FP32 pipe: %d flops per 2D cell-update (algorithmic), peak derived as for the "
                                 "1D kernel; whole gfdtd2d_step time (tile kernel, sources, probe folds)"
                                 % FLOPS_PER_CELL_UPDATE_2D}}


CASES = ["adjoint", "interface", "slab", "tfsf", "gradient-written", "te2d"] + \
    ["gradient-" + t for t in ("F32", "F32_KAHAN", "BF16", "F16", "F64")]


def run_case(args):
    """One side workload alone (for profiling it): `adjoint` (256 x 2^14 PWL
    profiles, gfdtd_adjoint over --time-steps steps), `tfsf` (the crystal of
    --instances instances with one-way sources), `interface` (FP64),
    `slab` (moving matter, FP32) or `gradient-<tier>` (2^20-cell ramp), through
    gfdtd_step with the tile shape of --tile if given.  Prints one JSON line."""
    import torch
    from paper_2304_06586_gb300 import binding as gb
    from paper_2304_06586_gb300 import workloads as w
    T = args.time_steps
    if args.case == "gradient-written":
        print(json.dumps({"case": args.case, **gradient_as_written(gb)}), flush=True)
        return
    if args.case == "te2d":
        print(json.dumps({"case": args.case, **te2d_measurement(gb, torch)}), flush=True)
        return
    if args.case == "adjoint":
        wl = w.config5(n_steps=T)
        sim = gb.Simulation([i.nz for i in wl.instances], wl.S, gb.F32)
        configure(sim, wl, gb)
        if args.tile:
            sim.set_tuning(*[int(x) for x in args.tile.split(",")])
        nv = [len(i.eps) for i in wl.instances]
        sim.adjoint(64, 0, 0, 16, nv)
        t0 = time.perf_counter()
        sim.adjoint(T, 0, 0, 16, nv)
        dt = time.perf_counter() - t0
    elif args.case == "tfsf":
        # the batched crystal (--instances of them) with a one-way source in place of each soft source
        wl = w.config3(n_inst=args.instances, n_steps=T)
        sim = gb.Simulation([i.nz for i in wl.instances], wl.S, gb.F32)
        for k, I in enumerate(wl.instances):
            sim.set_medium(k, I.kind, I.beta, I.interp, I.z, I.eps, I.mu, allow_unstable=True)
            for src in I.sources:
                sim.add_tfsf(k, *src)
            for p in I.probes:
                sim.add_probe(k, p[0], p[1])
        if args.tile:
            sim.set_tuning(*[int(x) for x in args.tile.split(",")])
        sim.step(64)
        sim.synchronize()
        t0 = time.perf_counter()
        sim.step(T)
        sim.synchronize()
        dt = time.perf_counter() - t0
    else:
        if args.case == "interface":
            wl, prec = w.config1(), gb.F64
        elif args.case == "slab":
            wl, prec = w.config2(), gb.F32
        else:
            wl, prec = w.config4("stable"), getattr(gb, args.case.split("-", 1)[1])
        sim = gb.Simulation([i.nz for i in wl.instances], wl.S, prec)
        configure(sim, wl, gb)
        if args.tile:
            sim.set_tuning(*[int(x) for x in args.tile.split(",")])
        sim.step(64)
        sim.synchronize()
        t0 = time.perf_counter()
        sim.step(T)
        sim.synchronize()
        dt = time.perf_counter() - t0
    st = sim.stats()
    cells = sum(i.nz for i in wl.instances)
    sim.close()
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "workload": wl.description, "steps": T, "seconds": dt,
                      "value": cells * T / dt / 1e9, "unit": "Gcell-updates/s",
                      "tile": [st["cells_per_lane"], st["time_block"], st["blocks_per_sm"]],
                      "uniform_split": bool(st["uniform_split"])}), flush=True)


E2E_PARTS = 4


def e2e_groups(cells, parts):
    """Contiguous groups of instance indices of about equal total cells."""
    cells = np.asarray(cells, dtype=np.int64)
    bounds = np.searchsorted(np.cumsum(cells), np.linspace(0, cells.sum(), parts + 1)[1:-1])
    return [g for g in np.split(np.arange(len(cells)), bounds) if len(g)]


def e2e_pipelined(gb, torch, wl, T, steps, tile, barrier, pg, world, cu):
    """End-to-end throughput through the public API: every bench step writes
    each part's state (B, D) from pinned host buffers, advances it T steps and
    reads it back; parts sit on their own streams, so copies and kernels of
    different parts overlap (host<->device copies counted in full)."""
    groups = e2e_groups([i.nz for i in wl.instances], E2E_PARTS)
    parts = []
    for g in groups:
        strm = torch.cuda.Stream()
        sub = type(wl)(wl.name, wl.S, wl.n_steps, [wl.instances[i] for i in g], wl.description)
        sim = gb.Simulation([i.nz for i in sub.instances], sub.S, gb.F32, stream=strm.cuda_stream)
        configure(sim, sub, gb)
        sim.set_tuning(*tile)
        n_el, eb, _ = sim.state_layout()
        nbytes = n_el * eb
        hB = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        hD = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        sim.step(T)                                  # tiling, graphs, fields away from rest
        sim.read_state(gb.FIELD_B, hB.data_ptr(), nbytes)
        sim.read_state(gb.FIELD_D, hD.data_ptr(), nbytes)
        parts.append((sim, hB, hD, nbytes))
    for sim, *_ in parts:
        sim.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        for sim, hB, hD, nbytes in parts:
            sim.write_state(gb.FIELD_B, hB.data_ptr(), nbytes)
            sim.write_state(gb.FIELD_D, hD.data_ptr(), nbytes)
            sim.step(T)
            sim.read_state(gb.FIELD_B, hB.data_ptr(), nbytes)
            sim.read_state(gb.FIELD_D, hD.data_ptr(), nbytes)
        for sim, *_ in parts:
            sim.synchronize()
    barrier()
    dt = max_over_ranks(time.perf_counter() - t0, pg, "cuda")
    total = sum(2 * p[3] for p in parts)
    for sim, *_ in parts:
        sim.close()
    return {"value": cu * world / dt / 1e9, "unit": "Gcell-updates/s",
            "h2d_bytes_per_step": total, "d2h_bytes_per_step": total,
            "pipeline": {"contexts": len(parts), "note": "one stream per context; copies overlap other parts' steps"}}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--time-steps", type=int, default=2000, help="leapfrog steps per bench step")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--instances", type=int, default=4096)
    ap.add_argument("--plain-steps", type=int, default=4)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-sweeps", action="store_true", help="skip the side timings (sweeps, adjoint, example workloads)")
    ap.add_argument("--case", default="", choices=[""] + CASES,
                    help="time one side workload alone instead of the batched crystal")
    ap.add_argument("--tile", default="", help="cells_per_lane,time_block[,blocks_per_sm] (default: autotune)")
    return ap.parse_args()


def dist_setup():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_workload(rank, n_inst, time_steps):
    """The batch a rank runs: instances are independent, so every rank steps its
    own seeded batch of the crystal workload (weak scaling, no data exchange)."""
    from paper_2304_06586_gb300 import workloads as w
    return w.config3(n_inst=n_inst, n_steps=time_steps, seed=w.SEED0 + 3 + 1000 * rank)


def max_over_ranks(value, dist=None, device="cpu"):
    """The job's time is the slowest rank's (all_reduce MAX); identity on one rank."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(mhz)}


def configure(sim, wl, gb):
    for k, I in enumerate(wl.instances):
        sim.set_medium(k, I.kind, I.beta, I.interp, I.z, I.eps, I.mu, allow_unstable=True)
        for s in I.sources:
            sim.add_source(k, *s)
        for p in I.probes:
            sim.add_probe(k, p[0], p[1])


def cpu_baseline(wl, n_inst=32, n_steps=100, seed=1, single_core=False):
    """The FP64 oracle, as it stands, on a bounded sample of the workload."""
    import oracle
    rng = np.random.default_rng(seed)
    pick = sorted(rng.choice(len(wl.instances), size=min(n_inst, len(wl.instances)), replace=False))
    orcs = []
    for k in pick:
        I = wl.instances[k]
        o = oracle.Instance(I.nz, wl.S, I.beta, kind=I.kind, interp=I.interp, z=I.z, eps=I.eps, mu=I.mu)
        for s in I.sources:
            o.add_source(*s)
        for p in I.probes:
            o.add_probe(p[0], p[1])
        orcs.append(o)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.run_many(orcs, n_steps, threads=threads)
    dt = time.perf_counter() - t0
    cu = sum(o.nz for o in orcs) * n_steps
    out = {"value": cu / dt / 1e9, "unit": "Gcell-updates/s", "cores": threads, "kind": "oracle",
           "sample": "%d of %d instances x %d steps (%.3g cell-updates, %.1f s)"
                     % (len(orcs), len(wl.instances), n_steps, cu, dt)}
    if single_core:   # the same instances on one core, a quarter of the steps
        n1 = max(1, n_steps // 4)
        t1 = time.perf_counter()
        oracle.run_many(orcs, n1, threads=1)
        out["single_core"] = sum(o.nz for o in orcs) * n1 / (time.perf_counter() - t1) / 1e9
        out["sample"] += "; one core: %d steps" % n1
    return out


METRIC = "Gcell-updates/s batched vs plain on 1 GB300 at <=1e-4 L2 vs FP64; % of roofline"


def run_reference(args, wl, rank):
    if rank != 0:
        return
    per = [cpu_baseline(wl, n_inst=32, n_steps=60, seed=100 + i) for i in range(args.warmup)]
    vals = []
    for i in range(args.steps):
        vals.append(cpu_baseline(wl, n_inst=32, n_steps=60, seed=200 + i))
    v = float(np.mean([x["value"] for x in vals]))
    del per
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gcell-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.description},
            "cpu_baseline": {"value": v, "unit": "Gcell-updates/s", "cores": vals[0]["cores"],
                             "kind": "oracle", "sample": "per step: " + vals[0]["sample"]},
            "e2e": {"value": v, "unit": "Gcell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.case:
        return run_case(args)
    rank, world, local = dist_setup()
    wl = rank_workload(rank, args.instances, args.time_steps)
    if args.impl == "reference":
        return run_reference(args, wl, rank)

    import torch
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist

    from paper_2304_06586_gb300 import binding as gb
    gb.use_torch_allocator()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = gb.Simulation([i.nz for i in wl.instances], wl.S, gb.F32, stream=stream.cuda_stream)
        configure(sim, wl, gb)
        if args.tile:
            sim.set_tuning(*[int(x) for x in args.tile.split(",")])
        T = args.time_steps

        def barrier():
            if pg:
                pg.barrier()
            torch.cuda.synchronize()

        for _ in range(args.warmup):
            sim.step(T)
        barrier()
        st = sim.stats()
        l0 = st["kernel_launches"]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with Clocks(local) as clk:
            barrier()
            e0.record(stream)
            for _ in range(args.steps):
                sim.step(T)
            e1.record(stream)
            barrier()
        ms = max_over_ranks(e0.elapsed_time(e1), pg, "cuda")
        st = sim.stats()
        # runtime watchdog over the warm-up and timed steps: instances whose fields
        # overflowed (non-finite) or passed 1e30, against the host's von Neumann count
        # of instances with max|zeta| > 1 (n|v| > 1 in their eps = 4 layers, Sec. 5)
        wflags, _ = sim.watchdog(limit=1e30)
        unstable_vn = sum(1 for I in wl.instances
                          if gb.stability(wl.S, I.beta, float(np.max(I.eps)), 1.0, gb.PERTURBATION) > 1 + 1e-9)
        watchdog = {"instances": len(wl.instances), "non_finite": int(np.sum(wflags & 1)),
                    "above_1e30_or_non_finite": int(np.sum((wflags & 2) != 0)),
                    "flagged": int(np.sum(wflags != 0)), "unstable_by_von_neumann": unstable_vn,
                    "steps_recorded": T * (args.steps + args.warmup)}
        launches = st["kernel_launches"] - l0
        cells = st["cells"]
        cu = cells * T * args.steps
        value = cu * world / (ms / 1e3) / 1e9

        # roofline of the dominant kernel: the same step, each batched launch
        # bracketed by CUDA events on the simulation's stream
        kt = sim.profile_kernels(T)
        roofline = roofline_of(kt, (st["cells_per_lane"], st["time_block"], st["blocks_per_sm"]))

        # end to end through the C ABI with pinned host buffers: the batch split into
        # E2E_PARTS contexts of about equal cells, each on its own stream, so that one
        # part's host<->device copies overlap another part's stepping
        e2e = None
        if not args.no_e2e:
            e2e = e2e_pipelined(gb, torch, wl, T, args.steps, (st["cells_per_lane"], st["time_block"],
                                                               st["blocks_per_sm"]), barrier, pg, world, cu)

        # space-time capture of the largest instance (every cell, FP16, one frame per time
        # block): throughput of the same step with frames recorded
        capture = None
        if not args.no_sweeps:
            big = int(np.argmax([i.nz for i in wl.instances]))
            tb = st["time_block"]
            sim.set_capture(big, gb.FIELD_E, 0, wl.instances[big].nz, 1, tb, max_frames=T // tb + 1, half=True)
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            c0.record(stream)
            sim.step(T)
            c1.record(stream)
            barrier()
            cms = c0.elapsed_time(c1)
            nfr = sim.capture()[0].shape[0]
            sim.set_capture(0, gb.FIELD_D, 0, 1, 1, 0)
            capture = {"value": cells * T / (cms / 1e3) / 1e9, "unit": "Gcell-updates/s",
                       "frames": nfr, "cells_per_frame": wl.instances[big].nz, "field": "E, FP16",
                       "t_stride": tb, "relative_to_value": (cells * T / (cms / 1e3) / 1e9) / (value / world)}

        # absorbing layers (64 cells at both ends of every instance): throughput of the same step
        absorber = None
        if not args.no_sweeps:
            for k in range(len(wl.instances)):
                sim.set_absorber(k, 64, 0.2)
            sim.step(T)                    # rebuilds the tiling, warms the new graphs
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            a0.record(stream)
            sim.step(T)
            a1.record(stream)
            barrier()
            ams = a0.elapsed_time(a1)
            av = cells * T / (ams / 1e3) / 1e9
            absorber = {"value": av, "unit": "Gcell-updates/s", "width": 64, "sigma": 0.2,
                        "relative_to_value": av / (value / world)}
            for k in range(len(wl.instances)):
                sim.set_absorber(k, 0, 0.0)

        # one-way sources: the same crystal with every soft source replaced by a
        # one-way source at its node (a second context, same tile shape)
        tfsf = None
        if not args.no_sweeps:
            sim2 = gb.Simulation([i.nz for i in wl.instances], wl.S, gb.F32, stream=stream.cuda_stream)
            for k, I in enumerate(wl.instances):
                sim2.set_medium(k, I.kind, I.beta, I.interp, I.z, I.eps, I.mu, allow_unstable=True)
                for src in I.sources:
                    sim2.add_tfsf(k, *src)
                for p in I.probes:
                    sim2.add_probe(k, p[0], p[1])
            sim2.set_tuning(st["cells_per_lane"], st["time_block"], st["blocks_per_sm"])
            sim2.step(T)
            t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            t0e.record(stream)
            sim2.step(T)
            t1e.record(stream)
            barrier()
            tv = cells * T / (t0e.elapsed_time(t1e) / 1e3) / 1e9
            tfsf = {"value": tv, "unit": "Gcell-updates/s",
                    "sources": sum(len(i.sources) for i in wl.instances),
                    "relative_to_value": tv / (value / world)}
            sim2.close()

        # plain kernel (one step, one instance per launch) on a few steps
        plain = None
        if args.plain_steps > 0:
            sim.step_plain(1)
            barrier()
            p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            p0.record(stream)
            sim.step_plain(args.plain_steps)
            p1.record(stream)
            barrier()
            pms = p0.elapsed_time(p1)
            pv = cells * args.plain_steps / (pms / 1e3) / 1e9
            # the same launch structure without the arithmetic: what one instance and one
            # step per launch allow on this batch
            sim.plain_floor(1)
            barrier()
            p0.record(stream)
            sim.plain_floor(args.plain_steps)
            p1.record(stream)
            barrier()
            fv = cells * args.plain_steps / (p0.elapsed_time(p1) / 1e3) / 1e9
            plain = {"value": pv, "unit": "Gcell-updates/s", "steps": args.plain_steps,
                     "batched_over_plain": value / world / pv,
                     "structure_floor": {"value": fv, "unit": "Gcell-updates/s", "plain_frac": pv / fv,
                                         "note": "gfdtd_plain_floor: the plain path's launches (one per "
                                                 "instance and step, same grids, in a CUDA graph) reading "
                                                 "and writing back B and D without the arithmetic"}}
        sim.close()
        sweeps = None if args.no_sweeps else sweep_measurements(torch, gb, stream)
        adjoint = None if args.no_sweeps else adjoint_measurement(gb)
        examples = None if args.no_sweeps else example_measurements(gb, torch)
        if examples is not None:
            examples["gradient as written (eps 1->6, 2^20 cells, v=0.7c, 2e5 steps, FP32)"] = \
                gradient_as_written(gb)
        te2d = None if args.no_sweeps else te2d_measurement(gb, torch)

    if rank != 0:
        return
    clocks = clk.summary()
    line = {"metric": METRIC,
            "value": value, "unit": "Gcell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.description, "instances": len(wl.instances), "cells": cells,
                       "time_steps_per_step": T, "tile": [st["cells_per_lane"], st["time_block"], st["blocks_per_sm"]],
                       "l2": "inputs larger than L2 (%.2f GB of fields)" % (cells * 16 / 1e9),
                       "parallelism": "instances sharded per rank" if world > 1 else "1 GPU"},
            "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "plain": plain, "watchdog": watchdog,
            "clocks": clocks, "sweeps": sweeps, "capture": capture, "absorber": absorber, "adjoint": adjoint,
            "tfsf": tfsf, "examples": examples, "te2d": te2d}
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(wl, single_core=True)
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
