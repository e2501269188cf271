"""Benchmark of the matrix-free CHNS hot path on one GB300 (replicas on N GPUs).

Workload: the 3D drop on a uniform level-6 octree (64^3 trilinear hexes, 274,625
nodes x 6 DOF = 1,647,750 DOF), density and viscosity ratios 10, Re=100, We=10, Pe=100,
Fr=1 (gravity along -z), Cn=0.02, dt=5e-4; phi0 a tanh drop of radius 0.2, v0 a
seeded divergence-free sum of 8 Fourier modes with max |v| = 0.1, mu0 from the
discrete potential equation.

One step = one mixed-precision Newton step (FP64 residual, FP32 block-Jacobi build,
GMRES with the FP32 J x kernel, FP64 classical Gram-Schmidt, FP64 update) from the
same U^k, to a relative residual of 1e-9 (GMRES(30)).  value = DOF x (J x applications) / step
time, i.e. the J x throughput sustained by the whole Newton step.  The dominant
kernel's roofline uses the CUDA-event time of the J x launches taken inside the step.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

LEVEL = 6
DIM = 3
WORKLOAD = ("3D CHNS drop, uniform octree level 6 (64^3 Q1 hexes, 274,625 nodes x 6 DOF), "
            "rho/eta ratios 10, Re=100 We=10 Pe=100 Fr=1 Cn=0.02 dt=5e-4; one mixed-precision "
            "Newton step to rel. residual 1e-9 per step")
METRIC = "CHNS J·x GDOF/s & % HBM roofline; mixed vs FP64 Newton step time at ≤1e-9 rel"
# Per-element counts of the element kernels taken by ncu from one launch on the 64^3 mesh
# (profiles/element_kernels_64cubed_counts.md): executed floating-point operations (2 x FMA
# + ADD + MUL thread instructions of the kernel's precision, divided by the element count)
# and DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch.  They belong to
# the kernel sources whose SHA-256 is KERNEL_SRC_SHA; when the sources change, the bench
# reports them as null (stale) until they are captured again.
# preconditioner of the timed Newton step (chns_solver_opts.pc_type)
BENCH_PC_TYPE = 1
KERNEL_SRC_FILES = ("paper_2009_06628_gb300/csrc/element_kernels.cu", "paper_2009_06628_gb300/csrc/pointwise.cuh")
KERNEL_SRC_SHA = "de8fd3eb9c4ab80e"
KERNEL_COUNTS = {
    "jvp_fp32": {"flop_per_element": 14769.6, "dram_bytes": 35048192},
    "jvp_fp64": {"flop_per_element": 15168.0, "dram_bytes": 61910016},
    "residual_fp64": {"flop_per_element": 9688.0, "dram_bytes": 48285440},
    "vjp_fp64": {"flop_per_element": 20776.0, "dram_bytes": 77077760},
}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


def kernel_src_sha():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SRC_FILES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def counts_for(name):
    """ncu counts of kernel `name` if they belong to the current sources, else None."""
    if KERNEL_SRC_SHA is None or kernel_src_sha() != KERNEL_SRC_SHA:
        return None
    return KERNEL_COUNTS.get(name)


def workload_state(x):
    U = np.zeros((x.shape[0], DIM + 3))
    cfg = synth.config_params("drop3d")
    U[:, DIM + 1] = synth.drop_phi(x, [[0.5, 0.5, 0.5]], [0.2], cfg["Cn"])
    U[:, :DIM] = synth.fourier_velocity(x, 8, 2, 0.1)
    bnd = np.any((x <= 0.0) | (x >= 1.0), axis=1)
    U[bnd, :DIM] = 0.0
    return cfg, U


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, gpu):
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline_oracle():
    """The oracle's J x (torch forward mode, FP64, host cores) on the bench workload itself
    (the 64^3 mesh): one full application with all host threads, and one with a single
    thread over a 1/16 element subset (32 of the 512 element rows of 512), scaled to the
    whole mesh by its element count (the oracle's cost is per element)."""
    from oracle import Mesh as OMesh, Oracle, Params as OParams
    om = OMesh(DIM, LEVEL, synth.uniform_leaves(DIM, LEVEL))
    cfg, U = workload_state(om.x)
    prm = OParams(**cfg)
    Ut = torch.tensor(U)
    Un = Ut + 1e-4 * torch.tensor(synth.random_vectors(U.size, 1, 7)[0]).reshape(U.shape)
    Un[torch.tensor(om.boundary), :DIM] = 0.0
    x = torch.tensor(synth.random_vectors(U.size, 1, 8)[0]).reshape(U.shape)
    dof = U.size
    threads = torch.get_num_threads()
    o = Oracle(om)
    t0 = time.perf_counter()
    o.jvp(prm, Ut, Un, x)
    t_all = time.perf_counter() - t0
    sub = np.arange(om.E // 16)
    os1 = Oracle(om, elements=sub)
    torch.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        os1.jvp(prm, Ut, Un, x)
        t_one = (time.perf_counter() - t0) * om.E / sub.size
    finally:
        torch.set_num_threads(threads)
    return {"value": dof / t_all / 1e9, "unit": "GDOF/s", "cores": threads, "kind": "oracle",
            "value_1core": dof / t_one / 1e9,
            "sample": f"oracle J x (FP64 torch forward mode) on the 64^3 bench mesh ({dof} DOF): one application "
                      f"on {threads} threads ({t_all:.2f} s); one thread over {sub.size} of {om.E} elements "
                      f"({t_one * sub.size / om.E:.2f} s, scaled to the mesh)"}


def run_reference(args, rank, world):
    """The oracle's J x on the bench workload (the 64^3 mesh), one bounded sample per step:
    the first 1/8 of the Morton-ordered elements (32,768 of 262,144), all host threads.
    value = the DOF share of that sample / time (the oracle's cost is per element)."""
    if rank != 0:
        return 0
    from oracle import Mesh as OMesh, Oracle, Params as OParams
    om = OMesh(DIM, LEVEL, synth.uniform_leaves(DIM, LEVEL))
    sub = np.arange(om.E // 8)
    o = Oracle(om, elements=sub)
    cfg, U = workload_state(om.x)
    prm = OParams(**cfg)
    Ut = torch.tensor(U)
    Un = Ut.clone()
    x = torch.tensor(synth.random_vectors(U.size, 1, 8)[0]).reshape(U.shape)
    for _ in range(args.warmup):
        o.jvp(prm, Ut, Un, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.jvp(prm, Ut, Un, x)
    dt = (time.perf_counter() - t0) / args.steps
    v = U.size * (sub.size / om.E) / dt / 1e9
    sample = (f"oracle J x (FP64 torch forward mode) over {sub.size} of the {om.E} elements of the 64^3 bench mesh "
              f"per step, {torch.get_num_threads()} host threads")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GDOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": v, "unit": "GDOF/s", "cores": torch.get_num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def kernel_table(chns, gm, prm, U0, pk, fp32_peak, fp64_peak, reps=10):
    """Each element kernel alone on the bench mesh: CUDA-event time per launch with L2
    flushed before every launch (a 256 MiB buffer is overwritten), GDOF/s, algorithmic
    HBM bytes and their fraction of the measured copy bandwidth, and (when the ncu counts
    match the sources) flop rate against the measured FMA peak and DRAM traffic."""
    E, N, nf = gm.E, gm.N, DIM + 3
    dof = N * nf
    g = torch.Generator(device="cuda").manual_seed(17)
    Un = U0 + 1e-4 * torch.randn(U0.shape, device="cuda", dtype=torch.float64, generator=g)
    x = torch.randn(U0.shape, device="cuda", dtype=torch.float64, generator=g)
    U0f, Unf, xf = U0.float(), Un.float(), x.float()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    idx = E * (8 * 4 + 1)       # e2n + level (the hanging table is empty on the uniform mesh)
    kernels = {
        # name: (launch, precision, algorithmic bytes per launch, unit description)
        "residual_fp64": (lambda: chns.residual(gm, prm, U0, Un), 0, 3 * dof * 8 + idx,
                          "read U^k, U^{k+1}; write R"),
        "jvp_fp64": (lambda: chns.jvp(gm, prm, U0, Un, x), 0, 4 * dof * 8 + idx, "read U^k, U^s, x; write y"),
        "jvp_fp32": (lambda: chns.jvp(gm, prm, U0f, Unf, xf), 1, 4 * dof * 4 + idx, "read U^k, U^s, x; write y"),
        "vjp_fp64": (lambda: chns.vjp(gm, prm, U0, Un, x), 0, 5 * dof * 8 + idx + N,
                     "read U^k, U^s, w, node flags; write g_new, g_old"),
    }
    out = {}
    for name, (fn, prec, nbytes, what) in kernels.items():
        fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(reps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        ms = tot / reps
        gbs = nbytes / (ms * 1e-3) / 1e9
        rec = {"ms": ms, "gdof_s": dof / (ms * 1e-3) / 1e9, "algorithmic_bytes": nbytes, "bytes_read_written": what,
               "achieved_gbs": gbs, "hbm_frac": gbs / pk.get("hbm_gbs", 6800.0)}
        cnt = counts_for(name)
        peak = fp32_peak if prec == 1 else fp64_peak
        if cnt:
            tf = cnt["flop_per_element"] * E / (ms * 1e-3) / 1e12
            rec.update({"flop_per_element": cnt["flop_per_element"], "achieved_tflops": tf,
                        "peak_tflops": peak, "alu_frac": tf / peak,
                        "dram_bytes_per_launch": cnt.get("dram_bytes")})
        else:
            rec.update({"flop_per_element": None, "achieved_tflops": None, "peak_tflops": peak, "alu_frac": None,
                        "dram_bytes_per_launch": None})
        out[name] = rec
    del flush
    return out


def aggregate_replicas(t_ms, work, dist=None, device="cpu"):
    """Whole-job timing of N independent replicas: the slowest rank's time and the
    total work of all ranks (no data-path collective; only these two reductions)."""
    if dist is None:
        return t_ms, work
    t = torch.tensor([t_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(w)
    return float(t), float(w)


def layer_workload(min_level=5, max_level=10):
    """Two-layer (Rayleigh-Taylor-shaped) workload: heavy fluid on top (density ratio 3),
    interface z = 0.5 + 0.05 cos(2 pi x + phase) with a seeded phase; octree levels 5-10
    refined in a band graded so that it is 2:1 balanced by construction (26.1M elements).
    The reduced version (levels 4-8) keeps Cn / h_min = 2.56 with Cn = 0.01."""
    rng = np.random.default_rng(5)
    phase = float(rng.uniform(0.0, 2.0 * np.pi))
    dist = synth.layer_distance(0.5, 0.05, 1.0, phase)
    leaves = synth.graded_band_leaves(DIM, min_level, max_level, dist, 0.0, grade=3.0)
    cfg = synth.config_params("layer3d")
    cfg["Cn"] *= 2.0 ** (10 - max_level)
    return leaves, max_level, cfg, phase


def twodrops_workload(min_level=4, max_level=9):
    """Two drops (radii 0.12, 0.15, centres 0.35 apart, seeded orientation), octree
    levels 4-9 refined within 3 Cn of the interfaces, 2:1 balanced (2.49M elements).
    The reduced version (levels 3-7, Cn = 0.02, band 0.03) has 101,368 elements."""
    cfg = synth.config_params("twodrops3d")
    centers, radii = synth.two_drops(3)
    if max_level == 9:
        leaves = synth.sphere_band_leaves(DIM, min_level, max_level, centers, radii, 3 * cfg["Cn"])
    else:
        cfg["Cn"] = 0.02
        leaves = synth.sphere_band_leaves(DIM, min_level, max_level, centers, radii, 0.03)
    return leaves, max_level, cfg, (centers, radii)


def workload_mesh(chns, args):
    """(device mesh, parameters, host state) of the workload chosen by --mesh / --level."""
    if args.mesh in ("layer", "layer_l8"):
        leaves, level, cfg, phase = layer_workload(*((4, 8) if args.mesh == "layer_l8" else (5, 10)))
        gm = chns.Mesh(DIM, level, leaves)
        x = gm.node_x()
        U = np.zeros((gm.N, DIM + 3))
        U[:, DIM + 1] = synth.layer_phi(x, 0.5, 0.05, 1.0, phase, cfg["Cn"])
    elif args.mesh in ("twodrops", "twodrops_l7"):
        leaves, level, cfg, (centers, radii) = twodrops_workload(*((3, 7) if args.mesh == "twodrops_l7" else (4, 9)))
        gm = chns.Mesh(DIM, level, leaves)
        x = gm.node_x()
        U = np.zeros((gm.N, DIM + 3))
        U[:, DIM + 1] = synth.drop_phi(x, centers, radii, cfg["Cn"])
        U[:, :DIM] = synth.fourier_velocity(x, 8, 4, 0.1)
        U[np.any((x <= 0.0) | (x >= 1.0), axis=1), :DIM] = 0.0
    else:
        leaves = synth.uniform_leaves(DIM, args.level)
        gm = chns.Mesh(DIM, args.level, leaves)
        cfg, U = workload_state(gm.node_x())
    return gm, cfg, U


def run_profile(args):
    """One kernel of the hot path, --reps launches, on the chosen mesh."""
    import paper_2009_06628_gb300 as chns
    gm, cfg, U = workload_mesh(chns, args)
    gm.set_scatter(args.scatter)
    prm = chns.Params.make(**cfg)
    U0 = torch.tensor(U, device="cuda")
    Un = U0 + 1e-4 * torch.randn(U0.shape, device="cuda", dtype=torch.float64,
                                 generator=torch.Generator(device="cuda").manual_seed(7))
    x = torch.randn(U0.shape, device="cuda", dtype=torch.float64, generator=torch.Generator(device="cuda").manual_seed(8))
    U0f, Unf, xf = U0.float(), Un.float(), x.float()

    def one():
        if args.profile == "jvp32":
            chns.jvp(gm, prm, U0f, Unf, xf)
        elif args.profile == "jvp64":
            chns.jvp(gm, prm, U0, Un, x)
        elif args.profile == "residual":
            chns.residual(gm, prm, U0, Un)
        else:
            chns.vjp(gm, prm, U0, Un, x)

    one()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        one()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.reps
    print(json.dumps({"profile": args.profile, "mesh": args.mesh, "level": args.level, "elements": gm.E, "nodes": gm.N,
                      "scatter": args.scatter, "colours": gm.num_colours,
                      "avg_ms_per_call": ms, "gdof_s": U0.numel() / (ms * 1e-3) / 1e9}))
    return 0


def run_trajectory(args):
    """--newton-steps mixed Newton steps on the chosen mesh (rel. residual 1e-9 each), with
    the phi integral and the energy parts after every step; the first --fp64-steps are
    repeated in FP64 along their own trajectory, and the per-field relative L2 difference
    mixed vs FP64 (velocity, p, phi, mu) is reported after each of them."""
    import paper_2009_06628_gb300 as chns
    gm, cfg, U = workload_mesh(chns, args)
    prm = chns.Params.make(**cfg)
    d = DIM
    U0 = torch.tensor(U, device="cuda")
    chns.initial_mu(gm, prm, U0)
    dof = U0.numel()
    kw = dict(rtol=1e-9, atol=1e-14, krylov_rtol=1e-3, restart=args.restart, max_krylov=args.max_krylov,
              pc_type=args.pc_type, pc_degree=args.pc_degree or (3 if args.pc_type >= 3 else 16),
              ew_eta0=args.ew_eta0, guess=1 if args.guess == "ptilde" else 0)
    o32 = chns.SolverOpts.make(precision=1, **kw)
    o64 = chns.SolverOpts.make(precision=0, **kw)
    fields = {"v": slice(0, d), "p": slice(d, d + 1), "phi": slice(d + 1, d + 2), "mu": slice(d + 2, d + 3)}
    out = {"run": args.mesh, "elements": gm.E, "nodes": gm.N, "dof": dof, "hanging": gm.H,
           "mass0": chns.mass(gm, U0), "energy0": chns.energy(gm, prm, U0), "steps": []}
    Um, U64 = U0.clone(), U0.clone()
    prev = {"m": None, "64": None}      # U^{k-1} of each trajectory (--guess ptilde)

    def first_iterate(U, key):
        """U^k with the pressure of U^{k-1}: the mid-point pressure continues the previous
        step's (the Crank-Nicolson pressure alternates around it)."""
        if args.guess != "ptilde":
            return None
        G = U.clone()
        if prev[key] is not None:
            G[:, d] = prev[key][:, d]
        return G

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for k in range(args.newton_steps):
        Gm = first_iterate(Um, "m")
        ev[0].record()
        Um_new, st = chns.newton_step(gm, prm, o32, Um, U_out=Gm, check=False)
        ev[1].record()
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1])
        rec = {"step": k + 1, "mixed_ms": ms, "stats": st.as_dict(),
               "gdof_s": dof * st.jvp_calls / (ms * 1e-3) / 1e9,
               "jvp_gdof_s": dof * st.jvp_calls / (st.jvp_ms * 1e-3) / 1e9 if st.jvp_ms > 0 else None,
               "mass": chns.mass(gm, Um_new), "energy": chns.energy(gm, prm, Um_new)}
        rec["mass_drift"] = rec["mass"] - out["mass0"]
        if st.reason != 0:
            out["steps"].append(rec)
            print(json.dumps(rec), flush=True)
            break
        if k < args.fp64_steps:
            G64 = first_iterate(U64, "64")
            ev[2].record()
            U64_new, s64 = chns.newton_step(gm, prm, o64, U64, U_out=G64, check=False)
            ev[3].record()
            torch.cuda.synchronize()
            rec["fp64_ms"] = ev[2].elapsed_time(ev[3])
            rec["fp64_stats"] = s64.as_dict()
            rec["rel_err_mixed_vs_fp64"] = {
                f: float((Um_new[:, sl] - U64_new[:, sl]).norm() / U64_new[:, sl].norm().clamp_min(1e-300))
                for f, sl in fields.items()}
            rec["rel_err_mixed_vs_fp64"]["all"] = float((Um_new - U64_new).norm() / U64_new.norm())
            prev["64"], U64 = U64, U64_new
        prev["m"], Um = Um, Um_new
        out["steps"].append(rec)
        print(json.dumps(rec), flush=True)
    E = [sum(out["energy0"])] + [sum(r["energy"]) for r in out["steps"]]
    out["energy_non_increasing"] = all(b <= a for a, b in zip(E, E[1:]))
    out["max_abs_mass_drift"] = max(abs(r["mass_drift"]) for r in out["steps"])
    print(json.dumps({k: v for k, v in out.items() if k != "steps"}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-kernels", action="store_true", help="skip the per-kernel table")
    ap.add_argument("--profile", choices=["jvp32", "jvp64", "residual", "vjp"],
                    help="run only this kernel --reps times on a uniform mesh of --level (for ncu)")
    ap.add_argument("--level", type=int, default=LEVEL)
    ap.add_argument("--mesh", choices=["uniform", "twodrops", "twodrops_l7", "layer", "layer_l8"], default="uniform")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--scatter", type=int, default=0, choices=[0, 1, 2],
                    help="element scatter for --profile: 0 atomics, 1 colouring, 2 warp-aggregated")
    ap.add_argument("--run", action="store_true",
                    help="multi-step Newton run on --mesh (mixed, and FP64 for --fp64-steps) instead of the bench")
    ap.add_argument("--newton-steps", type=int, default=5)
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--max-krylov", type=int, default=5000)
    ap.add_argument("--guess", choices=["old", "ptilde"], default="old",
                    help="--run: first Newton iterate U^k, or U^k with the pressure of U^{k-1}")
    ap.add_argument("--ew-eta0", type=float, default=0.0,
                    help="--run: Eisenstat-Walker forcing from this first tolerance (0: fixed krylov_rtol)")
    ap.add_argument("--pc-type", type=int, default=None,
                    help="preconditioner (default: 1 for the bench step and --run)")
    ap.add_argument("--pc-degree", type=int, default=None,
                    help="Chebyshev degree (default 16 for pc_type 1/2, 3 for the multigrid smoother of 3/4)")
    args = ap.parse_args()
    if args.pc_type is None:
        args.pc_type = BENCH_PC_TYPE
    if args.profile:
        return run_profile(args)
    if args.run:
        return run_trajectory(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    import paper_2009_06628_gb300 as chns
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    leaves = synth.uniform_leaves(DIM, LEVEL)
    gm = chns.Mesh(DIM, LEVEL, leaves)
    cfg, U = workload_state(gm.node_x())
    prm = chns.Params.make(**cfg)
    U0 = torch.tensor(U, device=dev)
    chns.initial_mu(gm, prm, U0)
    dof = U0.numel()
    pc_kw = dict(pc_type=args.pc_type, pc_degree=args.pc_degree or (3 if args.pc_type >= 3 else 16))
    opts = chns.SolverOpts.make(rtol=1e-9, atol=1e-14, krylov_rtol=1e-3, precision=1, restart=30, max_krylov=2000,
                                **pc_kw)
    U1 = torch.empty_like(U0)
    # clock samples cover the warm-up and the timed region (the sampler starts before both)
    clocks = ClockSampler(local)
    fp32_peak = chns.fma_peak(1, 20000) / 1e12
    fp64_peak = chns.fma_peak(0, 2000) / 1e12
    for _ in range(args.warmup):
        chns.newton_step(gm, prm, opts, U0, U1)
    torch.cuda.synchronize()

    # ---- timed region: K mixed Newton steps from the same U^k ----
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = chns.kernel_launches()
    torch.cuda.nvtx.range_push("timed")
    ev0.record(stream)
    jvp_calls, jvp_ms, stats = 0, 0.0, []
    for _ in range(args.steps):
        _, st = chns.newton_step(gm, prm, opts, U0, U1)
        jvp_calls += st.jvp_calls
        jvp_ms += st.jvp_ms
        stats.append(st.as_dict())
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = chns.kernel_launches() - launches0
    clk = clocks.stop()
    mass_drift = chns.mass(gm, U1) - chns.mass(gm, U0)
    t_ms, total_jvp = aggregate_replicas(ev0.elapsed_time(ev1), float(jvp_calls), dist, dev)
    value = dof * total_jvp / (t_ms * 1e-3) / 1e9

    # ---- end to end through the public API with host buffers ----
    host_in = torch.tensor(U0.cpu().numpy()).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    Ud = torch.empty_like(U0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_jvp = 0
    for _ in range(args.steps):
        Ud.copy_(host_in, non_blocking=True)
        out, st = chns.newton_step(gm, prm, opts, Ud, U1)
        host_out.copy_(out, non_blocking=True)
        e2e_jvp += st.jvp_calls
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e_value = dof * e2e_jvp * world / (e2e_ms * 1e-3) / 1e9

    # ---- FP64 Newton step on the same problem, and the mixed step's error against it ----
    newton = {"mixed_ms": t_ms / args.steps, "mixed_stats": stats[-1], "mixed_mass_drift": mass_drift}
    if not args.no_fp64:
        o64 = chns.SolverOpts.make(rtol=1e-9, atol=1e-14, krylov_rtol=1e-3, precision=0, restart=30, max_krylov=2000,
                                   **pc_kw)
        U64 = torch.empty_like(U0)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        _, s64 = chns.newton_step(gm, prm, o64, U0, U64)
        f1.record(stream)
        torch.cuda.synchronize()
        # the same step with the multigrid pressure preconditioner (pc_type 3, smoother degree 2)
        omg = chns.SolverOpts.make(rtol=1e-9, atol=1e-14, krylov_rtol=1e-3, precision=1, restart=30,
                                   max_krylov=2000, pc_type=3, pc_degree=2)
        Umg = torch.empty_like(U0)
        chns.newton_step(gm, prm, omg, U0, Umg)          # builds the hierarchy (untimed)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        _, smg = chns.newton_step(gm, prm, omg, U0, Umg)
        g1.record(stream)
        torch.cuda.synchronize()
        newton["mixed_multigrid"] = {"ms": g0.elapsed_time(g1), "krylov_its": smg.krylov_its,
                                     "jvp_calls": smg.jvp_calls, "apply_ms": smg.apply_ms,
                                     "rel_err_vs_fp64": float((Umg - U64).norm() / U64.norm())}
        newton.update({"fp64_ms": f0.elapsed_time(f1), "fp64_stats": s64.as_dict(),
                       "fp64_mass_drift": chns.mass(gm, U64) - chns.mass(gm, U0),
                       "rel_err_mixed_vs_fp64": float((U1 - U64).norm() / U64.norm()),
                       "speedup_mixed_vs_fp64": f0.elapsed_time(f1) / (t_ms / args.steps)})

    pk = peaks()
    kernels = kernel_table(chns, gm, prm, U0, pk, fp32_peak, fp64_peak) if not args.no_kernels else None
    E = gm.E
    jvp_avg_ms = jvp_ms / max(jvp_calls, 1)
    hbm_bytes = 4 * dof * 4 + E * (8 * 4 + 1)      # read U^k, U^s, x; write y; e2n + level
    cnt = counts_for("jvp_fp32")
    roof = {"bound": "alu", "unit": "TFLOP/s", "peak": fp32_peak,
            "peak_source": "measured in this run: chns_fma_peak FP32 (FFMA chains on all SMs, CUDA events)",
            "traffic": cnt.get("dram_bytes") if cnt else None,
            "flop_per_element": cnt["flop_per_element"] if cnt else None}
    if cnt:
        ach = cnt["flop_per_element"] * E / (jvp_avg_ms * 1e-3) / 1e12
        roof.update({"achieved": ach, "frac": ach / fp32_peak})
    else:
        roof.update({"achieved": None, "frac": None})
    hbm = {"algorithmic_bytes_per_launch": hbm_bytes, "achieved_gbs": hbm_bytes / (jvp_avg_ms * 1e-3) / 1e9,
           "peak_gbs": pk.get("hbm_gbs"), "frac": hbm_bytes / (jvp_avg_ms * 1e-3) / 1e9 / pk.get("hbm_gbs", 6800.0),
           "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}
    line = {"metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "elements": E, "nodes": gm.N, "dof": dof,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "preconditioner": pc_kw,
                       "l2": "inputs larger than L2 (GMRES basis 31 x 13.2 MB FP64, J x operands 26 MB, per step)"},
            "jvp_kernel": {"avg_ms": jvp_avg_ms, "launches": jvp_calls, "gdof_s": dof / (jvp_avg_ms * 1e-3) / 1e9},
            "roofline": roof, "hbm": hbm, "newton": newton, "clocks": clk, "gpu_launches": launches,
            "alu_peaks_tflops": {"fp32": fp32_peak, "fp64": fp64_peak, "source": "chns_fma_peak, this run"},
            "kernels": kernels,
            "e2e": {"value": e2e_value, "unit": "GDOF/s", "h2d_bytes_per_step": dof * 8,
                    "d2h_bytes_per_step": dof * 8}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_oracle()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
