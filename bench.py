"""Benchmark of the reduced-order Newton / FETI-DP hot path on one GB300.

Headline workload (default ``--case strut20``): the 3D lattice of 20 x 20 x 20 edge-strut cells
(each a 12^3 voxel grid of trilinear Q1 hexes keeping the voxels whose centre lies within 0.15 of
a cube edge: 344 elements, 880 nodes, 2 640 local DOF), 13 736 163 DOF, compressible neo-Hookean
mu = 1, lam = 4, per-cell shear-modulus factors theta_s ~ U[0.9, 1.1] (seed 4), bottom clamped,
top displaced -20 % in 20 steps; BF16 principal blocks (tcgen05, FP32 accumulation) in the
preconditioner, FP32 reduced tangent action inside the inner Krylov solve, FP64 residual, outer
operator and Newton update.  Load step 1 is solved untimed; a benchmark step is then one full
Newton iteration from the predictor of load step 2 (all rows of the hot path: gather, residual,
reduced-rule snapshots, greedy, coefficients, principal tangents, FETI-DP setup, FGMRES with the
reduced tangent action, Armijo line search, update).  Every step starts from the same state, so
every step does the same work.

``value`` is the metric's first quantity, the reduced tangent-apply throughput: stacked local
DOF (n_loc x N_s) per second of the FP32 reduced tangent action kernels (FP64 in FP64 mode) that
ran inside the timed Newton iterations, from CUDA events around each launch on the library's
stream.  ``ms_per_step`` is the Newton iteration.  The metric's second quantity, the Newton-step
time against the plain FP64 full-tangent GPU path at equal accuracy, is measured per load step
on the 32 x 32 ring lattice (where the plain path's 1 024 local inverses fit; on the strut20
lattice they would need 442 GB) and reported under ``vs_plain_fp64``.

One compact JSON line is printed last; ``--detail PATH`` writes the full breakdown (per-kernel
times and rooflines, sweeps) to a file.

``--impl reference`` times the FP64 CPU oracle on the host cores on the same metric: each step
is one oracle reduced tangent action (dense principal matrices times the cell vectors of a
bounded sample of the same lattice's cells, at the same state and with the oracle's own greedy
on the sample).
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
sys.path.insert(0, ROOT)

METRIC = "reduced tangent-apply GDOF/s & Newton-step time vs plain FP64 GPU path, 1 GB300"
WORKLOADS = {
    "strut20": "strut20: 3D 20x20x20 edge-strut cells (12^3 voxels, strut half-width 0.15), 344 Q1 hex per cell, "
               "13736163 DOF, theta~U[0.9,1.1] seed 4, mu=1 lam=4, -20% in 20 steps",
    "strut10": "strut10: 3D 10x10x10 edge-strut cells (12^3 voxels, strut half-width 0.15), 344 Q1 hex per cell, "
               "1760583 DOF, mu=1 lam=4, -15% in 15 steps",
    "ring32": "ring32: 2D 32x32 ring cells (hole r=0.3), 16x16 Q1 per cell, 556034 DOF, theta~U[0.9,1.1] seed 2, "
              "mu=1 lam=4, -20% in 20 steps",
}
DEFAULT_PRECISION = {"strut20": "bf16", "strut10": "fp32", "ring32": "fp32"}

# FP64 and FP32 CUDA-core peaks are not in the measured-peaks file: unit counts and clocks
FP64_PEAK_TFLOPS = 1.25      # GB300 FP64 (recipe table); 1.20 measured with an FMA loop
FP32_PEAK_TFLOPS = 80.5      # 152 SM x 128 FP32 lanes x 2 flop x 2.07 GHz


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--case", default="strut20", choices=sorted(WORKLOADS))
    p.add_argument("--precision", default=None, choices=["fp64", "fp32", "bf16"],
                   help="fp32 / bf16: mixed modes (FP32 reduced action in the inner Krylov solve, FP32 or BF16 "
                        "preconditioner blocks, FP64 residual and outer operator)")
    p.add_argument("--state-step", type=int, default=1, help="load steps solved before the timed iterations")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--quick", action="store_true", help="skip the plain-path comparison and the extras")
    p.add_argument("--detail", default=None, help="write the full breakdown as JSON to this path")
    p.add_argument("--sample-cells", type=int, default=512, help="cells in the oracle's bounded sample")
    p.add_argument("--profile-step", action="store_true",
                   help="bracket one more Newton iteration (after the timed region) with cudaProfilerStart/Stop, "
                        "for a profiler started with --profile-from-start off")
    args = p.parse_args()
    if args.precision is None:
        args.precision = DEFAULT_PRECISION[args.case]
    return args


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), \
            "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self, dev_index=0):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 9 and r[0].strip() == str(dev_index)]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = max(float(r[2]) for r in rows)
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(rows)}


def dist_init(args):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif args.impl == "ours":
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x, dev=None):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def threads_in_use():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info()]
        return max(n) if n else 1
    except Exception:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------------------------
# the oracle's reduced tangent action on a bounded sample (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------------------------
def oracle_apply_fn(case_name, load_step, n_sample):
    """One oracle reduced tangent action Y = sum_r alpha_r K^r X on a bounded sample of the
    lattice's cells: the first n_sample cells (cell order, x fastest), at the affine predictor of
    load step ``load_step``; principals and alpha from the oracle's greedy on the sample's
    snapshots (tolerance of the case), dense principal matrices.  Returns (fn, stacked DOF of
    the sample, description)."""
    import numpy as np

    import latgen
    from oracle import cell as OC
    from oracle import greedy as OG
    from oracle import newton as ON
    from oracle import rom as OR
    from oracle.assembly import Problem
    case = latgen.make_case(case_name)
    prob = Problem(case)
    u = ON.predictor(prob, load_step, None, None)
    n = min(n_sample, prob.lat.n_cells)
    ul = prob.local(u)[:n]
    mu = prob.mu_cells[:n]
    T = OC.snapshots(prob.cell, ul, mu, prob.lam)
    g = OG.greedy(T, case.eps, 256)
    alpha = OG.alpha_triangular(T, g)
    Kp = OC.tangent(prob.cell, ul[g.S], mu[g.S], prob.lam)
    X = latgen.uniform_field((prob.cell.n_nodes * prob.d, n), 7)

    def step():
        return OR.reduced_apply(prob.cell, Kp, alpha, X)

    desc = ("oracle reduced action (numpy, %d dense principals), first %d cells of %s, predictor of step %d"
            % (len(g.S), n, case_name, load_step))
    return step, prob.cell.n_nodes * prob.d * n, desc


def run_reference(args):
    ws, rank, _ = dist_init(args)
    if rank != 0:
        barrier(ws)
        return 0
    step, stacked, desc = oracle_apply_fn(args.case, args.state_step + 1, args.sample_cells)
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = stacked * args.steps / dt / 1e9
    cores = threads_in_use()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.case], "step": desc},
        "cpu_baseline": {"value": value, "unit": "GDOF/s", "cores": cores, "kind": "oracle",
                         "sample": "%d oracle reduced tangent actions; %s" % (args.steps, desc)},
        "e2e": {"value": value, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    barrier(ws)
    return 0


def cpu_baseline(args, seconds=10.0):
    step, stacked, desc = oracle_apply_fn(args.case, args.state_step + 1, args.sample_cells)
    step()
    n, t0 = 0, time.perf_counter()
    while True:
        step()
        n += 1
        dt = time.perf_counter() - t0
        if dt >= seconds:
            break
    return {"value": stacked * n / dt / 1e9, "unit": "GDOF/s", "cores": threads_in_use(), "kind": "oracle",
            "sample": "%d calls, %.1f s: %s" % (n, dt, desc)}


# ---------------------------------------------------------------------------------------------
# work models for the roofline entries
# ---------------------------------------------------------------------------------------------
KERNELS = ["residual", "tangent_full", "tangent_material", "tangent_reduced", "greedy_update", "apply_reduced",
           "apply_reduced_fp32", "apply_percell", "apply_percell_fp32", "local_segmm", "local_gemv", "local_tc",
           "gj_update", "gj_pivot", "densify", "phi_schur", "coarse_blocked", "coarse_gemv", "coarse_solve",
           "local_segmm_dual", "local_gemv_dual", "local_tc_dual", "local_segmm_dual_in", "local_gemv_dual_in",
           "local_tc_dual_in", "dual_schur", "dual_schur_tc", "krylov_orth"]


def kernel_work(name, s, n_r, mixed):
    """Algorithmic work per launch and its roofline kind.

    local_* : principal-block x cell-multivector products, 2 (n_R + n_P) n_R flops per cell
        (whole block), 2 (n_D + n_P) n_D (*_dual, inside the interface solve), 2 (n_R + n_P) n_D
        (*_dual_in); local_tc on the tensor cores (BF16), the others on the CUDA cores in the
        mode's precision;
    dual_schur: Dirichlet interface preconditioner, 2 n_D^2 flops per cell;
    apply_reduced(_fp32): Eq. romstiffnessmatrix, HBM bytes b (2 n_loc N_s + N_r N_s + N_r nnz)
        (X and Y streamed once, alpha and the principal values read once), b = 4 or 8;
    apply_percell: the plain path, b nnz N_s + 2 b n_loc N_s bytes;
    coarse_solve: block-LU solve of the block-tridiagonal coarse matrix (N blocks of size m),
        2 (3 N - 2) m^2 FP64 flops (FP64 ALU bound), or in the mixed modes the FP32 factor copies
        streamed once, 4 (3 N - 2) m^2 bytes (HBM bound); coarse_gemv: the explicit coarse
        inverse, 2 n_primal^2 FP64 flops (FP32 copy in the mixed modes: 4 n_primal^2 bytes).
    """
    n_s, n_loc, nnz = s.n_cells, s.n_loc, s.nnz
    n_rr, n_p = s.n_r_local, s.n_p_local
    n_d = n_rr - s.n_i_local
    tc = name.startswith("local_tc")
    unit = "tensor" if tc else "alu"
    if name in ("local_segmm", "local_gemv", "local_tc"):
        return 2.0 * (n_rr + n_p) * n_rr * n_s, unit
    if name in ("local_segmm_dual", "local_gemv_dual", "local_tc_dual"):
        return 2.0 * (n_d + n_p) * n_d * n_s, unit
    if name in ("local_segmm_dual_in", "local_gemv_dual_in", "local_tc_dual_in"):
        return 2.0 * (n_rr + n_p) * n_d * n_s, unit
    if name == "dual_schur":
        return 2.0 * n_d * n_d * n_s, "alu"
    if name == "dual_schur_tc":
        return 2.0 * n_d * n_d * n_s, "tensor"
    if name in ("apply_reduced", "apply_reduced_fp32") and n_r:
        b = 4.0 if name.endswith("fp32") else 8.0
        return b * (2.0 * n_loc * n_s + n_r * n_s + n_r * nnz), "hbm"
    if name in ("apply_percell", "apply_percell_fp32"):
        b = 4.0 if name.endswith("fp32") else 8.0
        return b * nnz * n_s + 2 * b * n_loc * n_s, "hbm"
    if name == "coarse_solve" and s.n_coarse_blocks:
        nb, mb = s.n_coarse_blocks, s.coarse_block
        if mixed:
            # FP32 copies of the factors U_i, U_i^T (N - 1 blocks each) and D_i^-1 (N blocks), each
            # streamed once per solve
            return 4.0 * (3 * nb - 2) * mb * mb, "hbm"
        return 2.0 * (3 * nb - 2) * mb * mb, "fp64"
    if name == "coarse_gemv":
        if mixed:
            return 4.0 * s.n_primal * s.n_primal + 16.0 * s.n_primal, "hbm"
        return 2.0 * s.n_primal * s.n_primal, "fp64"
    return None, None


def roofline_entry(name, k, s, n_r, precision, hbm_peak, bf16_peak, peak_src):
    work, kind = kernel_work(name, s, n_r, precision != "fp64")
    if work is None:
        return None
    avg_s = k["avg_us"] * 1e-6
    if kind == "hbm":
        ach = work / avg_s / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "peak_source": "%s copy bandwidth" % peak_src, "work_per_launch": work,
                "avg_us": k["avg_us"], "launches": k["launches"], "share": k.get("share")}
    if kind == "tensor":
        peak, src = bf16_peak, "%s bf16 tensor (sustained)" % peak_src
    elif kind == "fp64" or precision == "fp64":
        peak, src = FP64_PEAK_TFLOPS, "FP64 ALU, recipe table (1.20 measured with an FMA loop)"
    else:
        peak, src = FP32_PEAK_TFLOPS, "FP32 ALU, 152 SM x 128 lanes x 2 x 2.07 GHz"
    ach = work / avg_s / 1e12
    return {"kernel": name, "bound": "tensor" if kind == "tensor" else "alu", "achieved": ach, "peak": peak,
            "unit": "TFLOP/s", "frac": ach / peak, "peak_source": src, "work_per_launch": work,
            "avg_us": k["avg_us"], "launches": k["launches"], "share": k.get("share")}


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture, with
# the summary that holds the command, keyed by (case, precision, kernel); an entry is removed
# when its kernel changes
MEASURED_TRAFFIC = {}


# ---------------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__ as g
    g.build()
    import latgen
    from paper_2603_10741_gb300 import LAT_FP64, LAT_MIXED_BF16, LAT_MIXED_FP32, Lattice

    ws, rank, local = dist_init(args)
    dev = torch.device("cuda", torch.cuda.current_device())
    # the tensor-core product runs inside a seconds-long step: the sustained BF16 peak
    hbm_peak, _, bf16_peak, peak_src = peaks()
    prec = {"fp64": LAT_FP64, "fp32": LAT_MIXED_FP32, "bf16": LAT_MIXED_BF16}[args.precision]
    case = latgen.make_case(args.case)
    stream = torch.cuda.current_stream()
    detail = {}

    # state: converged load steps 1..state_step (untimed), then the predictor of the next step
    lat = Lattice.from_case(case, prec)
    opts = lat.lattice_default_opts()
    u1 = u2 = None
    t0 = time.perf_counter()
    for k in range(1, args.state_step + 1):
        u = lat.lattice_predictor(case.top_displacement(k), u1, u2)
        rep = lat.newton_step(u, opts)
        if not rep.converged:
            raise RuntimeError(f"load path failed at step {k}: {rep.as_dict()}")
        detail.setdefault("load_path", []).append(rep.as_dict())
        u2, u1 = u1, u
    detail["load_path_s"] = time.perf_counter() - t0
    u_start = lat.lattice_predictor(case.top_displacement(args.state_step + 1), u1, u2).clone()
    torch.cuda.synchronize()
    s = lat.sizes
    stacked = s.n_loc * s.n_cells
    apply_name = "apply_reduced" if args.precision == "fp64" else "apply_reduced_fp32"

    u = torch.empty_like(u_start)
    for _ in range(args.warmup):
        u.copy_(u_start)
        lat.newton_step(u, opts, max_iterations=1)
    torch.cuda.synchronize()
    barrier(ws)
    # timed region: K Newton iterations, CUDA events on the library's stream; the tangent-action
    # launches inside are bracketed by events too (timing mode 2 keeps the interface solve's
    # CUDA-graph replays)
    lat.lattice_set_timing(2)
    clocks = Clocks()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    reps = []
    e0.record(stream)
    for _ in range(args.steps):
        u.copy_(u_start)
        reps.append(lat.newton_step(u, opts, max_iterations=1).as_dict())
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop(local)
    barrier(ws)
    ms_step = max_over_ranks(ws, e0.elapsed_time(e1), dev) / args.steps
    t_apply, n_apply = lat.lattice_kernel_time(apply_name)
    lat.lattice_set_timing(0)
    apply_s = max_over_ranks(ws, t_apply * 1e-3, dev)
    value = ws * stacked * n_apply / apply_s / 1e9 if n_apply else 0.0
    n_launch = count_launches(lat, opts, u_start)

    if args.profile_step:
        u.copy_(u_start)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        lat.newton_step(u, opts, max_iterations=1)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    # per-kernel breakdown of one more iteration (every named kernel timed)
    lat.lattice_set_timing(1)
    u.copy_(u_start)
    rep_t = lat.newton_step(u, opts, max_iterations=1).as_dict()
    torch.cuda.synchronize()
    kt = {}
    for kname in KERNELS:
        t, n = lat.lattice_kernel_time(kname)
        if n:
            kt[kname] = {"total_ms": t, "launches": n, "avg_us": 1e3 * t / n}
    lat.lattice_set_timing(0)
    tot = sum(v["total_ms"] for v in kt.values())
    for v in kt.values():
        v["share"] = v["total_ms"] / tot if tot else None
    s = lat.sizes
    n_r = reps[-1]["n_r_last"]
    rl = [e for e in (roofline_entry(k, v, s, n_r, args.precision, hbm_peak, bf16_peak, peak_src)
                      for k, v in sorted(kt.items(), key=lambda kv: -kv[1]["total_ms"])) if e]
    detail["kernels"] = kt
    detail["kernel_rooflines"] = rl
    detail["timed_iteration_reports"] = reps
    # the dominant kernel: the timers that bracket one launch each, with the four views of the
    # tensor-core product (one kernel, k_local_tc) taken together; the coarse solve (a chain of
    # launches whose host-side issue the per-launch timers stretch) is reported in the detail
    roof = dominant_kernel(rl)
    if roof:
        tr = MEASURED_TRAFFIC.get((args.case, args.precision, roof["kernel"]))
        roof["traffic"] = tr[0] if tr else None
        if tr:
            roof["traffic_source"] = tr[1]
    apply_roof = next((dict(e) for e in rl if e["kernel"] == apply_name), None)
    if apply_roof and n_apply:
        # the same work model over the timed region's launches
        apply_roof["achieved"] = apply_roof["work_per_launch"] * n_apply / apply_s / 1e9
        apply_roof["frac"] = apply_roof["achieved"] / hbm_peak
        apply_roof["avg_us"] = apply_s / n_apply * 1e6
        apply_roof["launches"] = n_apply

    out = {
        "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f64+f32", "bf16": "f64+f32+bf16"}[args.precision],
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.case],
                   "precision": {"fp64": "FP64 reduced (EIM) path",
                                 "fp32": "FP32 action (inner Krylov) and preconditioner; FP64 residual, "
                                         "outer operator, update",
                                 "bf16": "FP32 action (inner Krylov), BF16-pair preconditioner blocks; FP64 "
                                         "residual, outer operator, update"}[args.precision],
                   "step": "one Newton iteration (all hot-path rows) from the predictor of load step %d"
                           % (args.state_step + 1),
                   "value": "%s: n_loc*N_s DOF/s over its %d launches in the timed iterations"
                            % (apply_name, n_apply),
                   "l2": "inputs larger than L2: cell vectors %.0f MB each, FGMRES bases %.0f MB"
                         % (4 * stacked / 1e6, 8.0 * (2 * opts.krylov_restart + 2 * opts.inner_its + 3) * s.n_krylov
                            / 1e6),
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "roofline": roof,
        "apply_roofline": apply_roof,
        "newton": {"ms_per_iteration": ms_step, "global_gdofs": ws * s.n_dof / (ms_step * 1e-3) / 1e9,
                   "n_r": n_r, "krylov_its": reps[-1]["krylov_its_total"],
                   "inner_its": reps[-1]["inner_its_total"], "pcg_its": reps[-1]["pcg_its_total"],
                   "enrich_level": reps[-1]["enrich_level"]},
        "gpu_launches": n_launch * args.steps,
        "clocks": ck,
    }
    # end to end through host buffers: the same metric through apply_reduced_tangent, with the
    # H2D copy of the cell vector from pinned memory and the D2H copy of the result per step
    out["e2e"] = bench_e2e(lat, args, ws, dev, u_start, stacked, args.precision)
    if not args.quick and rank == 0:
        detail["vs_plain_fp64"] = plain_vs_reduced("ring32", 1)
        out["vs_plain_fp64"] = vs_plain_summary(detail["vs_plain_fp64"])
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
    lat.close()
    if rank == 0:
        if args.detail:
            detail["line"] = out
            with open(args.detail, "w") as f:
                json.dump(detail, f, indent=1, default=str)
        print(json.dumps(compact(out)))
    return 0


TC_VIEWS = ("local_tc", "local_tc_dual", "local_tc_dual_in", "dual_schur_tc")
SINGLE_LAUNCH = TC_VIEWS + ("apply_reduced", "apply_reduced_fp32", "apply_percell", "apply_percell_fp32",
                            "residual", "local_segmm", "local_segmm_dual", "local_segmm_dual_in", "local_gemv",
                            "local_gemv_dual", "local_gemv_dual_in", "dual_schur", "gj_update", "coarse_gemv")


def dominant_kernel(rl):
    """Roofline entry of the kernel with the largest total time (tensor-core views combined)."""
    tc = [e for e in rl if e["kernel"] in TC_VIEWS]
    cand = [dict(e) for e in rl if e["kernel"] in SINGLE_LAUNCH and e["kernel"] not in TC_VIEWS]
    if tc:
        launches = sum(e["launches"] for e in tc)
        total_us = sum(e["avg_us"] * e["launches"] for e in tc)
        work = sum(e["work_per_launch"] * e["launches"] for e in tc) / launches
        ach = work / (total_us / launches * 1e-6) / 1e12
        cand.append({"kernel": "k_local_tc (" + ", ".join(e["kernel"] for e in tc) + ")", "bound": "tensor",
                     "achieved": ach, "peak": tc[0]["peak"], "unit": "TFLOP/s", "frac": ach / tc[0]["peak"],
                     "peak_source": tc[0]["peak_source"], "work_per_launch": work, "avg_us": total_us / launches,
                     "launches": launches, "share": sum(e["share"] or 0 for e in tc),
                     "issued_frac": 3 * ach / tc[0]["peak"]})
    if not cand:
        return None
    for e in cand:
        e["_total"] = e["avg_us"] * e["launches"]
    best = max(cand, key=lambda e: e["_total"])
    best.pop("_total", None)
    return best


def compact(out):
    """Round floats so that the final line stays short."""
    def r(x):
        if isinstance(x, float):
            return float("%.5g" % x)
        if isinstance(x, dict):
            return {k: r(v) for k, v in x.items() if v is not None or k in ("vs_baseline", "traffic")}
        if isinstance(x, list):
            return [r(v) for v in x]
        return x
    return r(out)


def count_launches(lat, opts, u_start):
    """Kernels the library launches in one step (its own launch counter, copies excluded)."""
    u = u_start.clone()
    n0 = lat.lattice_launch_count()
    lat.newton_step(u, opts, max_iterations=1)
    return lat.lattice_launch_count() - n0


def bench_e2e(lat, args, ws, dev, u_start, stacked, precision):
    import torch
    sel = lat.select_principal_cells(u_start, lat.lattice_default_opts().eps, 256)
    dt = torch.float64 if precision == "fp64" else torch.float32
    s = lat.sizes
    host_x = torch.rand((s.n_loc, s.n_cells), dtype=dt).pin_memory()
    host_y = torch.empty_like(host_x).pin_memory()
    x = torch.empty(host_x.shape, dtype=dt, device=dev)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        x.copy_(host_x, non_blocking=True)
        lat.apply_reduced_tangent(x, y)
        host_y.copy_(y, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(args.steps, 10)
    e0.record(stream)
    for _ in range(reps):
        x.copy_(host_x, non_blocking=True)
        lat.apply_reduced_tangent(x, y)
        host_y.copy_(y, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(ws, e0.elapsed_time(e1), dev) / reps
    nb = host_x.numel() * host_x.element_size()
    return {"value": ws * stacked / (ms * 1e-3) / 1e9, "unit": "GDOF/s", "ms_per_step": ms,
            "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb, "n_r": sel["n_r"],
            "what": "apply_reduced_tangent, X from pinned host memory and Y back every call"}


def vs_plain_summary(vp):
    """The line's short form of plain_vs_reduced's result (the full one goes to --detail)."""
    paths = ("plain_fp64", "reduced_fp64", "reduced_mixed_fp32")
    return {"workload": vp["workload"].split(":")[0] + " load step %d, each path to newton_rtol 1e-8" % vp["load_step"],
            "ms_per_load_step": {p: vp[p]["ms_per_load_step"] for p in paths},
            "converged": all(vp[p]["converged"] for p in paths),
            "speedup_reduced_fp64": vp["speedup_reduced_fp64"], "speedup_reduced_mixed": vp["speedup_reduced_mixed"]}


def plain_vs_reduced(case_name, load_step):
    """Newton-step time at equal accuracy: one load step from its predictor to newton_rtol 1e-8,
    the reduced FP64 path against the plain FP64 full-tangent path (every cell principal, exact
    local inverses), both through newton_step on the same GPU; final relative residuals and
    iteration counts beside the times."""
    import torch
    import latgen
    from paper_2603_10741_gb300 import LAT_FP64, LAT_MIXED_FP32, Lattice
    case = latgen.make_case(case_name)
    res = {"workload": WORKLOADS.get(case_name, case_name), "load_step": load_step}
    for tag, prec, force in (("reduced_fp64", LAT_FP64, 0), ("plain_fp64", LAT_FP64, 1),
                             ("reduced_mixed_fp32", LAT_MIXED_FP32, 0)):
        lat = Lattice.from_case(case, prec)
        opts = lat.lattice_default_opts(force_all=force)
        u0 = lat.lattice_predictor(case.top_displacement(load_step))
        u = torch.empty_like(u0)
        u.copy_(u0)
        lat.newton_step(u, opts)            # warm-up (allocations, graph capture)
        torch.cuda.synchronize()
        u.copy_(u0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rep = lat.newton_step(u, opts)
        e1.record()
        torch.cuda.synchronize()
        res[tag] = {"ms_per_load_step": e0.elapsed_time(e1), "newton_its": rep.iterations,
                    "rel_residual": rep.r_norm / rep.r0_norm, "converged": bool(rep.converged),
                    "krylov_its": rep.krylov_its_total}
        lat.close()
        torch.cuda.empty_cache()
    res["speedup_reduced_fp64"] = res["plain_fp64"]["ms_per_load_step"] / res["reduced_fp64"]["ms_per_load_step"]
    res["speedup_reduced_mixed"] = res["plain_fp64"]["ms_per_load_step"] / res["reduced_mixed_fp32"]["ms_per_load_step"]
    return res


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
