"""Benchmark: one Newton iteration of the reduced-order FETI-DP hot path on one GB300.

Workload: the 2D lattice of 32 x 32 ring cells (unit squares with a central hole r = 0.3), 16 x 16
mapped Q1 quads per cell, 556 034 DOF, per-cell shear modulus factors theta_s ~ U[0.9, 1.1]
(seed 2), plane-strain neo-Hookean mu = 1, lam = 4, bottom clamped, top displaced -20 % in 20
steps.  The load path is run on the GPU up to load step ``--state-step`` (untimed); a step of
the benchmark is then one full Newton iteration from the predictor of the next load step:
residual, snapshots + greedy + coefficients, principal tangents, FETI-DP preconditioner setup,
FGMRES with the reduced tangent, Armijo line search and update.  Every step starts from the same
state, so every step does the same work.

Reported: the reduced path in FP64 (the headline), the plain FP64 full-tangent path (every cell
principal, exact local solves) and the mixed FP32 reduced path on the same state; the reduced
tangent action alone (GDOF/s, FP64 and FP32, L2 flushed between calls); per-kernel times from
CUDA events on the library's stream; an end-to-end number through host buffers; the FP64 CPU
oracle on a bounded sample; clocks sampled during the timed region.

``--impl reference`` times the oracle (plain FP64 numpy/scipy Newton iteration with sparse LU)
on the host cores instead: each step is one oracle Newton iteration on the same lattice.
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
WORKLOAD = ("ring32: 2D 32x32 ring cells (hole r=0.3), 16x16 Q1 per cell, 556034 DOF, "
            "theta~U[0.9,1.1] seed 2, mu=1 lam=4, -20% in 20 steps")

# peaks: measured copy bandwidth / bf16 GEMM (driver file), FP64/FP32 ALU from unit counts
FP64_PEAK_TFLOPS = 1.25      # GB300 FP64 (recipe table); 1.20 measured with an FMA loop
FP32_PEAK_TFLOPS = 80.5      # 152 SM x 128 FP32 lanes x 2 flop x 2.07 GHz


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--case", default="ring32")
    p.add_argument("--state-step", type=int, default=10)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--quick", action="store_true", help="skip the full-path and mixed comparisons")
    p.add_argument("--profile-region", default="headline", choices=["headline", "apply"],
                   help="region bracketed by cudaProfilerStart/Stop (for --profile-from-start off)")
    p.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "bf16"],
                   help="precision of the headline leg (fp32/bf16: mixed modes, FP64 Krylov operator)")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    return 6800.0, 1900.0, "fallback"


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


# ---------------------------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle
# ---------------------------------------------------------------------------------------------
def oracle_step_fn(case_name, state_step):
    """One oracle Newton iteration (residual, assembled tangent, sparse LU, Armijo) from the
    affine predictor of load step state_step+1; returns (fn, n_dof)."""
    import numpy as np
    import scipy.sparse.linalg as spla

    import latgen
    from oracle import newton as ON
    from oracle.assembly import Problem
    case = latgen.make_case(case_name)
    prob = Problem(case)
    u0 = ON.predictor(prob, state_step + 1, None, None)

    def step():
        r = prob.residual(u0)
        K = prob.tangent(u0)
        free = prob.free
        du = spla.splu(K[free][:, free].tocsc()).solve(-r[free])
        rn = np.linalg.norm(r[free])
        for m in range(31):
            t = 0.5 ** m
            ut = u0.copy()
            ut[free] += t * du
            if prob.min_jacobian(ut) > 0 and np.linalg.norm(prob.residual(ut)[free]) <= (1 - 1e-4 * t) * rn:
                break
        return ut

    return step, prob.n_dof


def threads_in_use():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info()]
        return max(n) if n else 1
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    ws, rank, _ = dist_init(args)
    if rank != 0:
        barrier(ws)
        return 0
    step, n_dof = oracle_step_fn(args.case, args.state_step)
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = n_dof * args.steps / dt / 1e9
    cores = threads_in_use()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "step": "one oracle Newton iteration (residual, assembled tangent, "
                   "sparse LU solve, Armijo) from the affine predictor of load step %d" % (args.state_step + 1)},
        "cpu_baseline": {"value": value, "unit": "GDOF/s", "cores": cores, "kind": "oracle",
                         "sample": "%d oracle Newton iterations on the full lattice" % args.steps},
        "e2e": {"value": value, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    barrier(ws)
    return 0


# ---------------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------------
KERNELS = ["residual", "tangent_full", "tangent_reduced", "greedy_update", "apply_reduced", "apply_percell",
           "local_segmm", "local_gemv", "local_tc", "gj_update", "gj_pivot", "densify", "phi_schur",
           "coarse_blocked", "coarse_gemv", "coarse_solve", "local_segmm_dual", "local_gemv_dual", "local_tc_dual",
           "local_segmm_dual_in", "local_gemv_dual_in", "local_tc_dual_in", "dual_schur", "krylov_orth"]


def kernel_work(name, s, n_r, n_keys, prec_bytes, mixed=False):
    """Algorithmic work per launch (bytes or flops) and its roofline kind.

    local_segmm / local_gemv / local_tc: the principal-block x cell-multivector product,
        2 (n_R + n_P) n_R flops per cell (dense local inverse and coarse restriction);
    *_dual: the same on the dual block inside the interface solve, 2 (n_D + n_P) n_D per cell;
    *_dual_in: all rows, dual columns (input supported on the dual DOFs), 2 (n_R + n_P) n_D;
    dual_schur: the Dirichlet interface preconditioner's local products, 2 n_D^2 per cell;
    apply_reduced: 2 N_r nnz flops per cell (Eq. romstiffnessmatrix);
    apply_percell: the plain path, 8 nnz bytes of K^s and the two vectors per cell;
    coarse_gemv: the explicit coarse inverse streamed once: FP64 (2 n_primal^2 flops, FP64-ALU
        bound on GB300: one multiply-add per 8 bytes is above its FP64 rate) or, in the mixed
        modes, its FP32 copy (4 n_primal^2 bytes, HBM bound);
    coarse_solve: the FP64 block-LU solve of the block-tridiagonal coarse matrix, N blocks of
        size m: two sweeps of N - 1 block products and one of N, 2 (3 N - 2) m^2 flops.
    """
    n_s, n_loc, nnz = s.n_cells, s.n_loc, s.nnz
    n_rr, n_p = s.n_r_local, s.n_p_local
    n_d = n_rr - s.n_i_local
    if name in ("local_segmm", "local_gemv", "local_tc"):
        return 2.0 * (n_rr + n_p) * n_rr * n_s, "flops"
    if name in ("local_segmm_dual", "local_gemv_dual", "local_tc_dual"):
        return 2.0 * (n_d + n_p) * n_d * n_s, "flops"
    if name in ("local_segmm_dual_in", "local_gemv_dual_in", "local_tc_dual_in"):
        return 2.0 * (n_rr + n_p) * n_d * n_s, "flops"
    if name == "dual_schur":
        return 2.0 * n_d * n_d * n_s, "flops"
    if name == "apply_reduced" and n_r:
        return 2.0 * n_r * nnz * n_s, "flops"
    if name == "apply_percell":
        return 8.0 * nnz * n_s + 2 * 8.0 * n_loc * n_s, "bytes"
    if name == "coarse_solve" and s.n_coarse_blocks:
        nb, mb = s.n_coarse_blocks, s.coarse_block
        return 2.0 * (3 * nb - 2) * mb * mb, "flops"
    if name == "coarse_gemv":
        if mixed:
            return 4.0 * s.n_primal * s.n_primal + 16.0 * s.n_primal, "bytes"
        return 2.0 * s.n_primal * s.n_primal, "flops"
    return None, None


# DRAM bytes per launch from one ncu capture of the FP64 headline iteration (dram__bytes_read.sum
# + dram__bytes_write.sum), with the summary that holds the command; None once a kernel changes
MEASURED_TRAFFIC_FP64 = {
    "coarse_gemv": (305.54e6, "profiles/k_gemv_xs_fp64_ring32.md"),
    "local_segmm": (105.84e6, "profiles/k_local_segmm_n4_fp64_ring32.md"),
    "apply_reduced": (7.95e6, "profiles/k_apply_staged_fp64_ring32.md"),
}


def kernel_rooflines(kt, s, n_r, alu_peak, hbm_peak, tensor_peak=None, mixed=False):
    """Roofline entry for every timed kernel that has a work model, largest total time first."""
    rows = []
    for name, k in sorted(kt.items(), key=lambda kv: -kv[1]["total_ms"]):
        work, kind = kernel_work(name, s, n_r, None, 8, mixed)
        if work is None:
            continue
        avg_s = k["avg_us"] * 1e-6
        if kind == "flops":
            tc = name.startswith("local_tc")
            # the local products run in the mode's precision; the Krylov operator and the FP64
            # coarse product in FP64
            peak = tensor_peak if tc else (alu_peak if name.startswith(("local_", "dual_")) else FP64_PEAK_TFLOPS)
            ach = work / avg_s / 1e12
            rows.append({"kernel": name, "bound": "tensor" if tc else "alu", "achieved": ach, "peak": peak,
                         "unit": "TFLOP/s", "frac": ach / peak, "total_ms": k["total_ms"],
                         "work_per_launch": work})
        else:
            ach = work / avg_s / 1e9
            rows.append({"kernel": name, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                         "frac": ach / hbm_peak, "total_ms": k["total_ms"], "work_per_launch": work})
    return rows


def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__ as g
    g.build()
    import latgen
    from paper_2603_10741_gb300 import LAT_FP64, LAT_MIXED_BF16, LAT_MIXED_FP32, Lattice, solve_load_path

    ws, rank, local = dist_init(args)
    dev = torch.device("cuda", torch.cuda.current_device())
    hbm_peak, bf16_peak, peak_src = peaks()
    case = latgen.make_case(args.case)
    stream = torch.cuda.current_stream()

    # state: converged load steps 1..state_step (mixed precision path, untimed)
    lat_m = Lattice.from_case(case, LAT_MIXED_FP32)
    opts_m = lat_m.lattice_default_opts()
    u_prev, u_prev2 = None, None
    for k in range(1, args.state_step + 1):
        u = lat_m.lattice_predictor(case.top_displacement(k), u_prev, u_prev2)
        rep = lat_m.newton_step(u, opts_m)
        if not rep.converged:
            raise RuntimeError(f"load path failed at step {k}")
        u_prev2, u_prev = u_prev, u
    u_start = lat_m.lattice_predictor(case.top_displacement(args.state_step + 1), u_prev, u_prev2).clone()
    u_conv = u_prev.clone() if u_prev is not None else None   # converged state of the last load step
    torch.cuda.synchronize()

    def time_newton(lat, opts, steps, warmup, clocks=None, timing=False):
        """ms per Newton iteration over `steps` timed iterations (library kernel timers off, so
        that the interface PCG runs as CUDA-graph replays); with timing, one more untimed pass
        with the per-kernel timers on gives the kernel breakdown."""
        u = torch.empty_like(u_start)
        reps = []
        for _ in range(warmup):
            u.copy_(u_start)
            lat.newton_step(u, opts, max_iterations=1)
        torch.cuda.synchronize()
        barrier(ws)
        if clocks:
            clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        if clocks and args.profile_region == "headline":
            # headline leg: its timed region is the one a profiler started with
            # --profile-from-start off captures (no effect without a profiler)
            torch.cuda.profiler.start()
        e0.record(stream)
        for _ in range(steps):
            u.copy_(u_start)
            reps.append(lat.newton_step(u, opts, max_iterations=1).as_dict())
        e1.record(stream)
        torch.cuda.synchronize()
        if clocks and args.profile_region == "headline":
            torch.cuda.profiler.stop()
        ck = clocks.stop(local) if clocks else None
        barrier(ws)
        ms = e0.elapsed_time(e1)
        ktimes = {}
        if timing:
            lat.lattice_set_timing(True)
            u.copy_(u_start)
            lat.newton_step(u, opts, max_iterations=1)
            torch.cuda.synchronize()
            for kname in KERNELS:
                t, n = lat.lattice_kernel_time(kname)
                if n:
                    ktimes[kname] = {"total_ms": t, "launches": n, "avg_us": 1e3 * t / n}
            lat.lattice_set_timing(False)
        return max_over_ranks(ws, ms, dev) / steps, reps, ktimes, ck

    n_dof = lat_m.sizes.n_dof
    s = lat_m.sizes
    # headline: reduced path, FP64
    head_prec = {"fp64": LAT_FP64, "fp32": LAT_MIXED_FP32, "bf16": LAT_MIXED_BF16}[args.precision]
    lat = Lattice.from_case(case, head_prec)
    opts = lat.lattice_default_opts()
    clocks = Clocks()
    ms_red, reps_red, kt_red, ck = time_newton(lat, opts, args.steps, args.warmup, clocks, timing=True)
    value = ws * n_dof / (ms_red * 1e-3) / 1e9
    out = {
        "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_red, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f64+f32", "bf16": "f64+bf16"}[args.precision],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": {"fp64": "fp64 reduced (EIM) path",
                                                       "fp32": "mixed: FP32 preconditioner, FP64 operator",
                                                       "bf16": "mixed: BF16 local blocks, FP64 operator"}[args.precision],
                   "eps": opts.eps,
                   "step": "one Newton iteration (residual, snapshots+greedy+alpha, principal tangents, "
                           "FETI-DP setup, FGMRES, Armijo, update) from the predictor of load step %d"
                           % (args.state_step + 1),
                   "l2": "working set > L2 (FGMRES basis %.0f MB, local inverses)"
                         % (2 * (opts.krylov_restart + 1) * s.n_krylov * 8 / 1e6),
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "newton": {"n_r": reps_red[-1]["n_r_last"], "krylov_its": reps_red[-1]["krylov_its_total"],
                   "armijo_m": reps_red[-1]["armijo_m_max"], "pcg_its": reps_red[-1]["pcg_its_total"],
                   "phase_ms": {k: reps_red[-1][k] for k in ("t_residual_ms", "t_select_ms", "t_setup_ms",
                                                            "t_krylov_ms", "t_linesearch_ms")},
                   "kernels": kt_red},
    }
    # roofline of every modelled kernel; the headline entry is the one with the largest share
    rl = kernel_rooflines(kt_red, lat.sizes, out["newton"]["n_r"],
                          FP64_PEAK_TFLOPS if args.precision == "fp64" else FP32_PEAK_TFLOPS, hbm_peak, bf16_peak,
                          mixed=args.precision != "fp64")
    if rl:
        top = dict(rl[0])
        tr = MEASURED_TRAFFIC_FP64.get(top["kernel"]) if args.precision == "fp64" and args.case == "ring32" else None
        top["traffic"] = tr[0] if tr else None
        if tr:
            top["traffic_source"] = tr[1]
        top["peak_source"] = ({"fp64": "FP64 ALU, recipe table (1.20 measured)",
                               "fp32": "FP32 ALU, 152 SM x 128 lanes x 2 x 2.07 GHz"}.get(args.precision, peak_src)
                              if top["bound"] == "alu" else peak_src)
        out["roofline"] = top
        out["kernel_rooflines"] = rl
    out["clocks"] = ck
    # launches per step, counted with the CUDA profiler on one extra step
    out["gpu_launches"] = count_launches(lat, opts, u_start) * args.steps

    if not args.quick:
        # plain FP64 full-tangent path on the same state
        ms_full, reps_full, kt_full, _ = time_newton(lat, lat.lattice_default_opts(force_all=1),
                                                     max(2, args.steps // 2), 1, None, timing=True)
        out["fp64_full_path"] = {"ms_per_step": ms_full, "value": ws * n_dof / (ms_full * 1e-3) / 1e9,
                                 "krylov_its": reps_full[-1]["krylov_its_total"],
                                 "phase_ms": {k: reps_full[-1][k] for k in ("t_residual_ms", "t_select_ms",
                                                                            "t_setup_ms", "t_krylov_ms")},
                                 "kernels": kt_full}
        out["speedup_vs_fp64_full"] = ms_full / ms_red
        # mixed precision reduced path
        ms_mix, reps_mix, kt_mix, _ = time_newton(lat_m, opts_m, args.steps, 1, None, timing=True)
        out["mixed_fp32"] = {"ms_per_step": ms_mix, "value": ws * n_dof / (ms_mix * 1e-3) / 1e9,
                             "krylov_its": reps_mix[-1]["krylov_its_total"], "n_r": reps_mix[-1]["n_r_last"],
                             "phase_ms": {k: reps_mix[-1][k] for k in ("t_residual_ms", "t_select_ms",
                                                                       "t_setup_ms", "t_krylov_ms")},
                             "kernels": kt_mix}
        # BF16 principal blocks on the tensor cores (tcgen05), FP32 accumulation
        lat_b = Lattice.from_case(case, LAT_MIXED_BF16)
        opts_b = lat_b.lattice_default_opts()
        ms_bf, reps_bf, kt_bf, _ = time_newton(lat_b, opts_b, args.steps, 1, None, timing=True)
        out["mixed_bf16"] = {"ms_per_step": ms_bf, "value": ws * n_dof / (ms_bf * 1e-3) / 1e9,
                             "krylov_its": reps_bf[-1]["krylov_its_total"], "n_r": reps_bf[-1]["n_r_last"],
                             "phase_ms": {k: reps_bf[-1][k] for k in ("t_residual_ms", "t_select_ms",
                                                                      "t_setup_ms", "t_krylov_ms")},
                             "kernels": kt_bf}
        out["mixed_bf16"]["kernel_rooflines"] = kernel_rooflines(kt_bf, s, reps_bf[-1]["n_r_last"],
                                                                 FP32_PEAK_TFLOPS, hbm_peak, bf16_peak, mixed=True)
        out["mixed_fp32"]["kernel_rooflines"] = kernel_rooflines(kt_mix, s, reps_mix[-1]["n_r_last"],
                                                                 FP32_PEAK_TFLOPS, hbm_peak, mixed=True)
        out["fp64_full_path"]["kernel_rooflines"] = kernel_rooflines(kt_full, s, None, FP64_PEAK_TFLOPS, hbm_peak)
        lat_b.close()
    # reduced tangent action alone (selection of the benchmark state), L2 flushed between calls
    if not args.quick and u_conv is not None:
        # a11: the compliance gradient w.r.t. the per-cell mu scales at the converged state of
        # the last load step (adjoint through the reduced FETI-DP solve, FP64)
        lat.adjoint_gradient(u_conv, opts)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g_adj, J_adj, rep_adj = lat.adjoint_gradient(u_conv, opts)
        e1.record()
        torch.cuda.synchronize()
        out["adjoint"] = {"ms": e0.elapsed_time(e1), "n_theta": int(g_adj.numel()), "J": J_adj,
                          "krylov_its": rep_adj.krylov_its_total, "defect_corrections": rep_adj.iterations,
                          "state": "converged load step %d" % args.state_step}
    if args.profile_region == "apply":
        torch.cuda.profiler.start()
    out["apply"] = bench_apply(lat, lat_m, u_start, s, hbm_peak, peak_src)
    if not args.quick and rank == 0:
        # the 3D configuration's per-cell rows (a1-a7) at full size
        out["strut10_kernels"] = bench_kernels_3d("strut10", 1, hbm_peak, peak_src)
        out["strut20_apply"] = bench_apply_3d("strut20", 1, hbm_peak, peak_src)
    if args.profile_region == "apply":
        torch.cuda.profiler.stop()
    # end to end through host buffers: H2D of the state, one Newton iteration, D2H of the result
    out["e2e"] = bench_e2e(lat, opts, u_start, args, ws, dev, n_dof)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(out))
    lat.close()
    lat_m.close()
    return 0


def count_launches(lat, opts, u_start):
    """Kernels the library launches in one step (its own launch counter, copies excluded)."""
    u = u_start.clone()
    n0 = lat.lattice_launch_count()
    lat.newton_step(u, opts, max_iterations=1)
    return lat.lattice_launch_count() - n0


def _median_ms(fn, reps, flush=None):
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def bench_kernels_3d(case_name, load_step, hbm_peak, peak_src):
    """Rows a2 (residual), a3 (reduced-rule snapshots of every cell), a4-a6 (greedy, alpha,
    principal tangents) and a7 (reduced apply, FP64 and FP32) on a 3D lattice at full size, from
    the affine predictor of one load step; L2 flushed before every timed call."""
    import torch
    import latgen
    from paper_2603_10741_gb300 import LAT_MIXED_FP32, Lattice
    case = latgen.make_case(case_name)
    lat = Lattice.from_case(case, LAT_MIXED_FP32)
    s = lat.sizes
    u = lat.lattice_predictor(case.top_displacement(load_step))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    eps = lat.lattice_default_opts().eps
    stacked = s.n_loc * s.n_cells
    res = {"workload": "%s: %d cells, %d local DOF each, %d DOF, affine predictor of load step %d"
                       % (case_name, s.n_cells, s.n_loc, s.n_dof, load_step)}
    t = _median_ms(lambda: lat.assemble_residual_tangent(u), 10, flush)
    res["residual"] = {"ms": t, "gdofs": s.n_dof / t / 1e6, "qp": s.n_q_full * s.n_cells}
    K = torch.empty((s.n_cells, s.nnz), dtype=torch.float64, device="cuda")
    t = _median_ms(lambda: lat.assemble_residual_tangent(u, quad=1, residual=False, K_out=K), 10, flush)
    res["snapshots"] = {"ms": t, "qp": s.n_q_reduced * s.n_cells, "bytes_written": 8.0 * s.nnz * s.n_cells,
                        "write_gbs": 8.0 * s.nnz * s.n_cells / t / 1e6}
    t = _median_ms(lambda: lat.assemble_residual_tangent(u, quad=0, residual=False, K_out=K), 5, flush)
    res["tangents_full_rule"] = {"ms": t, "qp": s.n_q_full * s.n_cells,
                                 "note": "every cell at the full rule (the plain path's assembly)"}
    del K
    sel = lat.select_principal_cells(u, eps, 256)
    t = _median_ms(lambda: lat.select_principal_cells(u, eps, 256), 5, flush)
    res["select"] = {"ms": t, "eps": eps, "n_r": sel["n_r"],
                     "note": "snapshots + Algorithm 1 + alpha + principal tangents"}
    n_r = sel["n_r"]
    for tag, dt, eb in (("apply_fp64", torch.float64, 8), ("apply_fp32", torch.float32, 4)):
        x = torch.rand((s.n_loc, s.n_cells), dtype=dt, device="cuda")
        y = torch.empty_like(x)
        t = _median_ms(lambda: lat.apply_reduced_tangent(x, y), 50, flush) * 1e-3
        flops = 2.0 * n_r * s.nnz * s.n_cells
        byts = 2.0 * eb * stacked + eb * n_r * s.n_cells + eb * n_r * s.nnz
        alu = FP64_PEAK_TFLOPS if eb == 8 else FP32_PEAK_TFLOPS
        res[tag] = {"us": t * 1e6, "gdofs": stacked / t / 1e9, "n_r": n_r,
                    "hbm": {"achieved_gbs": byts / t / 1e9, "peak": hbm_peak, "frac": byts / t / 1e9 / hbm_peak,
                            "bytes": byts, "peak_source": peak_src},
                    "alu": {"achieved_tflops": flops / t / 1e12, "peak": alu, "frac": flops / t / 1e12 / alu},
                    "binding": max(byts / (hbm_peak * 1e9), flops / (alu * 1e12)) / t}
        del x, y
    del flush
    res["sweep_fp32"] = apply_sweep(lat, u, s, torch.float32, 4, FP32_PEAK_TFLOPS, hbm_peak)
    res["local_product"] = local_product_3d(case, lat, u, eps)
    lat.close()
    torch.cuda.empty_cache()
    return res


def local_product_3d(case, lat32, u, eps):
    """a9's principal-block x cell-multivector product on the 3D blocks (n_R ~ 2616): one
    application of K^-rom (the whole [G; Phi^T] of each key) in FP64, FP32 and on the tensor
    cores (BF16 pairs), timed by the library's kernel timers.  Corner-only primal set (no
    enrichment): only the product is measured here, not a solve."""
    import torch
    from paper_2603_10741_gb300 import LAT_FP64, LAT_MIXED_BF16, LAT_MIXED_FP32, Lattice
    _, bf16_peak, _ = peaks()
    out = {}
    for tag, prec, kname, peak in (("fp32", LAT_MIXED_FP32, "local_segmm", FP32_PEAK_TFLOPS),
                                   ("bf16", LAT_MIXED_BF16, "local_tc", bf16_peak),
                                   ("fp64", LAT_FP64, "local_segmm", FP64_PEAK_TFLOPS)):
        L = lat32 if prec == LAT_MIXED_FP32 else Lattice.from_case(case, prec)
        o = L.lattice_default_opts(max_enrich=0)
        L.select_principal_cells(u, eps, 256)
        L.lattice_prepare_solver(u, o)
        s = L.sizes
        v = L.krylov_vector()
        v.uniform_(-1.0, 1.0)
        L.feti_apply(1, v)
        torch.cuda.synchronize()
        L.lattice_set_timing(True)
        for _ in range(5):
            L.feti_apply(1, v)
        t, n = L.lattice_kernel_time(kname)
        L.lattice_set_timing(False)
        work = 2.0 * (s.n_r_local + s.n_p_local) * s.n_r_local * s.n_cells
        sec = t / n * 1e-3
        out[tag] = {"kernel": kname, "us": sec * 1e6, "flops": work, "tflops": work / sec / 1e12,
                    "frac": work / sec / 1e12 / peak, "peak": peak, "n_r_local": s.n_r_local}
        if L is not lat32:
            L.close()
        torch.cuda.empty_cache()
    return out


NR_SWEEP = (1, 2, 4, 8, 16, 32, 64)


def bench_apply_3d(case_name, load_step, hbm_peak, peak_src):
    """Row a7 on the largest 3D lattice (20^3 strut cells: 8000 cells x 2640 local DOF): the FP32
    reduced action against N_r, beside a device copy of the same bytes from X to Y (the stream
    rate this traffic pattern reaches); L2 flushed before every timed call."""
    import torch
    import latgen
    from paper_2603_10741_gb300 import LAT_MIXED_FP32, Lattice
    case = latgen.make_case(case_name)
    lat = Lattice.from_case(case, LAT_MIXED_FP32)
    s = lat.sizes
    u = lat.lattice_predictor(case.top_displacement(load_step))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    x = torch.rand((s.n_loc, s.n_cells), dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    t = _median_ms(lambda: y.copy_(x), 20, flush) * 1e-3
    copy = {"us": t * 1e6, "bytes": 8.0 * x.numel(), "gbs": 8.0 * x.numel() / t / 1e9,
            "frac": 8.0 * x.numel() / t / 1e9 / hbm_peak, "peak_source": peak_src}
    del x, y, flush
    res = {"workload": "%s: %d cells, %d local DOF each, %d DOF, affine predictor of load step %d"
                       % (case_name, s.n_cells, s.n_loc, s.n_dof, load_step),
           "copy_x_to_y": copy,
           "sweep_fp32": apply_sweep(lat, u, s, torch.float32, 4, FP32_PEAK_TFLOPS, hbm_peak)}
    lat.close()
    torch.cuda.empty_cache()
    return res


def apply_sweep(lat, u, s, dt, eb, alu_peak, hbm_peak, reps=20):
    """Reduced action with caller-given principals (the first N_r cells) and coefficients drawn
    per cell from a flat Dirichlet distribution (rng 8), N_r over NR_SWEEP; L2 flushed before
    every timed call."""
    import numpy as np
    import torch
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    x = torch.rand((s.n_loc, s.n_cells), dtype=dt, device="cuda")
    y = torch.empty_like(x)
    stacked = s.n_loc * s.n_cells
    out = []
    for n_r in NR_SWEEP:
        S = torch.arange(n_r, dtype=torch.int32)
        al = torch.tensor(np.random.default_rng(8).dirichlet(np.ones(n_r), size=s.n_cells).T.copy())
        lat.set_principal_cells(u, S, al)
        t = _median_ms(lambda: lat.apply_reduced_tangent(x, y), reps, flush) * 1e-3
        flops = 2.0 * n_r * s.nnz * s.n_cells
        byts = 2.0 * eb * stacked + eb * n_r * s.n_cells + eb * n_r * s.nnz
        out.append({"n_r": n_r, "us": t * 1e6, "gdofs": stacked / t / 1e9,
                    "hbm_frac": byts / t / 1e9 / hbm_peak, "alu_frac": flops / t / 1e12 / alu_peak,
                    "binding": max(byts / (hbm_peak * 1e9), flops / (alu_peak * 1e12)) / t})
    del flush, x, y
    return out


def bench_apply(lat, lat_m, u_start, s, hbm_peak, peak_src):
    """apply_reduced_tangent on the benchmark state's selection, FP64 and FP32."""
    import torch
    res = {}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for tag, L, dt, eb in (("fp64", lat, torch.float64, 8), ("fp32", lat_m, torch.float32, 4)):
        sel = L.select_principal_cells(u_start, L.lattice_default_opts().eps, 256)
        n_r = sel["n_r"]
        x = torch.rand((s.n_loc, s.n_cells), dtype=dt, device="cuda")
        y = torch.empty_like(x)
        for _ in range(5):
            L.apply_reduced_tangent(x, y)
        times = []
        for _ in range(50):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            L.apply_reduced_tangent(x, y)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) * 1e-3)
        t = statistics.median(times)
        stacked = s.n_loc * s.n_cells
        flops = 2.0 * n_r * s.nnz * s.n_cells
        byts = 2.0 * eb * stacked + eb * n_r * s.n_cells + eb * n_r * s.nnz
        alu_peak = FP64_PEAK_TFLOPS if tag == "fp64" else FP32_PEAK_TFLOPS
        res[tag] = {"gdofs": stacked / t / 1e9, "us": t * 1e6, "n_r": n_r,
                    "roofline": {"hbm": {"achieved_gbs": byts / t / 1e9, "peak": hbm_peak, "frac": byts / t / 1e9 / hbm_peak,
                                         "bytes": byts, "peak_source": peak_src},
                                 "alu": {"achieved_tflops": flops / t / 1e12, "peak": alu_peak,
                                         "frac": flops / t / 1e12 / alu_peak, "flops": flops},
                                 "binding": max(byts / (hbm_peak * 1e9), flops / (alu_peak * 1e12)) / t}}
    del flush
    res["sweep_fp64"] = apply_sweep(lat, u_start, s, torch.float64, 8, FP64_PEAK_TFLOPS, hbm_peak)
    res["sweep_fp32"] = apply_sweep(lat_m, u_start, s, torch.float32, 4, FP32_PEAK_TFLOPS, hbm_peak)
    return res


def bench_e2e(lat, opts, u_start, args, ws, dev, n_dof):
    import torch
    host = u_start.cpu().pin_memory()
    out_host = torch.empty_like(host).pin_memory()
    u = torch.empty_like(u_start)
    stream = torch.cuda.current_stream()
    for _ in range(1):
        u.copy_(host, non_blocking=True)
        lat.newton_step(u, opts, max_iterations=1)
        out_host.copy_(u, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        u.copy_(host, non_blocking=True)
        lat.newton_step(u, opts, max_iterations=1)
        out_host.copy_(u, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(ws, e0.elapsed_time(e1), dev) / args.steps
    nb = n_dof * 8
    return {"value": ws * n_dof / (ms * 1e-3) / 1e9, "unit": "GDOF/s", "ms_per_step": ms,
            "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb}


def cpu_baseline(args):
    step, n_dof = oracle_step_fn(args.case, args.state_step)
    t0 = time.perf_counter()
    step()
    dt = time.perf_counter() - t0
    return {"value": n_dof / dt / 1e9, "unit": "GDOF/s", "cores": threads_in_use(), "kind": "oracle",
            "sample": "one oracle Newton iteration (residual, assembled tangent, sparse LU, Armijo) on the "
                      "full lattice from the affine predictor of load step %d, %.1f s" % (args.state_step + 1, dt)}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
