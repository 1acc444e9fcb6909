"""bench.py's final JSON line on CPU: the short form of the plain-path comparison and the size of
the compacted line (the driver reads the line from the tail of the output)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _vp():
    # the shape plain_vs_reduced returns (values of one GB300 run)
    path = lambda ms, its, rel, k: {"ms_per_load_step": ms, "newton_its": its, "rel_residual": rel,
                                    "converged": True, "krylov_its": k}
    return {"workload": "ring32: 2D 32x32 ring cells (hole r=0.3), 16x16 Q1 per cell, 556034 DOF, "
                        "theta~U[0.9,1.1] seed 2, mu=1 lam=4, -20% in 20 steps",
            "load_step": 1, "reduced_fp64": path(128.34, 4, 3.3879e-09, 32),
            "plain_fp64": path(1116.2, 3, 2.2784e-10, 18), "reduced_mixed_fp32": path(95.659, 4, 3.3879e-09, 12),
            "speedup_reduced_fp64": 8.6967, "speedup_reduced_mixed": 11.668}


def test_vs_plain_summary_keeps_times_and_speedups():
    import bench
    s = bench.vs_plain_summary(_vp())
    assert s["workload"].startswith("ring32 load step 1")
    assert s["ms_per_load_step"] == {"plain_fp64": 1116.2, "reduced_fp64": 128.34, "reduced_mixed_fp32": 95.659}
    assert s["converged"] is True
    assert s["speedup_reduced_fp64"] == 8.6967 and s["speedup_reduced_mixed"] == 11.668


def test_compact_line_is_short_and_complete():
    """A line with every key the GPU arm prints (values of one GB300 run) stays under 2.5 KB
    once compacted, and keeps the contract's keys."""
    import bench
    out = {
        "metric": bench.METRIC, "value": 223.48123, "unit": "GDOF/s", "n_gpus": 1, "steps": 3, "warmup": 3,
        "ms_per_step": 2930.4123, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32+bf16", "data": "synthetic",
        "config": {"workload": "strut20: 3D 20x20x20 edge-strut cells (12^3 voxels, strut half-width 0.15), "
                               "344 Q1 hex per cell, 13736163 DOF, theta~U[0.9,1.1] seed 4, mu=1 lam=4, "
                               "-20% in 20 steps",
                   "precision": "FP32 action (inner Krylov), BF16-pair preconditioner blocks; FP64 "
                                "residual, outer operator, update",
                   "step": "one Newton iteration (all hot-path rows) from the predictor of load step 2",
                   "value": "apply_reduced_fp32: n_loc*N_s DOF/s over its 16 launches in the timed iterations",
                   "l2": "inputs larger than L2: cell vectors 84 MB each, FGMRES bases 36922 MB",
                   "parallelism": "single GPU"},
        "roofline": {"kernel": "k_local_tc (dual_schur_tc, local_tc_dual, local_tc, local_tc_dual_in)",
                     "bound": "tensor", "achieved": 162.12, "peak": 1746.8, "unit": "TFLOP/s", "frac": 0.092809,
                     "peak_source": "measured bf16 tensor (sustained)", "work_per_launch": 46618000000.0,
                     "avg_us": 287.55, "launches": 2936, "share": 0.43086, "issued_frac": 0.27843,
                     "traffic": None},
        "apply_roofline": {"kernel": "apply_reduced_fp32", "bound": "hbm", "achieved": 1793.4, "peak": 6662.6,
                           "unit": "GB/s", "frac": 0.26917, "peak_source": "measured copy bandwidth",
                           "work_per_launch": 169480000.0, "avg_us": 94.504, "launches": 80, "share": 0.00077517},
        "newton": {"ms_per_iteration": 2930.4, "global_gdofs": 0.0046875, "n_r": 1, "krylov_its": 3,
                   "inner_its": 16, "pcg_its": 1444, "enrich_level": 0},
        "gpu_launches": 132865,
        "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 73},
        "e2e": {"value": 22.51, "unit": "GDOF/s", "ms_per_step": 0.93826, "h2d_bytes_per_step": 84480000,
                "d2h_bytes_per_step": 84480000, "n_r": 1,
                "what": "apply_reduced_tangent, X from pinned host memory and Y back every call"},
        "vs_plain_fp64": bench.vs_plain_summary(_vp()),
        "cpu_baseline": {"value": 0.092139, "unit": "GDOF/s", "cores": 16, "kind": "oracle",
                         "sample": "682 calls, 10.0 s: oracle reduced action (numpy, 1 dense principals), "
                                   "first 512 cells of strut20, predictor of step 2"},
    }
    line = json.dumps(bench.compact(out))
    assert len(line) < 2500, len(line)
    back = json.loads(line)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks",
              "cpu_baseline"):
        assert k in back, k
    assert back["roofline"]["traffic"] is None and "workload" in back["config"]
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in back["e2e"]


def test_work_models_of_the_roofline_entries():
    """The algorithmic work the roofline entries divide by, for the 20^3 strut lattice's sizes:
    the FP32 reduced action streams X and Y once plus alpha and one principal's values, 4 (2 n_loc
    N_s + N_r N_s + N_r nnz) bytes; the mixed-mode coarse block-LU solve streams the FP32 factors
    U, U^T (N - 1 blocks each) and D^{-1} (N blocks) once, 4 (3 N - 2) m^2 bytes; the dual-block
    product is 2 (n_D + n_P) n_D flops per cell."""
    import types

    import bench
    import latgen
    cell_nodes = latgen.strut_cell(12, 0.15)[0].shape[0]
    assert cell_nodes == 880
    s = types.SimpleNamespace(n_cells=8000, n_loc=3 * cell_nodes, nnz=122112, n_r_local=2616, n_p_local=24,
                              n_i_local=924, n_coarse_blocks=19, coarse_block=1324, n_primal=24000)
    w, kind = bench.kernel_work("apply_reduced_fp32", s, 1, True)
    assert kind == "hbm" and w == 4 * (2 * 2640 * 8000 + 8000 + 122112) == 169480448
    w, kind = bench.kernel_work("coarse_solve", s, 1, True)
    assert kind == "hbm" and w == 4 * 55 * 1324 ** 2
    w, kind = bench.kernel_work("coarse_solve", s, 1, False)
    assert kind == "fp64" and w == 2 * 55 * 1324 ** 2
    n_d = 2616 - 924
    w, kind = bench.kernel_work("local_tc_dual", s, 1, True)
    assert kind == "tensor" and w == 2.0 * (n_d + 24) * n_d * 8000
    w, kind = bench.kernel_work("dual_schur_tc", s, 1, True)
    assert kind == "tensor" and w == 2.0 * n_d * n_d * 8000
