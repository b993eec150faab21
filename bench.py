#!/usr/bin/env python
"""Benchmark: pressure-Poisson PCG throughput (DOFs/s) and time per CHNS step on one GB300.

Workload: the rising-drop octree (levels 5..8, refined where |phi| < 0.9 around a drop of radius
0.15 at (0.5, 0.5, 0.3), Cn = 0.01, density ratio 1000, viscosity ratio 100, Re 35, We 1, Fr 1,
dt 5e-4), seeded synthetic fields. One bench step = one chns_step (two blocks of CH Newton,
velocity prediction, pressure Poisson, velocity update) to relative residual 1e-8.

value       = n_nodes x (Poisson solves in the timed steps) / (their device time), for the headline
              path: FP32 Krylov iterations and applies inside FP64 refinement (FP64 dot products);
plain_fp64  = the same numbers for the all-FP64 path on the same GPU;
bf16_coefficients = the headline path with bfloat16 coefficient storage for Poisson / mass;
e2e         = one Poisson solve through the C ABI from pinned host buffers (copies timed);
roofline    = the dominant apply kernel timed alone from a cold L2 (algorithmic bytes / time);
cpu_baseline= the FP64 CPU oracle (assembled matrix + Jacobi-PCG) on a bounded sample;
large_interface = the Rayleigh-Taylor workload at scale (~7e6 leaves): its pressure-Poisson
              solve in the three precisions, their difference, the Poisson apply alone, and
              full time steps (CH with the Schur-complement preconditioner) in mixed precision
              and in FP64 (see run_large);
learned     = the learned coarse correction for the pressure-Poisson solve on the 8-drop
              workload: pairs from time steps, training, and the solves of one more step with
              and without it (untimed setup; see run_learned).

Under torchrun (N > 1) every rank runs an independent replica (the method is not sharded) and
value sums the replicas; timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Poisson+PCG DOFs/s and time/step vs plain FP64 GPU at 1e-8 residual; HBM frac"
UNIT = "DOFs/s"
WORKLOAD = "rising_drop_levels5-8"
APPLY_DRAM_BYTES = 11.27e6  # DRAM bytes of one launch of the roofline kernel (ncu, see below)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if s[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_max(pg, values, device):
    """Max over ranks of per-rank times (one all-reduce; identity without a process group)."""
    if not pg:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return [float(v) for v in t]


def whole_job_value(ws, n_nodes, solves_per_rank, ms_max):
    """DOFs/s of the whole job: every replica solves the same number of systems of n_nodes
    unknowns; the slowest rank's time counts."""
    return ws * n_nodes * solves_per_rank / (ms_max * 1e-3)


# --------------------------------------------------------------------------- our arm
def field_errors(final_fields, n_steps):
    """Relative L2 difference per field between the reduced-precision paths and the all-FP64
    path after the same number of steps from the same initial state."""
    import numpy as np

    ref = final_fields.get("fp64")
    if ref is None:
        return None
    out = {"steps": n_steps}
    for label, f in final_fields.items():
        if label == "fp64":
            continue
        e = {}
        for k in ("phi", "mu", "p"):
            e[k] = float(np.linalg.norm(f[k] - ref[k]) / max(np.linalg.norm(ref[k]), 1e-300))
        e["u"] = float(np.linalg.norm(f["u"] - ref["u"]) / max(np.linalg.norm(ref["u"]), 1e-300))
        out[label] = e
    return out


def run_ours(args):
    import numpy as np
    import torch

    from chns_workloads import configs
    from paper_2107_05123_gb300 import capi
    from paper_2107_05123_gb300.session import DeviceState, Mesh, default_step_params

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist

    w = configs.rising_drop(5, 8)
    mesh = Mesh(w.anchors, w.levels, w.extent)
    N = mesh.n_nodes
    f0 = w.init(mesh.node_xyz)
    prm_d = w.params.as_dict()
    prm = capi.make_params(prm_d)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def flush_l2():
        flush.fill_(1.0)

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize()

    def run_path(inner, label):
        ds = DeviceState(dict(phi=f0["phi"], mu=f0["mu"], u=f0["u"], p=f0["p"]))
        sp = default_step_params(rtol=1e-8, inner=inner, pp_check_every=8)
        for _ in range(args.warmup):
            capi.chns_step(mesh.handle, ds.c, prm, sp)
        step_ms, pp_ms, pp_n, pp_it, stats = [], 0.0, 0, 0, []
        l0 = capi.chns_kernel_launches()
        for _ in range(args.steps):
            flush_l2()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.nvtx.range_push("timed_step")
            e0.record()
            st = capi.chns_step(mesh.handle, ds.c, prm, sp)
            e1.record()
            torch.cuda.nvtx.range_pop()
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            for l in range(2):
                pp_ms += st.pp[l].ms
                pp_n += 1
                pp_it += st.pp[l].iterations
            stats.append(st)
        launches = capi.chns_kernel_launches() - l0
        tmax, pp_ms = replica_max(pg, [sum(step_ms), pp_ms], "cuda")
        last = stats[-1]
        final_fields[label] = ds.host()
        return dict(label=label, ms_per_step=tmax / args.steps,
                    value=whole_job_value(ws, N, pp_n, pp_ms),
                    pp_ms_per_solve=pp_ms / pp_n, pp_iters_per_solve=pp_it / pp_n,
                    launches=launches,
                    phases_ms=dict(ch=last.ms_ch, vp=last.ms_vp, pp=last.ms_pp, vu=last.ms_vu),
                    newton_its=list(last.newton_its),
                    mass_drift=abs(last.phi_mass_after - last.phi_mass_before),
                    pp_refinements=last.pp[1].refinements)

    final_fields = {}

    with ClockSampler(local) as clk:
        headline = plain = bf16 = None
        if args.paths in ("both", "headline"):
            headline = run_path(capi.FP32, "fp32_fp64refine")
        if args.paths in ("both", "plain"):
            plain = run_path(capi.FP64, "fp64")
        if args.paths == "both":
            bf16 = run_path(capi.FP32_BF16COEF, "fp32_bf16coef_fp64refine")
    clocks = clk.summary()
    if args.paths != "both":
        if rank == 0:
            print(json.dumps({"paths": args.paths, "detail": headline or plain, "clocks": clocks}))
        return

    # ---- roofline of the dominant kernel: the matrix-free Poisson apply of the headline path,
    # timed alone from a cold L2 on the launching stream.
    stream = torch.cuda.current_stream()
    phit = torch.as_tensor(f0["phi"], device="cuda")
    x32 = torch.randn(N, device="cuda", dtype=torch.float32)
    y32 = torch.empty_like(x32)
    c32 = capi.make_coef(phit.float())
    times = []
    for i in range(13):
        flush_l2()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        capi.chns_apply_poisson(mesh.handle, prm, c32, x32, y32, capi.FP32, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= 3:
            times.append(e0.elapsed_time(e1))
    t_apply = statistics.mean(times) * 1e-3
    E, H = mesh.n_elem, mesh.n_hanging
    # algorithmic bytes: x read + y written + phi~ read (4 B each per node), the element table
    # (8 x int32 + level byte per element), the hanging table (16 B per entry)
    alg_bytes = N * (4 + 4 + 4) + E * 33 + H * 16
    peak, peak_kind = _peaks()
    achieved = alg_bytes / t_apply / 1e9
    # DRAM bytes of one launch from an ncu capture of this kernel on this workload
    # (dram__bytes_read.sum 11.27 MB + dram__bytes_write.sum 0, summarised under profiles/);
    # --traffic overrides it
    traffic = args.traffic if args.traffic is not None else APPLY_DRAM_BYTES

    # ---- end to end: one Poisson solve through the C ABI with pinned host buffers
    b_dev = torch.zeros(N, dtype=torch.float64, device="cuda")
    zero3 = [torch.zeros(N, dtype=torch.float64, device="cuda") for _ in range(3)]
    mu_d = torch.as_tensor(f0["mu"], device="cuda")
    cpp = capi.make_coef(phit, zero3, mu_d)
    capi.chns_rhs_poisson(mesh.handle, prm, cpp, zero3, zero3, torch.zeros_like(b_dev), b_dev)
    b_h = b_dev.cpu().pin_memory()
    phi_h = phit.cpu().pin_memory()
    x_h = torch.zeros(N, dtype=torch.float64).pin_memory()
    bd, xd, pd = torch.empty_like(b_dev), torch.empty_like(b_dev), torch.empty_like(b_dev)
    solver = capi.make_solver(capi.KSP_CG, capi.PC_JACOBI, 1e-8, 20000, 30, capi.FP32,
                              1e-6, 30, check_every=8)
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        barrier()
        t0 = time.perf_counter()
        bd.copy_(b_h, non_blocking=True)
        pd.copy_(phi_h, non_blocking=True)
        xd.zero_()
        capi.chns_krylov_solve(mesh.handle, capi.OP_POISSON, prm, capi.make_coef(pd), bd, xd,
                               solver)
        x_h.copy_(xd, non_blocking=True)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_val = whole_job_value(ws, N, 1, replica_max(pg, [statistics.mean(e2e_ms)], "cuda")[0])

    large = None
    if rank == 0 and not args.no_large:
        try:
            large = run_large(args)
        except Exception as e:  # the headline line is printed whatever happens here
            large = {"error": f"{type(e).__name__}: {e}"}
    learned = None
    if rank == 0 and not args.no_learned:
        try:
            learned = run_learned(args)
        except Exception as e:  # the headline line is printed whatever happens here
            learned = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0:
        cpu = cpu_baseline(w, mesh.node_xyz, f0, budget_s=args.cpu_budget) if not args.no_cpu else None
        line = {
            "metric": METRIC, "value": headline["value"], "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": headline["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_elem": int(E), "n_nodes": int(N),
                       "n_hanging": int(H), "rtol": 1e-8, "l2": "flushed before every step",
                       "parallelism": "replicas" if ws > 1 else "single"},
            "plain_fp64": {"value": plain["value"], "ms_per_step": plain["ms_per_step"],
                           "pp_ms_per_solve": plain["pp_ms_per_solve"],
                           "pp_iters_per_solve": plain["pp_iters_per_solve"],
                           "phases_ms": plain["phases_ms"]},
            "headline_detail": headline,
            "bf16_coefficients": {"value": bf16["value"], "ms_per_step": bf16["ms_per_step"],
                                  "pp_ms_per_solve": bf16["pp_ms_per_solve"],
                                  "pp_iters_per_solve": bf16["pp_iters_per_solve"]},
            "speedup_vs_plain_fp64": {"pp": headline["value"] / plain["value"],
                                      "step": plain["ms_per_step"] / headline["ms_per_step"]},
            "field_error_vs_fp64": field_errors(final_fields, args.warmup + args.steps),
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(2 * N * 8),
                    "d2h_bytes_per_step": int(N * 8)},
            "roofline": {"kernel": "k_apply_patch<PoissonK<float,float>>", "bound": "hbm",
                         "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "alg_bytes": int(alg_bytes), "ms": t_apply * 1e3},
            "cpu_baseline": cpu,
            "large_interface": large,
            "learned": learned,
            "clocks": clocks,
            "gpu_launches": headline["launches"],
        }
        print(json.dumps(line))
    if pg:
        pg.destroy_process_group()


def run_large(args):
    """The Rayleigh-Taylor interface at scale (box 1 x 4 x 1, levels 6-10 refined in the
    interface band, Cn 0.005, density ratio 3, Re 1000): the pressure-Poisson solve of the
    initial state (right-hand side from chns_rhs_poisson at rest: the gravity term of R_m) to
    1e-8 with Jacobi-PCG in the three precisions (BF16 coefficients + FP32 Krylov + FP64
    refinement, FP32 + FP64 refinement, all FP64), the difference of the reduced-precision
    solutions from the FP64 one, and the Poisson apply timed alone from a cold L2 (HBM regime).
    Then full time steps from the initial state: the Cahn-Hilliard GMRES uses the
    Schur-complement preconditioner, since the 2x2 block-Jacobi one does not reach 1e-8 within
    4,000 iterations at this resolution."""
    import numpy as np
    import torch

    from chns_workloads import configs
    from paper_2107_05123_gb300 import capi
    from paper_2107_05123_gb300.session import Mesh

    t_all = time.perf_counter()
    w = configs.rayleigh_taylor(6, 10, 0.005)
    t0 = time.perf_counter()
    mesh = Mesh(w.anchors, w.levels, w.extent)
    t_mesh = time.perf_counter() - t0
    N, E, H = mesh.n_nodes, mesh.n_elem, mesh.n_hanging
    f0 = w.init(mesh.node_xyz)
    prm = capi.make_params(w.params.as_dict())
    out = {"workload": "rayleigh_taylor_levels6-10", "n_elem": int(E), "n_nodes": int(N),
           "n_hanging": int(H), "mesh_create_s": round(t_mesh, 1)}
    phit = torch.as_tensor(f0["phi"], device="cuda")
    zero3 = [torch.zeros(N, dtype=torch.float64, device="cuda") for _ in range(3)]
    b = torch.zeros(N, dtype=torch.float64, device="cuda")
    capi.chns_rhs_poisson(mesh.handle, prm,
                          capi.make_coef(phit, zero3, torch.as_tensor(f0["mu"], device="cuda")),
                          zero3, zero3, torch.zeros_like(b), b)
    sols = {}
    for label, inner in (("fp32_bf16coef_fp64refine", capi.FP32_BF16COEF),
                         ("fp32_fp64refine", capi.FP32), ("fp64", capi.FP64)):
        solver = capi.make_solver(capi.KSP_CG, capi.PC_JACOBI, 1e-8, 40000, 30, inner, 1e-6, 40,
                                  check_every=8)
        x = torch.zeros_like(b)
        st = capi.chns_krylov_solve(mesh.handle, capi.OP_POISSON, prm, capi.make_coef(phit), b,
                                    x, solver, check=False)
        sols[label] = x.cpu().numpy()
        out[label] = {"pp_ms": round(st.ms, 2), "pp_iters": st.iterations,
                      "refinements": st.refinements, "escalations": st.escalations,
                      "rel_residual": st.rel_residual, "status": st.status,
                      "dofs_per_s": N / (1e-3 * st.ms) if st.ms > 0 else None}
    ref = sols["fp64"]
    out["p_error_vs_fp64"] = {k: float(np.linalg.norm(v - ref) / max(np.linalg.norm(ref), 1e-300))
                              for k, v in sols.items() if k != "fp64"}
    # the Poisson apply alone, FP32, from a cold L2
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    c32 = capi.make_coef(phit.float())
    x32 = torch.randn(N, device="cuda", dtype=torch.float32)
    y32 = torch.empty_like(x32)
    ts = []
    for i in range(8):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        capi.chns_apply_poisson(mesh.handle, prm, c32, x32, y32, capi.FP32)
        e1.record()
        torch.cuda.synchronize()
        if i >= 3:
            ts.append(e0.elapsed_time(e1) * 1e-3)
    alg = N * 12 + E * 33 + H * 16
    peak, kind = _peaks()
    ach = alg / statistics.mean(ts) / 1e9
    out["poisson_apply_fp32"] = {"ms": round(statistics.mean(ts) * 1e3, 4), "alg_bytes": int(alg),
                                 "achieved_gbs": ach, "peak_gbs": peak, "peak_kind": kind,
                                 "frac": ach / peak}
    del flush, x32, y32
    # full time steps from the initial state: CH Newton with GMRES and the Schur-complement
    # preconditioner (the nodal block-Jacobi one stalls at this resolution), velocity
    # prediction, pressure Poisson, velocity update; mixed precision (FP32 Krylov + FP64
    # refinement) for args.large_steps steps and the all-FP64 path for one
    from paper_2107_05123_gb300.session import DeviceState, default_step_params

    def step_params(inner):
        sp = default_step_params(rtol=1e-8, inner=inner, pp_check_every=8)
        sp.ch.pc = capi.PC_SCHUR
        sp.ch.inner_its = 20
        sp.ch.max_it = 400
        return sp

    def timed_steps(inner, n):
        ds = DeviceState(dict(phi=f0["phi"], mu=f0["mu"], u=f0["u"], p=f0["p"]))
        sp = step_params(inner)
        res, first = [], None
        for k in range(n):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st = capi.chns_step(mesh.handle, ds.c, prm, sp)
            e1.record()
            torch.cuda.synchronize()
            res.append({"ms": round(e0.elapsed_time(e1), 1),
                        "phases_ms": {"ch": round(st.ms_ch, 1), "vp": round(st.ms_vp, 1),
                                      "pp": round(st.ms_pp, 1), "vu": round(st.ms_vu, 1)},
                        "newton_its": list(st.newton_its),
                        "ch_gmres_its": [st.ch[l].iterations for l in range(2)],
                        "vp_gmres_its": [st.vp[l].iterations for l in range(2)],
                        "pp_cg_its": [st.pp[l].iterations for l in range(2)],
                        "mass_drift": abs(st.phi_mass_after - st.phi_mass_before)})
            if k == 0:
                first = ds.host()
        return res, first

    steps_mixed, f_mixed = timed_steps(capi.FP32, max(1, args.large_steps))
    steps_fp64, f_fp64 = timed_steps(capi.FP64, 1)
    err = {}
    for key in ("phi", "mu", "p", "u"):
        a, b_ = np.asarray(f_mixed[key]), np.asarray(f_fp64[key])
        if key == "p":
            a, b_ = a - a.mean(), b_ - b_.mean()
        err[key] = float(np.linalg.norm(a - b_) / max(np.linalg.norm(b_), 1e-300))
    ms_mixed = statistics.mean(r["ms"] for r in steps_mixed)
    out["time_step"] = {"ch_pc": "schur (inner_its 20), flexible GMRES",
                        "fp32_fp64refine": {"ms_per_step": round(ms_mixed, 1),
                                            "steps": steps_mixed},
                        "fp64": {"ms_per_step": steps_fp64[0]["ms"], "steps": steps_fp64},
                        "speedup_vs_fp64": round(steps_fp64[0]["ms"] / ms_mixed, 2),
                        "field_error_vs_fp64_after_1_step": err}
    out["wall_s"] = round(time.perf_counter() - t_all, 1)
    return out


def run_learned(args):
    """The learned coarse correction on the 8-drop workload (levels 5-8, drops of radius
    0.05-0.12, Cn 0.01, density ratio 1000): training pairs from the pressure-Poisson solves of
    `--learned-steps` time steps (iterates of FP64 Jacobi-PCG, every 8th, at most 24 per solve),
    energy-norm training on the GPU, then the pressure-Poisson solves of one more step from the
    same state in mixed precision with Jacobi-PCG, Chebyshev-PCG (degree 3) and FCG + learned
    correction, and the same step on the all-FP64 path (Jacobi). Returns the summary object of the
    bench line."""
    import torch

    from chns_workloads import configs
    from paper_2107_05123_gb300 import capi
    from paper_2107_05123_gb300.session import DeviceState, Mesh, default_step_params

    t_all = time.perf_counter()
    w = configs.many_drops(seed=0, n=8, rmin=0.05, rmax=0.12, lmin=5, lmax=8, Cn=0.01)
    mesh = Mesh(w.anchors, w.levels, w.extent)
    prm = capi.make_params(w.params.as_dict())
    f0 = w.init(mesh.node_xyz)
    D = args.learned_grid
    net = capi.chns_learned_create(D, 4096, 1)

    def params(pp=None, collect=None):
        sp = default_step_params(rtol=1e-8, inner=capi.FP32, pp_check_every=8)
        sp.vp.max_it = 20000
        if pp is not None:
            sp.pp = pp
        if collect is not None:
            sp.collect, sp.collect_every, sp.collect_max = collect, 8, 24
        return sp

    ds = DeviceState(dict(phi=f0["phi"], mu=f0["mu"], u=f0["u"], p=f0["p"]))
    t0 = time.perf_counter()
    steps_done, step_error = 0, None
    snap = ds.host()
    for _ in range(args.learned_steps):
        try:
            capi.chns_step(mesh.handle, ds.c, prm, params(collect=net))
        except capi.ChnsError as e:  # a failed step leaves the state unusable: keep the last one
            step_error = str(e)
            ds = DeviceState(snap)
            break
        steps_done += 1
        snap = ds.host()
    torch.cuda.synchronize()
    t_collect = time.perf_counter() - t0
    pairs = capi.chns_learned_num_samples(net)
    if pairs == 0:
        capi.chns_learned_destroy(net)
        return {"workload": "drops8_levels5-8", "error": step_error or "no training pairs"}
    t0 = time.perf_counter()
    loss = capi.chns_learned_train(net, mesh.handle, prm, args.learned_iters, args.learned_lr, 0)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    res = {}
    # one more step from the same state: mixed precision (FP32 Krylov + FP32 applies + FP64
    # refinement) with three pressure preconditioners, and the all-FP64 path with Jacobi
    runs = {
        "mixed_jacobi": params(pp=capi.make_solver(
            capi.KSP_CG, capi.PC_JACOBI, 1e-8, 20000, 30, capi.FP32, 1e-6, 30, check_every=8)),
        "mixed_chebyshev3": params(pp=capi.make_solver(
            capi.KSP_CG, capi.PC_CHEBYSHEV, 1e-8, 20000, 3, capi.FP32, 1e-6, 30, check_every=8)),
        "mixed_learned": params(pp=capi.make_solver(
            capi.KSP_FCG, capi.PC_LEARNED, 1e-8, 20000, 30, capi.FP32, 1e-6, 30, check_every=8,
            learned=net)),
        "plain_fp64_jacobi": default_step_params(rtol=1e-8, inner=capi.FP64, pp_check_every=8),
    }
    runs["plain_fp64_jacobi"].vp.max_it = 20000
    for name, sp in runs.items():
        try:
            st = capi.chns_step(mesh.handle, DeviceState(snap).c, prm, sp)
        except capi.ChnsError as e:
            st = getattr(e, "stats", None)
            res[name] = {"error": str(e)}
            if st is None:
                continue
        res.setdefault(name, {}).update(
            ms_step=round(st.ms_total, 2),
            pp_iters=[st.pp[l].iterations for l in range(2)],
            pp_ms=[round(st.pp[l].ms, 3) for l in range(2)],
            fallbacks=[st.pp[l].fallbacks for l in range(2)],
            rel_residual=[st.pp[l].rel_residual for l in range(2)])
    capi.chns_learned_destroy(net)
    small = _learned_small_drops(args)
    return {"workload": "drops8_levels5-8", "n_elem": int(mesh.n_elem),
            "n_nodes": int(mesh.n_nodes), "grid": D, "channels": 16, "levels": 4,
            "collect_steps": steps_done, "collect_step_error": step_error, "pairs": int(pairs),
            "train_iterations": args.learned_iters, "lr": args.learned_lr,
            "collect_s": round(t_collect, 2), "train_s": round(t_train, 2),
            "train_ms_per_iteration": round(1e3 * t_train / max(args.learned_iters, 1), 3),
            "energy_loss_first_100": float(loss[:100].mean()) if len(loss) else None,
            "energy_loss_last_500": float(loss[-500:].mean()) if len(loss) else None,
            "next_step": res, "small_drops": small,
            "wall_s": round(time.perf_counter() - t_all, 1)}


def _learned_small_drops(args):
    """The same method on a small 4-drop octree (levels 3-6, Cn 0.02, density ratio 1000) with
    D = 16: pairs from FP64 Jacobi-PCG solves of 16 seeded smooth right-hand sides, 1,500
    training iterations, then Jacobi-PCG and FCG + learned correction (FP64) on 3 unseen ones."""
    import numpy as np
    import torch

    from chns_workloads import configs
    from paper_2107_05123_gb300 import capi
    from paper_2107_05123_gb300.session import Mesh

    w = configs.many_drops(seed=3, n=4, lmin=3, lmax=6, Cn=0.02)
    mesh = Mesh(w.anchors, w.levels, w.extent)
    n = mesh.n_nodes
    prm = capi.make_params(w.params.as_dict())
    phi = torch.as_tensor(w.init(mesh.node_xyz)["phi"], device="cuda")
    coef = capi.make_coef(phi)
    rng = np.random.default_rng(12)

    def rhs():
        f = np.zeros(n)
        for _ in range(6):
            k = rng.integers(1, 4, size=3)
            f += rng.standard_normal() * np.cos(np.pi * (k * mesh.node_xyz).sum(axis=1)
                                                + rng.uniform(0, 6.3))
        return torch.as_tensor(f - f.mean(), device="cuda")

    net = capi.chns_learned_create(16, 512, 5)
    for _ in range(16):
        capi.chns_learned_collect(net, mesh.handle, prm, coef, rhs(), 4, 32)
    t0 = time.perf_counter()
    capi.chns_learned_train(net, mesh.handle, prm, 1500, 1e-3, 1)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    out = {"jacobi_pcg": [], "fcg_learned": [], "jacobi_ms": [], "learned_ms": []}
    for _ in range(3):
        b = rhs()
        for pc, ksp, key in ((capi.PC_JACOBI, capi.KSP_CG, "jacobi"),
                             (capi.PC_LEARNED, capi.KSP_FCG, "learned")):
            x = torch.zeros(n, device="cuda", dtype=torch.float64)
            st = capi.chns_krylov_solve(mesh.handle, capi.OP_POISSON, prm, coef, b, x,
                                        capi.make_solver(ksp, pc, 1e-8, 20000, 30, capi.FP64,
                                                         check_every=8, learned=net))
            out["jacobi_pcg" if key == "jacobi" else "fcg_learned"].append(st.iterations)
            out[key + "_ms"].append(round(st.ms, 3))
    pairs = capi.chns_learned_num_samples(net)
    capi.chns_learned_destroy(net)
    out.update(workload="drops4_levels3-6", n_nodes=int(n), grid=16, pairs=int(pairs),
               train_iterations=1500, train_s=round(t_train, 2))
    return out


# --------------------------------------------------------------------------- CPU oracle
def cpu_baseline(w, node_xyz, f0, budget_s=30.0):
    """Time the oracle's Poisson solve (assembly + Jacobi-PCG to 1e-8) on the same mesh."""
    import numpy as np

    from oracle import fem, solvers
    from oracle.mesh import Mesh as OMesh

    t0 = time.perf_counter()
    om = OMesh(w.anchors, w.levels, w.extent)
    el, co = fem.Elem(om), fem.Coeffs(w.params.as_dict())
    N = om.n_nodes
    z = np.zeros((3, N))
    vs = fem.VMSState(el, co, f0["phi"], z, f0["mu"])
    b = fem.pp_rhs(vs, z, z, np.zeros(N))
    t1 = time.perf_counter()
    A = fem.poisson(el, co, f0["phi"])
    t2 = time.perf_counter()
    x, it, rel = solvers.pcg(A, b, rtol=1e-8, mean_zero=True, maxit=100000)
    t3 = time.perf_counter()
    return {"value": N / (t3 - t1), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"one pressure-Poisson solve on the same mesh ({N} nodes): scipy CSR "
                       f"assembly {t2 - t1:.1f} s + Jacobi-PCG {it} its to 1e-8 in {t3 - t2:.1f} s "
                       f"(value counts assembly + solve; setup {t1 - t0:.1f} s excluded); host "
                       f"cores {os.cpu_count()}, numpy/scipy single-threaded")}


# --------------------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    import numpy as np

    from chns_workloads import configs
    from oracle import fem, solvers
    from oracle.mesh import Mesh as OMesh

    w = configs.rising_drop(5, 8)
    om = OMesh(w.anchors, w.levels, w.extent)
    f0 = w.init(om.node_xyz)
    el, co = fem.Elem(om), fem.Coeffs(w.params.as_dict())
    N = om.n_nodes
    z = np.zeros((3, N))
    vs = fem.VMSState(el, co, f0["phi"], z, f0["mu"])
    b = fem.pp_rhs(vs, z, z, np.zeros(N))
    times = []
    its = 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        A = fem.poisson(el, co, f0["phi"])
        x, its, rel = solvers.pcg(A, b, rtol=1e-8, mean_zero=True, maxit=100000)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    v = N / statistics.mean(times)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(times) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_nodes": int(N), "rtol": 1e-8},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": (f"per step: assembly + Jacobi-PCG ({its} its) of one "
                                    f"pressure-Poisson solve on the full mesh; host cores "
                                    f"{os.cpu_count()}")},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_apply_only(args):
    """Profiling aid: the roofline kernel alone (Poisson apply, FP32 coefficients and vectors)
    on the bench mesh, a few launches from a cold L2, with one timing line."""
    import torch

    from chns_workloads import configs
    from paper_2107_05123_gb300 import capi
    from paper_2107_05123_gb300.session import Mesh

    w = configs.rising_drop(5, 8)
    mesh = Mesh(w.anchors, w.levels, w.extent)
    f0 = w.init(mesh.node_xyz)
    prm = capi.make_params(w.params.as_dict())
    coef = capi.make_coef(torch.as_tensor(f0["phi"], device="cuda").float())
    x = torch.randn(mesh.n_nodes, device="cuda")
    y = torch.empty_like(x)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    ts = []
    for i in range(args.steps + args.warmup):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        capi.chns_apply_poisson(mesh.handle, prm, coef, x, y, capi.FP32)
        e1.record()
        torch.cuda.synchronize()
        if i >= args.warmup:
            ts.append(e0.elapsed_time(e1))
    print(json.dumps({"mode": "apply", "n_elem": mesh.n_elem, "n_nodes": mesh.n_nodes,
                      "ms": statistics.mean(ts)}))


def run_pp_only(args):
    """Profiling aid: pressure-Poisson solves alone (headline precision) on the bench mesh, with
    the right-hand side of the initial state, inside an NVTX range "pp_solve"."""
    import torch

    from chns_workloads import configs
    from paper_2107_05123_gb300 import capi
    from paper_2107_05123_gb300.session import Mesh

    w = configs.rising_drop(5, 8)
    mesh = Mesh(w.anchors, w.levels, w.extent)
    N = mesh.n_nodes
    f0 = w.init(mesh.node_xyz)
    prm = capi.make_params(w.params.as_dict())
    phit = torch.as_tensor(f0["phi"], device="cuda")
    zero3 = [torch.zeros(N, dtype=torch.float64, device="cuda") for _ in range(3)]
    b = torch.zeros(N, dtype=torch.float64, device="cuda")
    capi.chns_rhs_poisson(mesh.handle, prm,
                          capi.make_coef(phit, zero3, torch.as_tensor(f0["mu"], device="cuda")),
                          zero3, zero3, torch.zeros_like(b), b)
    solver = capi.make_solver(capi.KSP_CG, capi.PC_JACOBI, 1e-8, 20000, 30, capi.FP32, 1e-6, 30,
                              check_every=8)
    x = torch.zeros_like(b)
    res = []
    for i in range(args.steps + args.warmup):
        x.zero_()
        torch.cuda.synchronize()
        if i >= args.warmup:
            torch.cuda.nvtx.range_push("pp_solve")
        st = capi.chns_krylov_solve(mesh.handle, capi.OP_POISSON, prm, capi.make_coef(phit), b, x,
                                    solver)
        if i >= args.warmup:
            torch.cuda.nvtx.range_pop()
            res.append((st.ms, st.iterations, st.refinements, st.rel_residual))
    print(json.dumps({"mode": "pp", "n_nodes": N, "solves": res}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-budget", type=float, default=30.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--paths", choices=["both", "headline", "plain"], default="both",
                    help="time only one path and print a detail line (profiling runs)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the roofline kernel from an ncu capture")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the Rayleigh-Taylor workload at scale (~7e6 leaves)")
    ap.add_argument("--large-steps", type=int, default=2,
                    help="mixed-precision time steps of the Rayleigh-Taylor workload")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-preconditioner measurement (8-drop workload)")
    ap.add_argument("--learned-steps", type=int, default=3,
                    help="time steps whose pressure-Poisson solves give the training pairs")
    ap.add_argument("--learned-iters", type=int, default=6000, help="training iterations")
    ap.add_argument("--learned-lr", type=float, default=3e-4)
    ap.add_argument("--learned-grid", type=int, default=64, help="grid size D of the network")
    ap.add_argument("--mode", choices=["bench", "apply", "pp", "large", "learned"], default="bench",
                    help="apply / pp: time only the roofline kernel / the Poisson solve "
                         "(profiling); large / learned: only that part of the bench line")
    args = ap.parse_args()
    if args.mode == "apply":
        run_apply_only(args)
    elif args.mode == "pp":
        run_pp_only(args)
    elif args.mode == "large":
        print(json.dumps(run_large(args)))
    elif args.mode == "learned":
        print(json.dumps(run_learned(args)))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
