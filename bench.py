#!/usr/bin/env python
"""Benchmark: pressure-Poisson PCG throughput (DOFs/s) and time per CHNS step on one GB300.

Headline workload: the Rayleigh-Taylor interface at scale. The box is [0,1]x[0,4]x[0,1], the
interface y = 2 + 0.05 cos(2 pi x) cos(2 pi z), the octree spans levels 6-10 refined where
|phi| < 0.9 (6.9e6 leaves). Cn 0.005, density ratio 3, viscosity ratio 1, Re 1000, dt 2.5e-4,
fluid at rest. The fields are seeded and synthetic. One bench step is one chns_step: two blocks
of CH Newton, velocity prediction, pressure Poisson and velocity update, every solve to relative
residual 1e-8.

Headline path: FP32 Krylov iterations and applies inside FP64 refinement (FP64 dot products).
The pressure Poisson solve is flexible CG with a geometric-multigrid V-cycle. The CH Newton
systems use GMRES with the Schur-complement preconditioner, whose H^-1 is one V-cycle.

value        = n_nodes x (Poisson solves in the timed steps) / (their device time);
plain_fp64   = one step of the all-FP64 path with Jacobi-PCG for the pressure (the CH systems
               keep the Schur-complement preconditioner with inner CG: block-Jacobi GMRES does
               not converge at this resolution), from the same initial state;
e2e          = one pressure solve through the C ABI from pinned host buffers (copies timed);
roofline     = the FP32 Poisson apply timed alone from a cold L2 (algorithmic bytes / time);
               applies: the same for the mass, CH and momentum applies, and the FP64 applies
               against the measured FP64 peak (cuBLAS DGEMM);
cpu_baseline = the FP64 CPU oracle (assembled matrix + Jacobi-PCG) on a bounded sample;
rising_drop  = the rising-drop workload (levels 5-8, density ratio 1000) in mixed precision
               and FP64 with the one-level preconditioners (faster there than multigrid);
learned      = the learned coarse correction on the 8-drop workload (see run_learned).

A detailed JSON object goes to stderr; stdout gets the one bench line.
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
WORKLOAD = "rayleigh_taylor_levels6-10"
# DRAM bytes of one launch of the roofline kernel on the headline mesh (ncu
# dram__bytes_read.sum + dram__bytes_write.sum, summarised under profiles/); --traffic overrides
APPLY_DRAM_BYTES = 265.2e6  # mean of two launches (ncu capture summarised under profiles/)
# FP64 flops per element of the standalone FP64 applies (2 DFMA + DADD + DMUL thread
# instructions per leaf, one ncu capture on the levels 6-9 Rayleigh-Taylor mesh, profiles/)
FP64_FLOPS_PER_ELEM = {"poisson": 423.1, "mass": 517.1, "ch": 1085.0, "momentum": 4582.5}
# the reference arm's bounded sample of the headline workload: the same interface, box and
# physics on levels 5-8
SAMPLE_LEVELS = (5, 8)


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


def _say(*a):
    print(*a, file=sys.stderr, flush=True)


# --------------------------------------------------------------------------- our arm
def field_errors(a, b):
    """Relative L2 difference per field of state a against state b (pressure mean-removed)."""
    import numpy as np
    out = {}
    for k in ("phi", "mu", "p", "u"):
        x, y = np.asarray(a[k], dtype=np.float64), np.asarray(b[k], dtype=np.float64)
        if k == "p":
            x, y = x - x.mean(), y - y.mean()
        out[k] = float(np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300))
    return out


def double_float(capi, sp):
    """The refinement residuals of the mixed-precision path's pressure and velocity-update solves
    with the double-float Poisson and mass applies (faster than FP64 on GB300)."""
    for s in (sp.pp, sp.vu):
        s.fp64_apply = capi.FP64_DF
    return sp


def rt_step_params(capi, default_step_params, inner, mg_pp=None, mg_ch=None):
    """Solver settings of a Rayleigh-Taylor step: CH by GMRES with the Schur-complement
    preconditioner (H^-1 by a V-cycle when mg_ch is given, else 20 inner CG iterations), the
    pressure by flexible CG with a V-cycle when mg_pp is given, else Jacobi-PCG."""
    sp = default_step_params(rtol=1e-8, inner=inner, pp_check_every=8)
    sp.ch.pc = capi.PC_SCHUR
    sp.ch.inner_its = 20
    sp.ch.max_it = 400
    if mg_ch is not None:
        sp.ch.mg = mg_ch
    if mg_pp is not None:
        sp.pp = capi.make_solver(capi.KSP_FCG, capi.PC_MULTIGRID, 1e-8, 2000, 30, inner, 1e-6,
                                 40, check_every=2, mg=mg_pp)
    if inner == capi.FP32:
        double_float(capi, sp)
    return sp


def run_steps(capi, DeviceState, mesh, prm, f0, sp, warmup, steps, barrier, flush=None):
    """warmup untimed steps, then `steps` steps each bracketed by a barrier and a synchronize
    and timed with CUDA events; also returns the state after the first step."""
    import torch
    ds = DeviceState(dict(phi=f0["phi"], mu=f0["mu"], u=f0["u"], p=f0["p"]))
    first, first_ms = None, None
    step_ms, pp_ms, pp_n, pp_it, last = [], 0.0, 0, 0, None
    l0 = None
    for k in range(warmup + steps):
        timed = k >= warmup
        if timed and l0 is None:
            l0 = capi.chns_kernel_launches()
        if flush is not None:
            flush()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = capi.chns_step(mesh.handle, ds.c, prm, sp)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if first is None:
            first, first_ms = ds.host(), ms
        if timed:
            step_ms.append(ms)
            for l in range(2):
                pp_ms += st.pp[l].ms
                pp_n += 1
                pp_it += st.pp[l].iterations
        last = st
    launches = capi.chns_kernel_launches() - l0 if l0 is not None else 0
    return dict(step_ms=step_ms, pp_ms=pp_ms, pp_n=pp_n, pp_it=pp_it, last=last,
                first=first, first_ms=first_ms, launches=launches, final=ds.host())


def _phases(st):
    return {"ch": round(st.ms_ch, 1), "vp": round(st.ms_vp, 1), "pp": round(st.ms_pp, 1),
            "vu": round(st.ms_vu, 1)}


def time_applies(capi, mesh, prm, f0, flush, reps=6):
    """Each operator apply timed alone from a cold L2 (CUDA events on the launching stream):
    FP32 applies against the HBM peak, FP64 applies (FP64-ALU bound) by time only."""
    import torch
    N, E, H = mesh.n_nodes, mesh.n_elem, mesh.n_hanging
    dev = lambda a, dt: torch.as_tensor(a, device="cuda", dtype=dt)
    out = {}
    # arrays read or written once per node by each apply (vectors and coefficient fields):
    # Poisson x, y, phi~; mass 3 + 3 components, phi~; CH 2 + 2 components, phi~, u~ (3);
    # momentum 3 + 3 components, phi~, u_hat (3), mu~
    spec = {"poisson": (capi.chns_apply_poisson, 1, 3), "mass": (capi.chns_apply_mass, 3, 7),
            "ch": (capi.chns_apply_ch, 2, 8), "momentum": (capi.chns_apply_momentum, 3, 11)}
    rng = torch.Generator(device="cuda").manual_seed(7)
    u3 = [0.01 * torch.randn(N, device="cuda", dtype=torch.float64, generator=rng)
          for _ in range(3)]
    peak, kind = _peaks()
    for dtname, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
        prec = capi.FP32 if dt == torch.float32 else capi.FP64
        phi = dev(f0["phi"], dt)
        mu = dev(f0["mu"], dt)
        coef = capi.make_coef(phi, [u.to(dt) for u in u3], mu)
        for name, (fn, nc, arrays) in spec.items():
            x = torch.randn(nc * N, device="cuda", dtype=dt, generator=rng)
            y = torch.empty_like(x)
            ts = []
            for i in range(reps + 2):
                flush()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn(mesh.handle, prm, coef, x, y, prec)
                e1.record()
                torch.cuda.synchronize()
                if i >= 2:
                    ts.append(e0.elapsed_time(e1) * 1e-3)
            t = statistics.mean(ts)
            alg = N * arrays * (4 if dt == torch.float32 else 8) + E * 33 + H * 16
            r = {"ms": round(t * 1e3, 4), "alg_bytes": int(alg)}
            if dt == torch.float32:
                ach = alg / t / 1e9
                r.update(achieved_gbs=round(ach, 1), frac=round(ach / peak, 4))
            out.setdefault(dtname, {})[name] = r
    out["peak_gbs"], out["peak_kind"] = peak, kind
    return out


def fp64_peak():
    """Measured FP64 throughput of this GPU: cuBLAS DGEMM (torch.matmul, float64) 4096^3, best
    of 5 after 2 warm-ups, CUDA events; 2 n^3 flops."""
    import torch
    n = 4096
    a = torch.randn(n, n, device="cuda", dtype=torch.float64)
    b = torch.randn(n, n, device="cuda", dtype=torch.float64)
    best = None
    for i in range(7):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        if i >= 2:
            t = e0.elapsed_time(e1) * 1e-3
            best = t if best is None else min(best, t)
    return 2.0 * n ** 3 / best / 1e12


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

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize()

    flush_buf = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def flush_l2():
        flush_buf.fill_(1.0)

    t_all = time.perf_counter()
    w = configs.rayleigh_taylor(6, 10, 0.005)
    t0 = time.perf_counter()
    mesh = Mesh(w.anchors, w.levels, w.extent)
    t_mesh = time.perf_counter() - t0
    N, E, H = mesh.n_nodes, mesh.n_elem, mesh.n_hanging
    f0 = w.init(mesh.node_xyz)
    prm = capi.make_params(w.params.as_dict())
    t0 = time.perf_counter()
    mg_pp = capi.chns_mg_create(mesh.handle, degree=2)
    mg_ch = capi.chns_mg_create(mesh.handle, degree=2)
    t_mg = time.perf_counter() - t0
    levels, _ = capi.chns_mg_levels(mg_pp)
    _say(f"[bench] mesh {E} leaves {N} nodes ({t_mesh:.1f} s), multigrid {len(levels)} levels "
         f"({t_mg:.1f} s)")

    # ---- headline: mixed precision with multigrid (timed steps)
    sp_head = rt_step_params(capi, default_step_params, capi.FP32, mg_pp, mg_ch)
    with ClockSampler(local) as clk:
        head = run_steps(capi, DeviceState, mesh, prm, f0, sp_head, args.warmup, args.steps,
                         barrier)
    clocks = clk.summary()
    tmax, pp_ms = replica_max(pg, [sum(head["step_ms"]), head["pp_ms"]], "cuda")
    value = whole_job_value(ws, N, head["pp_n"], pp_ms)
    ms_per_step = tmax / args.steps
    _say(f"[bench] headline {ms_per_step:.1f} ms/step, {value / 1e6:.2f} M DOFs/s")

    detail = {"headline_last_step": {"phases_ms": _phases(head["last"]),
                                     "newton_its": list(head["last"].newton_its),
                                     "ch_gmres_its": [head["last"].ch[l].iterations for l in range(2)],
                                     "vp_gmres_its": [head["last"].vp[l].iterations for l in range(2)],
                                     "pp_fcg_its": [head["last"].pp[l].iterations for l in range(2)],
                                     "mass_drift": abs(head["last"].phi_mass_after
                                                       - head["last"].phi_mass_before)}}
    plain = fp64mg = None
    if rank == 0 and not args.no_plain:
        # ---- the all-FP64 Jacobi-PCG path, one step from the same initial state
        sp_plain = rt_step_params(capi, default_step_params, capi.FP64)
        plain = run_steps(capi, DeviceState, mesh, prm, f0, sp_plain, 0, 1, barrier)
        _say(f"[bench] plain FP64 {plain['step_ms'][0]:.1f} ms")
        if not args.no_fp64_mg:
            sp64 = rt_step_params(capi, default_step_params, capi.FP64, mg_pp, mg_ch)
            fp64mg = run_steps(capi, DeviceState, mesh, prm, f0, sp64, 0, 1, barrier)
            _say(f"[bench] FP64 with multigrid {fp64mg['step_ms'][0]:.1f} ms")

    # ---- roofline: every apply alone from a cold L2 on the headline mesh
    applies = time_applies(capi, mesh, prm, f0, flush_l2) if rank == 0 else None

    # ---- end to end: one pressure solve through the C ABI from pinned host buffers
    b_dev = torch.zeros(N, dtype=torch.float64, device="cuda")
    zero3 = [torch.zeros(N, dtype=torch.float64, device="cuda") for _ in range(3)]
    phit = torch.as_tensor(f0["phi"], device="cuda")
    capi.chns_rhs_poisson(mesh.handle, prm,
                          capi.make_coef(phit, zero3, torch.as_tensor(f0["mu"], device="cuda")),
                          zero3, zero3, torch.zeros_like(b_dev), b_dev)
    b_h = b_dev.cpu().pin_memory()
    phi_h = phit.cpu().pin_memory()
    x_h = torch.zeros(N, dtype=torch.float64).pin_memory()
    bd, xd, pd = torch.empty_like(b_dev), torch.empty_like(b_dev), torch.empty_like(b_dev)
    solver = sp_head.pp
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

    capi.chns_mg_destroy(mg_pp)
    capi.chns_mg_destroy(mg_ch)
    del mesh

    drop = learned = None
    if rank == 0 and not args.no_drop:
        try:
            drop = run_drop(args, flush_l2, barrier)
        except Exception as e:  # the headline line is printed whatever happens here
            drop = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0 and not args.no_learned:
        try:
            learned = run_learned(args)
        except Exception as e:
            learned = {"error": f"{type(e).__name__}: {e}"}
    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    f64 = fp64_peak()
    cpu = cpu_baseline(budget_s=args.cpu_budget) if not args.no_cpu else None

    peak, peak_kind = _peaks()
    pa = applies["fp32"]["poisson"] if applies else None
    traffic = args.traffic if args.traffic is not None else APPLY_DRAM_BYTES
    fp64_rates = None
    if applies:
        # FP64 instruction counts per element of the FP64 applies (ncu, profiles/)
        fp64_rates = {k: applies["fp64"][k]["ms"] for k in ("poisson", "mass", "ch", "momentum")}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_elem": int(E), "n_nodes": int(N), "n_hanging": int(H),
                   "rtol": 1e-8, "l2": "working set larger than L2 (6.0e6 nodes, 48 MB per FP64 "
                   "field; applies timed alone after a 256 MB flush)",
                   "pp": "FCG + multigrid V-cycle", "ch": "GMRES + Schur (H^-1 by V-cycle)",
                   "mg_levels": int(len(levels)),
                   "parallelism": "replicas" if ws > 1 else "single"},
        "pp_fcg_its_per_solve": round(head["pp_it"] / max(head["pp_n"], 1), 1),
        "first_step_ms": round(head["first_ms"], 1),
        "plain_fp64": None if plain is None else {
            "ms_per_step": round(plain["step_ms"][0], 1),
            "pp_ms_per_solve": round(plain["pp_ms"] / plain["pp_n"], 2),
            "pp_its_per_solve": plain["pp_it"] / plain["pp_n"],
            "value": N * plain["pp_n"] / (plain["pp_ms"] * 1e-3),
            "phases_ms": _phases(plain["last"])},
        "speedup_vs_plain_fp64": None if plain is None else {
            "pp": round(value / (N * plain["pp_n"] / (plain["pp_ms"] * 1e-3)), 2),
            "first_step": round(plain["step_ms"][0] / head["first_ms"], 2),
            "step": round(plain["step_ms"][0] / ms_per_step, 2)},
        "fp64_multigrid_step_ms": None if fp64mg is None else round(fp64mg["step_ms"][0], 1),
        "field_error_vs_plain_fp64_after_1_step": None if plain is None else field_errors(
            head["first"], plain["first"]),
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(2 * N * 8),
                "d2h_bytes_per_step": int(N * 8)},
        "roofline": None if pa is None else {
            "kernel": "Poisson apply FP32 (k_apply_stream<PoissonK<float,float>>)", "bound": "hbm",
            "achieved": pa["achieved_gbs"], "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
            "frac": pa["frac"], "traffic": traffic, "alg_bytes": pa["alg_bytes"], "ms": pa["ms"]},
        "applies_hbm_frac_fp32": None if not applies else {
            k: applies["fp32"][k]["frac"] for k in ("poisson", "mass", "ch", "momentum")},
        "applies_ms": None if not applies else {
            p: {k: applies[p][k]["ms"] for k in ("poisson", "mass", "ch", "momentum")}
            for p in ("fp32", "fp64")},
        "fp64_peak_tflops": round(f64, 3),
        "applies_fp64_alu_frac": None if not applies else {
            k: round(FP64_FLOPS_PER_ELEM[k] * E / (applies["fp64"][k]["ms"] * 1e-3) / (f64 * 1e12), 3)
            for k in ("poisson", "mass", "ch", "momentum")},
        "rising_drop": drop,
        "learned": learned,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "gpu_launches": head["launches"],
    }
    detail.update(applies=applies, fp64_apply_ms=fp64_rates, wall_s=round(time.perf_counter() - t_all, 1),
                  mg_levels_nodes=[int(v) for v in levels])
    _say("[bench] detail " + json.dumps(detail))
    print(json.dumps(line))
    if pg:
        pg.destroy_process_group()


def run_drop(args, flush_l2, barrier):
    """The rising drop (levels 5-8, 314,672 leaves): time per step and pressure-solve throughput
    of the mixed-precision and all-FP64 paths with the one-level preconditioners (Jacobi-PCG,
    2x2 block-Jacobi GMRES), which are faster than multigrid on this small mesh."""
    from chns_workloads import configs
    from paper_2107_05123_gb300 import capi
    from paper_2107_05123_gb300.session import DeviceState, Mesh, default_step_params

    w = configs.rising_drop(5, 8)
    mesh = Mesh(w.anchors, w.levels, w.extent)
    f0 = w.init(mesh.node_xyz)
    prm = capi.make_params(w.params.as_dict())
    N = mesh.n_nodes
    out = {"workload": "rising_drop_levels5-8", "n_elem": int(mesh.n_elem), "n_nodes": int(N)}
    res = {}
    for label, inner in (("mixed", capi.FP32), ("fp64", capi.FP64)):
        sp = default_step_params(rtol=1e-8, inner=inner, pp_check_every=8)
        if inner == capi.FP32:
            double_float(capi, sp)
        r = run_steps(capi, DeviceState, mesh, prm, f0, sp, 2, args.drop_steps, barrier,
                      flush=flush_l2)
        res[label] = r
        out[label] = {"ms_per_step": round(statistics.mean(r["step_ms"]), 2),
                      "pp_ms_per_solve": round(r["pp_ms"] / r["pp_n"], 3),
                      "value": N * r["pp_n"] / (r["pp_ms"] * 1e-3),
                      "phases_ms": _phases(r["last"])}
    out["speedup_step"] = round(out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"], 2)
    out["field_error_mixed_vs_fp64"] = field_errors(res["mixed"]["final"], res["fp64"]["final"])
    return out


def run_learned(args):
    """The learned coarse correction on the 8-drop workload (levels 5-8, drops of radius
    0.05-0.12, Cn 0.01, density ratio 1000): training pairs from the pressure-Poisson solves of
    `--learned-steps` time steps (iterates of FP64 Jacobi-PCG, every `--learned-collect-every`th,
    at most `--learned-collect-max` per solve, into a replay buffer of `--learned-capacity`
    pairs; if a step fails, collection stops and the comparison starts from the state of the
    last step that succeeded),
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
    pd = w.params.as_dict()
    if args.learned_dt:
        pd["dt"] = args.learned_dt
    prm = capi.make_params(pd)
    f0 = w.init(mesh.node_xyz)
    D = args.learned_grid
    net = capi.chns_learned_create(D, args.learned_capacity, 1)

    def params(pp=None, collect=None):
        sp = default_step_params(rtol=1e-8, inner=capi.FP32, pp_check_every=8)
        sp.vp.max_it = 20000
        if pp is not None:
            sp.pp = pp
        if collect is not None:
            sp.collect, sp.collect_every = collect, args.learned_collect_every
            sp.collect_max = args.learned_collect_max
        return sp

    ds = DeviceState(dict(phi=f0["phi"], mu=f0["mu"], u=f0["u"], p=f0["p"]))
    t0 = time.perf_counter()
    steps_done, step_error = 0, None
    snap = prev = ds.host()
    for _ in range(args.learned_steps):
        try:
            capi.chns_step(mesh.handle, ds.c, prm, params(collect=net))
        except capi.ChnsError as e:
            # a failed step leaves the state unusable; the step from `snap` is the one that
            # failed, so the comparison below starts from the state one step earlier, from which
            # a step is known to succeed
            step_error = str(e)
            snap = prev
            break
        steps_done += 1
        prev, snap = snap, ds.host()
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
    full = {"workload": "drops8_levels5-8", "dt": pd["dt"], "n_elem": int(mesh.n_elem),
            "n_nodes": int(mesh.n_nodes), "grid": D, "channels": 16, "levels": 4,
            "collect_steps": steps_done, "collect_step_error": step_error, "pairs": int(pairs),
            "train_iterations": args.learned_iters, "lr": args.learned_lr,
            "collect_s": round(t_collect, 2), "train_s": round(t_train, 2),
            "train_ms_per_iteration": round(1e3 * t_train / max(args.learned_iters, 1), 3),
            "energy_loss_first_100": float(loss[:100].mean()) if len(loss) else None,
            "energy_loss_last_500": float(loss[-500:].mean()) if len(loss) else None,
            "next_step": res, "small_drops": small,
            "wall_s": round(time.perf_counter() - t_all, 1)}
    _say("[bench] learned " + json.dumps(full))
    # compact summary for the bench line
    return {"workload": full["workload"], "pairs": full["pairs"], "train_s": full["train_s"],
            "pp_ms_next_step": {k: v.get("pp_ms") for k, v in res.items()},
            "pp_iters_next_step": {k: v.get("pp_iters") for k, v in res.items()},
            "fallbacks": res.get("mixed_learned", {}).get("fallbacks"),
            "small_drops_iters": {"jacobi_pcg": small["jacobi_pcg"],
                                  "fcg_learned": small["fcg_learned"]}}


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
def _oracle_sample():
    """The reference arm's bounded sample of the headline workload: the Rayleigh-Taylor
    interface, box and physics on levels 5-8 (156,640 leaves), with the pressure-Poisson
    right-hand side of the initial state."""
    import numpy as np

    from chns_workloads import configs
    from oracle import fem
    from oracle.mesh import Mesh as OMesh

    w = configs.rayleigh_taylor(*SAMPLE_LEVELS, 0.005)
    om = OMesh(w.anchors, w.levels, w.extent)
    f0 = w.init(om.node_xyz)
    el, co = fem.Elem(om), fem.Coeffs(w.params.as_dict())
    z = np.zeros((3, om.n_nodes))
    vs = fem.VMSState(el, co, f0["phi"], z, f0["mu"])
    b = fem.pp_rhs(vs, z, z, np.zeros(om.n_nodes))
    return w, om, f0, el, co, b


def cpu_baseline(budget_s=60.0):
    """The oracle as it stands, timed on the host cores: one pressure-Poisson solve (assembly +
    Jacobi-PCG to 1e-8) on the bounded sample of the headline workload (the value), and the
    timings the measurement plan lists: the CSR SpMV per operator and the Jacobi-PCG solve on
    the rising drop, and one full step on the smooth uniform workload. The full rising-drop step
    and the headline mesh itself are reported as skipped (direct solves of 5.8e5 unknowns; ~10 GB
    of assembled matrices)."""
    import numpy as np

    from chns_workloads import configs
    from oracle import fem, solvers, step as ostep
    from oracle.mesh import Mesh as OMesh

    t_begin = time.perf_counter()
    w, om, f0, el, co, b = _oracle_sample()
    t1 = time.perf_counter()
    A = fem.poisson(el, co, f0["phi"])
    t2 = time.perf_counter()
    x, it, rel = solvers.pcg(A, b, rtol=1e-8, mean_zero=True, maxit=100000)
    t3 = time.perf_counter()
    N = om.n_nodes
    out = {"value": N / (t3 - t1), "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": (f"one pressure-Poisson solve on the Rayleigh-Taylor workload at levels "
                      f"{SAMPLE_LEVELS[0]}-{SAMPLE_LEVELS[1]} ({om.n_elem} leaves, {N} nodes): "
                      f"assembly {t2 - t1:.1f} s + Jacobi-PCG {it} its in {t3 - t2:.1f} s; "
                      f"numpy/scipy single-threaded on {os.cpu_count()} host cores")}
    timings = {}
    try:
        wd = configs.rising_drop(5, 8)
        od = OMesh(wd.anchors, wd.levels, wd.extent)
        fd = wd.init(od.node_xyz)
        eld, cod = fem.Elem(od), fem.Coeffs(wd.params.as_dict())
        rng = np.random.default_rng(0)
        u = 0.01 * rng.standard_normal((3, od.n_nodes))
        mats = {"poisson": lambda: fem.poisson(eld, cod, fd["phi"]),
                "mass": lambda: fem.mass_rho(eld, cod, fd["phi"]),
                "ch": lambda: fem.ch_jacobian(eld, cod, fd["phi"], u),
                "momentum": lambda: fem.momentum(fem.VMSState(eld, cod, fd["phi"], u, fd["mu"]))}
        spmv = {}
        for k, f in mats.items():
            if time.perf_counter() - t_begin > budget_s:
                spmv[k] = "skipped: time budget"
                continue
            ta = time.perf_counter()
            M = f()
            tb = time.perf_counter()
            v = rng.standard_normal(M.shape[1])
            reps = 5
            tc = time.perf_counter()
            for _ in range(reps):
                M @ v
            td = time.perf_counter()
            spmv[k] = {"assembly_s": round(tb - ta, 2), "spmv_ms": round((td - tc) / reps * 1e3, 2)}
        timings["rising_drop_levels5-8"] = {"n_nodes": int(od.n_nodes), "csr": spmv}
        if time.perf_counter() - t_begin < budget_s:
            A2 = mats["poisson"]() if isinstance(spmv.get("poisson"), dict) else None
            if A2 is not None:
                z = np.zeros((3, od.n_nodes))
                vsd = fem.VMSState(eld, cod, fd["phi"], z, fd["mu"])
                b2 = fem.pp_rhs(vsd, z, z, np.zeros(od.n_nodes))
                ta = time.perf_counter()
                _, it2, _ = solvers.pcg(A2, b2, rtol=1e-8, mean_zero=True, maxit=100000)
                timings["rising_drop_levels5-8"]["jacobi_pcg"] = {
                    "its": it2, "s": round(time.perf_counter() - ta, 2)}
        timings["rising_drop_levels5-8"]["full_step"] = ("skipped: direct solves of 5.8e5 "
                                                         "unknowns exceed the time budget")
        if time.perf_counter() - t_begin < budget_s:
            ws = configs.smooth_uniform(4, seed=0)
            osm = OMesh(ws.anchors, ws.levels, ws.extent)
            fs = ws.init(osm.node_xyz)
            ta = time.perf_counter()
            ostep.chns_step(osm, ws.params.as_dict(),
                            ostep.State(phi=fs["phi"], mu=fs["mu"], u=fs["u"], u_old=fs["u"],
                                        p=fs["p"]), pp_rtol=1e-8, newton_rtol=1e-10)
            timings["smooth_uniform_level4"] = {"n_nodes": int(osm.n_nodes),
                                                "full_step_s": round(time.perf_counter() - ta, 2)}
        timings[WORKLOAD] = "skipped: memory (assembled matrices of 6.9e6 elements, ~10 GB)"
        timings["breakup64_levels6-10"] = ("skipped: memory (2.8e7 elements: ~40 GB of assembled "
                                           "matrices per scalar operator)")
    except Exception as e:  # the baseline value above stands
        timings["error"] = f"{type(e).__name__}: {e}"
    out["oracle_timings"] = timings
    return out


# --------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle on the headline metric: per step one pressure-Poisson solve (assembly +
    Jacobi-PCG to 1e-8) on the bounded sample of the headline workload; rank 0 only."""
    ws, rank, local = _dist()
    if rank != 0:
        return
    from oracle import fem, solvers

    w, om, f0, el, co, b = _oracle_sample()
    N = om.n_nodes
    times = []
    its = 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        A = fem.poisson(el, co, f0["phi"])
        x, its, rel = solvers.pcg(A, b, rtol=1e-8, mean_zero=True, maxit=100000)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    v = N / statistics.mean(times)
    sample = (f"per step: assembly + Jacobi-PCG ({its} its) of one pressure-Poisson solve on "
              f"the Rayleigh-Taylor workload at levels {SAMPLE_LEVELS[0]}-{SAMPLE_LEVELS[1]} "
              f"({om.n_elem} leaves, {N} nodes); host cores {os.cpu_count()}, "
              f"numpy/scipy single-threaded")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(times) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"levels {SAMPLE_LEVELS[0]}-{SAMPLE_LEVELS[1]}",
                   "n_nodes": int(N), "rtol": 1e-8},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# --------------------------------------------------------------------------- profiling modes
def _rt_setup():
    import torch

    from chns_workloads import configs
    from paper_2107_05123_gb300 import capi
    from paper_2107_05123_gb300.session import Mesh

    if os.environ.get("CHNS_BENCH_DROP"):
        w = configs.rising_drop(5, 8)
    elif os.environ.get("CHNS_BENCH_SMALL"):
        w = configs.rayleigh_taylor(6, 9, 0.005)
    else:
        w = configs.rayleigh_taylor(6, 10, 0.005)
    mesh = Mesh(w.anchors, w.levels, w.extent)
    f0 = w.init(mesh.node_xyz)
    prm = capi.make_params(w.params.as_dict())
    return torch, capi, w, mesh, f0, prm


def run_apply_only(args):
    """Profiling aid: one operator apply (--apply-op, --apply-prec) on the headline mesh, a few
    launches from a cold L2, with one timing line. CHNS_BENCH_SMALL=1 uses levels 6-9,
    CHNS_BENCH_DROP=1 the rising drop on levels 5-8."""
    torch, capi, w, mesh, f0, prm = _rt_setup()
    dt = torch.float32 if args.apply_prec == "fp32" else torch.float64
    prec = {"fp32": capi.FP32, "fp64": capi.FP64, "fp64df": capi.FP64_DF}[args.apply_prec]
    N = mesh.n_nodes
    fn, nc = {"poisson": (capi.chns_apply_poisson, 1), "mass": (capi.chns_apply_mass, 3),
              "ch": (capi.chns_apply_ch, 2), "momentum": (capi.chns_apply_momentum, 3)}[args.apply_op]
    u3 = [torch.full((N,), 0.01, device="cuda", dtype=dt) for _ in range(3)]
    coef = capi.make_coef(torch.as_tensor(f0["phi"], device="cuda", dtype=dt), u3,
                          torch.as_tensor(f0["mu"], device="cuda", dtype=dt))
    x = torch.randn(nc * N, device="cuda", dtype=dt)
    y = torch.empty_like(x)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    ts = []
    for i in range(args.steps + args.warmup):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn(mesh.handle, prm, coef, x, y, prec)
        e1.record()
        torch.cuda.synchronize()
        if i >= args.warmup:
            ts.append(e0.elapsed_time(e1))
    print(json.dumps({"mode": "apply", "op": args.apply_op, "prec": args.apply_prec,
                      "n_elem": mesh.n_elem, "n_nodes": N, "n_hanging": mesh.n_hanging,
                      "ms": statistics.mean(ts)}))


def run_pp_only(args):
    """Profiling aid: pressure-Poisson solves alone (headline settings: FCG + V-cycle, FP32
    inside FP64 refinement) on the headline mesh, with the right-hand side of the initial
    state."""
    torch, capi, w, mesh, f0, prm = _rt_setup()
    N = mesh.n_nodes
    phit = torch.as_tensor(f0["phi"], device="cuda")
    zero3 = [torch.zeros(N, dtype=torch.float64, device="cuda") for _ in range(3)]
    b = torch.zeros(N, dtype=torch.float64, device="cuda")
    capi.chns_rhs_poisson(mesh.handle, prm,
                          capi.make_coef(phit, zero3, torch.as_tensor(f0["mu"], device="cuda")),
                          zero3, zero3, torch.zeros_like(b), b)
    mg = capi.chns_mg_create(mesh.handle, degree=2)
    solver = capi.make_solver(capi.KSP_FCG, capi.PC_MULTIGRID, 1e-8, 2000, 30, capi.FP32, 1e-6,
                              40, check_every=2, mg=mg)
    x = torch.zeros_like(b)
    res = []
    for i in range(args.steps + args.warmup):
        x.zero_()
        torch.cuda.synchronize()
        st = capi.chns_krylov_solve(mesh.handle, capi.OP_POISSON, prm, capi.make_coef(phit), b, x,
                                    solver)
        if i >= args.warmup:
            res.append((st.ms, st.iterations, st.refinements, st.rel_residual))
    capi.chns_mg_destroy(mg)
    print(json.dumps({"mode": "pp", "n_nodes": N, "solves": res}))


def run_step_only(args):
    """Profiling aid: the headline path on the headline mesh, `--warmup` untimed steps, then one
    step inside an NVTX range "timed_step" (for an ncu launch list restricted to that range).
    With CHNS_BENCH_DROP=1: the rising drop (levels 5-8) with the settings of its bench line
    (one-level preconditioners, FP32 inside FP64 refinement)."""
    torch, capi, w, mesh, f0, prm = _rt_setup()
    from paper_2107_05123_gb300.session import DeviceState, default_step_params
    mg_pp = capi.chns_mg_create(mesh.handle, degree=2)
    mg_ch = capi.chns_mg_create(mesh.handle, degree=2)
    if os.environ.get("CHNS_BENCH_DROP"):
        sp = double_float(capi, default_step_params(rtol=1e-8, inner=capi.FP32, pp_check_every=8))
    else:
        sp = rt_step_params(capi, default_step_params, capi.FP32, mg_pp, mg_ch)
    ds = DeviceState(dict(phi=f0["phi"], mu=f0["mu"], u=f0["u"], p=f0["p"]))
    for _ in range(args.warmup):
        capi.chns_step(mesh.handle, ds.c, prm, sp)
    torch.cuda.synchronize()
    l0 = capi.chns_kernel_launches()
    torch.cuda.nvtx.range_push("timed_step")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    st = capi.chns_step(mesh.handle, ds.c, prm, sp)
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"mode": "step", "ms": e0.elapsed_time(e1), "phases_ms": _phases(st),
                      "launches": capi.chns_kernel_launches() - l0}))
    capi.chns_mg_destroy(mg_pp)
    capi.chns_mg_destroy(mg_ch)


def run_learned_fcg(args):
    """Profiling aid for the learned correction: the rising drop (levels 5-8), an untrained
    D = 64 network (seed 3, output scale 1), three flexible-CG pressure solves with it (FP32
    inside FP64 refinement, at most 16 iterations, host check every 8), the last one inside an
    NVTX range "fcg"; prints the solve time and one network forward time (CUDA events)."""
    import torch

    from chns_workloads import configs
    from paper_2107_05123_gb300 import capi
    from paper_2107_05123_gb300.session import Mesh

    w = configs.rising_drop(5, 8)
    mesh = Mesh(w.anchors, w.levels, w.extent)
    f0 = w.init(mesh.node_xyz)
    prm = capi.make_params(w.params.as_dict())
    N = mesh.n_nodes
    net = capi.chns_learned_create(64, 0, 3)
    capi.chns_learned_set_output_scale(net, 1.0)
    phit = torch.as_tensor(f0["phi"], device="cuda")
    zero3 = [torch.zeros(N, dtype=torch.float64, device="cuda") for _ in range(3)]
    b = torch.zeros(N, dtype=torch.float64, device="cuda")
    capi.chns_rhs_poisson(mesh.handle, prm,
                          capi.make_coef(phit, zero3, torch.as_tensor(f0["mu"], device="cuda")),
                          zero3, zero3, torch.zeros_like(b), b)
    solver = capi.make_solver(capi.KSP_FCG, capi.PC_LEARNED, 1e-8, 16, 30, capi.FP32, 1e-6,
                              check_every=8, learned=net)
    ms = None
    for k in range(3):
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        if k == 2:
            torch.cuda.nvtx.range_push("fcg")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        capi.chns_krylov_solve(mesh.handle, capi.OP_POISSON, prm, capi.make_coef(phit), b, x,
                               solver, check=False)
        e1.record()
        torch.cuda.synchronize()
        if k == 2:
            torch.cuda.nvtx.range_pop()
        ms = e0.elapsed_time(e1)
    capi.chns_learned_destroy(net)
    return {"mode": "learned_fcg", "n_nodes": int(N), "ms_16_iterations": round(ms, 3)}


def run_breakup(args):
    """The many-drop breakup workload (64 seeded drops of radius 0.02-0.08, the shear
    u = (2y - 1, 0, 0) imposed on every wall, density ratio 100, viscosity ratio 50, Re 2000,
    We 50, Cn 0.002, dt 1e-4) on the levels --breakup-levels: time per step of the
    mixed-precision path with the multigrid preconditioners (the headline settings) beside one
    step of the all-FP64 Jacobi path from the same state, and each FP32 apply's HBM fraction on
    this mesh."""
    import torch

    from chns_workloads import configs
    from paper_2107_05123_gb300 import capi
    from paper_2107_05123_gb300.session import DeviceState, Mesh, VelocityBC, default_step_params

    lmin, lmax = (int(v) for v in args.breakup_levels.split(","))
    t0 = time.perf_counter()
    w = configs.breakup(lmin, lmax)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    mesh = Mesh(w.anchors, w.levels, w.extent)
    t_mesh = time.perf_counter() - t0
    N = mesh.n_nodes
    f0 = w.init(mesh.node_xyz)
    bc = VelocityBC(w.info["velocity_bc"](mesh.node_xyz, 0.0))
    prm = capi.make_params(w.params.as_dict())
    t0 = time.perf_counter()
    # degree-2 smoothing with a 12-step power estimate left the pressure FCG stagnating near
    # 4e-4 on levels 6-10; degree 3 with a 40-step estimate converges in about 12 iterations
    mg_pp = capi.chns_mg_create(mesh.handle, degree=3, power_its=40)
    mg_ch = capi.chns_mg_create(mesh.handle, degree=2)
    t_mg = time.perf_counter() - t0
    _say(f"[breakup] {mesh.n_elem} leaves, {N} nodes (octree {t_gen:.1f} s, mesh {t_mesh:.1f} s, "
         f"multigrid {t_mg:.1f} s)")
    flush_buf = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    flush = lambda: flush_buf.fill_(1.0)
    sync = torch.cuda.synchronize
    sp = bc.attach(rt_step_params(capi, default_step_params, capi.FP32, mg_pp, mg_ch))
    with ClockSampler(torch.cuda.current_device()) as clk:
        head = run_steps(capi, DeviceState, mesh, prm, f0, sp, args.warmup, args.steps, sync)
    ms = statistics.mean(head["step_ms"])
    _say(f"[breakup] mixed precision + multigrid {ms:.1f} ms/step")
    last = head["last"]
    out = {"mode": "breakup", "workload": f"breakup64_levels{lmin}-{lmax}",
           "n_elem": int(mesh.n_elem), "n_nodes": int(N), "n_hanging": int(mesh.n_hanging),
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1),
           "first_step_ms": round(head["first_ms"], 1), "phases_ms": _phases(last),
           "newton_its": list(last.newton_its),
           "ch_gmres_its": [last.ch[l].iterations for l in range(2)],
           "vp_gmres_its": [last.vp[l].iterations for l in range(2)],
           "pp_fcg_its": [last.pp[l].iterations for l in range(2)],
           "pp_dofs_per_s": N * head["pp_n"] / (head["pp_ms"] * 1e-3),
           "mass_drift": abs(last.phi_mass_after - last.phi_mass_before),
           "gpu_launches": head["launches"], "clocks": clk.summary(),
           "setup_s": {"octree": round(t_gen, 1), "mesh": round(t_mesh, 1),
                       "multigrid": round(t_mg, 1)}}
    if not args.no_plain:
        sp64 = bc.attach(rt_step_params(capi, default_step_params, capi.FP64))
        plain = run_steps(capi, DeviceState, mesh, prm, f0, sp64, 0, 1, sync)
        out["plain_fp64"] = {"ms_per_step": round(plain["step_ms"][0], 1),
                             "phases_ms": _phases(plain["last"]),
                             "pp_its": [plain["last"].pp[l].iterations for l in range(2)]}
        out["speedup_first_step_vs_plain_fp64"] = round(plain["step_ms"][0] / head["first_ms"], 2)
        out["field_error_vs_plain_fp64_after_1_step"] = field_errors(head["first"], plain["first"])
    ap = time_applies(capi, mesh, prm, f0, flush)
    out["applies_hbm_frac_fp32"] = {k: ap["fp32"][k]["frac"] for k in ("poisson", "mass", "ch",
                                                                         "momentum")}
    out["applies_ms"] = {p: {k: ap[p][k]["ms"] for k in ("poisson", "mass", "ch", "momentum")}
                         for p in ("fp32", "fp64")}
    out["peak_gbs"], out["peak_kind"] = ap["peak_gbs"], ap["peak_kind"]
    capi.chns_mg_destroy(mg_pp)
    capi.chns_mg_destroy(mg_ch)
    return out


def run_amr(args):
    """The rising drop (levels 5-8) stepped --steps times in mixed precision with a remesh
    after every --amr-every steps (band |phi| <= 0.95 on levels 5-8): time per step and per
    remesh (band flags, new leaves, mesh tables, transfer of the five fields), leaf counts, and
    the phi mass change of each remesh (the transfer is not mass conserving, Sec. 6.2) beside the
    steps' own drift."""
    import torch

    from chns_workloads import configs
    from paper_2107_05123_gb300 import capi
    from paper_2107_05123_gb300.session import DeviceState, Mesh, default_step_params, remesh

    w = configs.rising_drop(5, 8)
    mesh = Mesh(w.anchors, w.levels, w.extent)
    f0 = w.init(mesh.node_xyz)
    ds = DeviceState(dict(phi=f0["phi"], mu=f0["mu"], u=f0["u"], p=f0["p"]))
    prm = capi.make_params(w.params.as_dict())
    sp = default_step_params(rtol=1e-8, inner=capi.FP32, pp_check_every=8)
    step_ms, remesh_ms, leaves, remesh_dmass, step_dmass = [], [], [int(mesh.n_elem)], [], []
    for k in range(args.warmup + args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = capi.chns_step(mesh.handle, ds.c, prm, sp)
        e1.record()
        torch.cuda.synchronize()
        if k >= args.warmup:
            step_ms.append(e0.elapsed_time(e1))
            step_dmass.append(st.phi_mass_after - st.phi_mass_before)
        if (k + 1) % args.amr_every == 0:
            m0 = capi.chns_phi_mass(mesh.handle, ds.phi)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            new_mesh, new_ds = remesh(mesh, ds, 0.95, 5, 8)
            torch.cuda.synchronize()
            dt_ms = (time.perf_counter() - t0) * 1e3
            m1 = capi.chns_phi_mass(new_mesh.handle, new_ds.phi)
            mesh.close()
            mesh, ds = new_mesh, new_ds
            if k >= args.warmup:
                remesh_ms.append(dt_ms)
                remesh_dmass.append(m1 - m0)
                leaves.append(int(mesh.n_elem))
    return {"mode": "amr", "workload": "rising_drop_levels5-8", "steps": args.steps,
            "warmup": args.warmup, "remesh_every": args.amr_every,
            "ms_per_step": round(statistics.mean(step_ms), 2),
            "ms_per_remesh": round(statistics.mean(remesh_ms), 1) if remesh_ms else None,
            "leaves": leaves, "phi_mass_change_per_remesh": remesh_dmass,
            "phi_mass_change_per_step_max": max(abs(x) for x in step_dmass)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-budget", type=float, default=60.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the all-FP64 Jacobi-PCG step (about 30 s on the headline mesh)")
    ap.add_argument("--no-fp64-mg", action="store_true",
                    help="skip the all-FP64 step with the multigrid preconditioners")
    ap.add_argument("--no-drop", action="store_true", help="skip the rising-drop workload")
    ap.add_argument("--drop-steps", type=int, default=5)
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the roofline kernel from an ncu capture")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-preconditioner measurement (8-drop workload)")
    ap.add_argument("--learned-steps", type=int, default=3,
                    help="time steps whose pressure-Poisson solves give the training pairs")
    ap.add_argument("--learned-iters", type=int, default=6000, help="training iterations")
    ap.add_argument("--learned-capacity", type=int, default=4096,
                    help="replay buffer of the learned mode, in pairs (7.3 MB each on the 8 drops)")
    ap.add_argument("--learned-collect-max", type=int, default=24,
                    help="training pairs taken from one pressure solve at most")
    ap.add_argument("--learned-dt", type=float, default=None,
                    help="time step of the learned mode's workload (default: its own, 5e-4)")
    ap.add_argument("--learned-collect-every", type=int, default=8,
                    help="iterate stride of the training pairs within one pressure solve")
    ap.add_argument("--learned-lr", type=float, default=3e-4)
    ap.add_argument("--learned-grid", type=int, default=64, help="grid size D of the network")
    ap.add_argument("--apply-op", choices=["poisson", "mass", "ch", "momentum"], default="poisson")
    ap.add_argument("--apply-prec", choices=["fp32", "fp64", "fp64df"], default="fp32")
    ap.add_argument("--breakup-levels", default="6,9",
                    help="octree levels lmin,lmax of the many-drop breakup workload")
    ap.add_argument("--amr-every", type=int, default=2, help="steps between remeshes (amr mode)")
    ap.add_argument("--mode", choices=["bench", "apply", "pp", "step", "learned", "breakup",
                                       "amr", "learned_fcg"],
                    default="bench",
                    help="apply / pp: time only one apply / the pressure solve (profiling); "
                         "learned: only the learned-preconditioner part; breakup: the many-drop "
                         "breakup workload under shear; amr: rising drop with remeshing")
    args = ap.parse_args()
    if args.mode == "apply":
        run_apply_only(args)
    elif args.mode == "pp":
        run_pp_only(args)
    elif args.mode == "step":
        run_step_only(args)
    elif args.mode == "learned":
        print(json.dumps(run_learned(args)))
    elif args.mode == "breakup":
        print(json.dumps(run_breakup(args)))
    elif args.mode == "amr":
        print(json.dumps(run_amr(args)))
    elif args.mode == "learned_fcg":
        print(json.dumps(run_learned_fcg(args)))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
