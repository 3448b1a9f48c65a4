"""Benchmark of the DG advection hot path on the 6D workload.

One step = one fused LSRK(5,4) stage on the 6D, degree-3 problem
(8^3 x 8^3 cells, 1,073,741,824 DoFs): the operator application M^{-1} A(w)
(FP32 sweeps and fluxes on the FP32 stage vector w) fused with the FP64
state update u += b_s dt K and the next stage vector.  The metric is DoFs
per second (GDoF/s) of such operator applications; the line also reports
the stand-alone operator applications in FP32, FP32-with-FP64-vectors and
FP64, each against the HBM roofline.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica of the whole
workload (the method needs no exchange between independent problems;
"replicas only"), and the value is the total over ranks / max time.
"""
import argparse
import hashlib
import re
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "6D DG advection GDoF/s per operator apply (FP32 vs FP64), % of HBM roofline"
UNIT = "GDoF/s"
# algorithmic bytes per DoF (each vector element read or written once)
BYTES_PER_DOF = {
    "stage_fp32w_fp64u": 4 + 8 + 8 + 4,   # read w_in, read+write u, write w_out
    "stage_fp64": 8 + 8 + 8 + 8,
    "apply_fp32": 4 + 4,
    "apply_fp32_fp64io": 8 + 8,
    "apply_fp64": 8 + 8,
}
# FP32 peak of the non-tensor pipes from the unit counts and the maximum SM
# clock: 152 SMs x 128 FP32 lanes x 2 FLOP per fused multiply-add x 2.070 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def flop_entry(dofs, ms, d, n, stage):
    """FP32 arithmetic of one launch of an FP32-sweep kernel against the FP32
    peak.  Per DoF and direction the folded line operator takes 2n + 5 FLOP
    (the neighbour's trace 2, the matrix row 2n, the lift 1 and the speed 2);
    the stage update adds 3 (the FP64 add of the state is not counted)."""
    per_dof = d * (2 * n + 5) + (3 if stage else 0)
    tflops = per_dof * dofs / (ms * 1e-3) / 1e12
    return {"per_dof": per_dof, "achieved_tflops": tflops, "fp32_peak_tflops": FP32_PEAK_TFLOPS,
            "frac": tflops / FP32_PEAK_TFLOPS,
            "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}

KERNEL_SOURCES = ["dg_cell6d.cu", "dg_generic.cuh", "dg_internal.h", "dg_tma.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cells", type=int, default=8, help="cells per direction (default 8)")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--basis", choices=["gl", "gll", "gll_gauss"], default="gl",
                    help="element of the timed step: Gauss-Legendre collocation (default), "
                         "Gauss-Lobatto collocation, or Lobatto nodes with Gauss quadrature")
    ap.add_argument("--kernel-variant", type=int, default=None,
                    help="6D cell kernel for the FP32-sweep paths (1: 64 threads per cell, "
                         "2: 128 threads per cell); default: the library's choice")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-reps", type=int, default=2)
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 2D, 4D, batched and adjoint configurations")
    ap.add_argument("--configs", default=None,
                    help="comma-separated subset of the other configurations (6d_fp32_vs_fp64, "
                         "6d_gll, 6d_curved, 2d, 4d, 4d_k5, batched, adjoint); default: all")
    ap.add_argument("--step-kind", default="stage",
                    choices=["stage", "apply_fp32", "apply_fp32_fp64io", "apply_fp64"],
                    help="what one timed step is (default: the fused LSRK stage)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_hash():
    """Hash of the stage kernel's sources with comments and whitespace runs
    removed (a comment edit does not change the kernel the recorded DRAM
    bytes were taken on)."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        p = os.path.join(ROOT, "paper_2002_08110_gb300", "csrc", f)
        if os.path.exists(p):
            text = open(p, encoding="utf-8").read()
            text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
            text = re.sub(r"//[^\n]*", " ", text)
            h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(workload)
    if not e or e.get("kernel_hash") != kernel_hash():
        return None
    return e.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.file.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def reduce_max(x, world):
    """Max over ranks (identity for one rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# the CPU oracle (cpu_baseline and the reference arm): the sum-factorised FP64
# OpenMP evaluation of oracle/cpu_sumfac.cpp on all host cores
# ---------------------------------------------------------------------------
def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def _mem_available_gb():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) / 1e6
    except Exception:
        pass
    return 0.0


def _sumfac_worker(cells_per_dim, reps, slabs, q):
    """One fused LSRK stage (FP64) of the 6D workload per repetition, on the
    v3 slabs [0, slabs) of the mesh (slabs = all: the whole mesh)."""
    import numpy as np
    import workloads as W
    from oracle import lsrk
    from oracle.sumfac import SumFac, threads
    w = W.config_6d(cells=cells_per_dim)
    zeta = np.polynomial.legendre.leggauss(w.n)[0]
    sf = SumFac(w.dx, w.dv, w.k, w.cells_x, w.cells_v, w.x_lo, w.x_hi, w.v_lo, w.v_hi,
                e_nodes=W.e_table(w, zeta))
    u = W.separable_state(w, zeta)
    w_in = u.copy()
    w_out = np.empty_like(u)
    dt, _ = W.time_step(w)
    per_slab = sf.ncells // w.cells_v[-1]
    cells = (0, per_slab * slabs)
    times = []
    for r in range(reps):
        t0 = time.perf_counter()
        sf.rk_stage(w_in, w_out, u, lsrk.A[0] * dt, lsrk.B[0] * dt, cells=cells)
        times.append(time.perf_counter() - t0)
    q.put({"seconds": times, "dofs": (cells[1] - cells[0]) * w.n ** w.d, "threads": threads(),
           "total_dofs": sf.n_dofs, "slabs": slabs, "of_slabs": w.cells_v[-1]})


def cpu_oracle(cells_per_dim, reps, slabs=None):
    """Times the CPU oracle in a fresh (spawned) process: ``reps`` fused
    stages on ``slabs`` v3 slabs of the 6D mesh (None: all of them)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    qu = ctx.Queue()
    pr = ctx.Process(target=_sumfac_worker, args=(cells_per_dim, reps, slabs or cells_per_dim, qu))
    pr.start()
    res = qu.get()
    pr.join()
    res["cpu"] = _cpu_model()
    return res


def _cpu_line(res, value):
    whole = res["slabs"] == res["of_slabs"]
    return {"value": value, "unit": UNIT, "cores": res["threads"], "kind": "oracle",
            "implementation": "oracle/cpu_sumfac.cpp: FP64 sum factorisation, OpenMP over cells",
            "cpu": res["cpu"],
            "sample": ("the whole 6D mesh, one fused FP64 LSRK stage per step" if whole else
                       f"{res['slabs']} of {res['of_slabs']} v3 slabs of the 6D mesh "
                       f"({res['dofs']} of {res['total_dofs']} DoFs) per step, one fused FP64 "
                       "LSRK stage")}


def reference_arm(args, world, rank):
    """--impl reference: the CPU oracle, as it stands, on all host cores."""
    if rank != 0:
        return
    need = 3 * 8 * (args.cells ** 6) * 64 / 1e9 + 10
    if _mem_available_gb() < need:
        print(json.dumps({"impl": "reference", "unavailable":
                          f"the CPU oracle needs about {need:.0f} GB of host memory"}), flush=True)
        return
    # one v3 slab per step keeps warm-up + steps within a few minutes
    res = cpu_oracle(args.cells, args.warmup + args.steps, slabs=1)
    ts = res["seconds"][args.warmup:]
    total = sum(ts)
    value = res["dofs"] * len(ts) / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(ts),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"6d_k3_{args.cells}^6", "step": "fused LSRK(5,4) stage, FP64",
                   "sample": f"{res['slabs']} of {res['of_slabs']} v3 slabs per step"},
        "cpu_baseline": _cpu_line(res, value),
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the other workloads (2D, 4D, batched, adjoint)
# ---------------------------------------------------------------------------
def _timed(torch, fn, reps):
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def measure_configs(torch, hbm_peak, only=None):
    """Throughput of the other synthetic workloads, GDoF/s per LSRK stage
    (each stage = one operator application fused with the state update)."""
    import workloads as W
    from paper_2002_08110_gb300 import DG, DGBatch, PREC_FP32, PREC_FP64, reference_nodes
    from paper_2002_08110_gb300.autograd import misfit_gradient
    out = {}

    def want(name):
        return only is None or name in only

    def make(w):
        zeta, _ = reference_nodes(w.k)
        return DG(e_nodes=W.e_table(w, zeta), **W.dg_kwargs(w)), zeta

    def stage_entry(dg, ms_step, prec):
        bpd = 32 if prec == PREC_FP64 else 24
        st = ms_step / 5
        gbs = bpd * dg.n_dofs / (st * 1e-3) / 1e9
        return {"ms_per_step": ms_step, "GDoF/s_per_stage": dg.n_dofs / (st * 1e-3) / 1e9,
                "frac_hbm": gbs / hbm_peak, "bytes_per_dof": bpd}

    # 6D: FP32 sweeps / FP64 state against the plain FP64 path on the same
    # GPU -- error per operator application and at the workload's final time
    # (its 50 steps); the temporal error of the run, estimated from a second
    # run at half the step (Richardson: (16/15) ||u_dt - u_dt/2|| for a
    # fourth-order scheme), says what "the same final-time accuracy" means
    if want("6d_fp32_vs_fp64"):
        w = W.config_6d()
        dg, zeta = make(w)
        dt, nacc = W.time_step(w)
        u0 = W.separable_state(w, zeta, xp=torch, device="cuda")
        k64 = dg.apply(u0, prec=PREC_FP64)
        k32 = dg.apply(u0.float(), prec=PREC_FP32).double()
        rel_apply = float(torch.linalg.vector_norm(k32 - k64) / torch.linalg.vector_norm(k64))
        del k32
        u64 = u0.clone()
        ms64 = _timed(torch, lambda: dg.rk_step(u64, dt, nsteps=nacc, prec=PREC_FP64), 1)
        u32 = u0.clone()
        ms32 = _timed(torch, lambda: dg.rk_step(u32, dt, nsteps=nacc, prec=PREC_FP32), 1)
        u32h = u0.clone()
        dg.rk_step(u32h, dt / 2, nsteps=2 * nacc, prec=PREC_FP32)
        dg.check()
        nrm = lambda x: float(torch.linalg.vector_norm(x))
        n64 = nrm(u64)
        time_err = 16.0 / 15.0 * nrm(u32 - u32h) / n64
        del u32h
        # delta-f form around the Maxwellian equilibrium: FP32 sweeps on u - u_eq
        u_eq = W.separable_state(W.equilibrium_6d(w), zeta, xp=torch, device="cuda")
        dg.set_reference(u_eq)
        kdf = dg.apply_df(u0)
        rel_apply_df = float(torch.linalg.vector_norm(kdf - k64) / torch.linalg.vector_norm(k64))
        del kdf, u_eq
        udf = u0.clone()
        dg.rk_step_df(udf, dt, nsteps=1)
        udf.copy_(u0)
        msdf = _timed(torch, lambda: dg.rk_step_df(udf, dt, nsteps=nacc), 1)
        dg.check()
        m0, l0, _ = dg.integrals(u0)

        def drift(x):
            m, l2, _ = dg.integrals(x)
            return {"mass_drift": (m - m0) / m0, "l2_change": (l2 - l0) / l0}
        out["6d_fp32_vs_fp64"] = {
            "workload": w.name, "steps": nacc, "final_time": dt * nacc,
            "apply_rel_l2_diff_fp32": rel_apply, "apply_rel_l2_diff_deltaf": rel_apply_df,
            "state_change_rel_l2": nrm(u64 - u0) / nrm(u0),
            "temporal_error_estimate_rel_l2": time_err,
            "fp64": {"ms_per_step": ms64 / nacc, **drift(u64)},
            "fp32_sweeps_fp64_state": {"ms_per_step": ms32 / nacc, **drift(u32),
                                       "state_rel_l2_diff_vs_fp64": nrm(u32 - u64) / n64},
            "deltaf_fp32_sweeps": {"ms_per_step": msdf / nacc, **drift(udf),
                                   "state_rel_l2_diff_vs_fp64": nrm(udf - u64) / n64},
            "note": "K of the FP64 path matches the FP64 oracle to 1e-12 (tests); the plain relative "
                    "difference of K is large for smooth data (K << its terms); see tests for the "
                    "term-scale error.  The final-time differences against FP64 are to be read "
                    "against the temporal error estimate of the run"}
        dg.close()
        del u0, u64, u32, k64, udf
        torch.cuda.empty_cache()

    # 6D in the Gauss-Lobatto bases: the collocation variant (FP32 stage; its
    # v neighbours arrive as face layers) and the paper's Lobatto-node,
    # Gauss-quadrature element (steps between two changes of basis)
    if want("6d_gll"):
        from paper_2002_08110_gb300 import BASIS_GLL, BASIS_GLL_GAUSS, basis_nodes
        w = W.config_6d()
        dt, _ = W.time_step(w)
        for name, basis in (("6d_gll_collocation", BASIS_GLL), ("6d_gll_gauss", BASIS_GLL_GAUSS)):
            nodes, qpts, _ = basis_nodes(basis, w.k)
            dg = DG(e_nodes=W.e_table(w, qpts), basis=basis, **W.dg_kwargs(w))
            u = W.separable_state(w, nodes, xp=torch, device="cuda")
            if basis == BASIS_GLL:
                a, b = u.float(), torch.empty(dg.n_dofs, dtype=torch.float32, device="cuda")
                for i in range(3):
                    dg.rk_stage(a, b, u, i, dt, prec=PREC_FP32)
                    a, b = b, a
                reps = 20
                ms = _timed(torch, lambda: dg.rk_stage(a, b, u, 1, dt, prec=PREC_FP32), reps)
                dg.check()
                gbs = 24 * dg.n_dofs / (ms * 1e-3) / 1e9
                out[name] = {"workload": w.name + "_gll_collocation", "dofs": dg.n_dofs,
                             "ms_per_stage": ms, "GDoF/s_per_stage": dg.n_dofs / (ms * 1e-3) / 1e9,
                             "frac_hbm": gbs / hbm_peak, "bytes_per_dof": 24,
                             "uniform_sides": int(dg.info.uniform_sides)}
                del a, b
            else:
                nst = 5
                dg.rk_step(u, dt, nsteps=1, prec=PREC_FP32)
                ms = _timed(torch, lambda: dg.rk_step(u, dt, nsteps=nst, prec=PREC_FP32), 1)
                dg.check()
                out[name] = {"workload": w.name + "_gll_gauss", "dofs": dg.n_dofs, "steps_per_call": nst,
                             "ms_per_step": ms / nst,
                             "GDoF/s_per_stage": dg.n_dofs / (ms / nst / 5 * 1e-3) / 1e9,
                             "note": "each call changes the FP64 state to the Gauss points and back "
                                     "around its steps (two tensor-product passes)"}
            dg.close()
            del u
            torch.cuda.empty_cache()

    # 6D on a curved x-mesh (a Jacobian per quadrature point, deformation
    # 0.1 in every x direction): FP32 stage in the generic kernel
    if want("6d_curved"):
        w = W.config_6d()
        dt, _ = W.time_step(w)
        zeta, _ = reference_nodes(w.k)
        dg = DG(e_nodes=W.e_table(w, zeta), deform=(0.1, 0.1, 0.1), **W.dg_kwargs(w))
        u = W.separable_state(w, zeta, xp=torch, device="cuda")
        a, b = u.float(), torch.empty(dg.n_dofs, dtype=torch.float32, device="cuda")
        dg.rk_stage(a, b, u, 0, dt, prec=PREC_FP32)
        ms = _timed(torch, lambda: dg.rk_stage(a, b, u, 1, dt, prec=PREC_FP32), 5)
        dg.check()
        out["6d_curved"] = {"workload": w.name + "_curved0.1", "dofs": dg.n_dofs, "ms_per_stage": ms,
                            "GDoF/s_per_stage": dg.n_dofs / (ms * 1e-3) / 1e9,
                            "frac_hbm": 24 * dg.n_dofs / (ms * 1e-3) / 1e9 / hbm_peak,
                            "kernel": "generic (the specialised 6D kernels are affine-only)"}
        dg.close()
        del u, a, b
        torch.cuda.empty_cache()

    # 2D: one period (T = 2, 240 steps), FP64
    if want("2d"):
        w = W.config_2d()
        dg, zeta = make(w)
        dt, steps = W.time_step(w)
        u = W.separable_state(w, zeta, xp=torch, device="cuda")
        ms = _timed(torch, lambda: dg.rk_step(u, dt, nsteps=steps, prec=PREC_FP64), 1)
        dg.check()
        out["2d"] = {"workload": w.name, "dofs": dg.n_dofs, "steps": steps,
                     **stage_entry(dg, ms / steps, PREC_FP64)}
        dg.close()

    # 4D sheared phase space: 200 steps, FP64 and FP32 sweeps / FP64 state
    if want("4d"):
        w = W.config_4d()
        dg, zeta = make(w)
        dt, steps = W.time_step(w)
        u0 = torch.tensor(W.initial_state(w, zeta), device="cuda")
        for prec, name in ((PREC_FP64, "4d_fp64"), (PREC_FP32, "4d_fp32_fp64state")):
            u = u0.clone()
            dg.rk_step(u, dt, nsteps=1, prec=prec)
            ms = _timed(torch, lambda: dg.rk_step(u, dt, nsteps=steps, prec=prec), 1)
            dg.check()
            out[name] = {"workload": w.name, "dofs": dg.n_dofs, "steps": steps,
                         **stage_entry(dg, ms / steps, prec)}
        dg.close()
        del u0, u

    # 4D sheared phase space at degree 5 (n = 6 points per direction): 200
    # FP32-sweep steps with the FP64 state
    if want("4d_k5"):
        w = W.config_4d(k=5)
        dg, zeta = make(w)
        dt, steps = W.time_step(w)
        u = torch.tensor(W.initial_state(w, zeta), device="cuda")
        dg.rk_step(u, dt, nsteps=1, prec=PREC_FP32)
        ms = _timed(torch, lambda: dg.rk_step(u, dt, nsteps=steps, prec=PREC_FP32), 1)
        dg.check()
        out["4d_k5_fp32_fp64state"] = {"workload": w.name, "dofs": dg.n_dofs, "steps": steps,
                                       **stage_entry(dg, ms / steps, PREC_FP32)}
        dg.close()
        del u

    # batched: 64 instances, one persistent launch per stage, autotuned
    if want("batched"):
        ws = W.batched_instances()
        dgs = [DG(**W.dg_kwargs(w)) for w in ws]
        batch = DGBatch(dgs)
        us = [W.separable_state(w, reference_nodes(w.k)[0], xp=torch, device="cuda") for w in ws]
        w0s = [torch.empty(w.n_dofs, device="cuda", dtype=torch.float32) for w in ws]
        w1s = [torch.empty(w.n_dofs, device="cuda", dtype=torch.float32) for w in ws]
        dts = [W.time_step(w)[0] for w in ws]
        best = batch.autotune(us, w0s, w1s, dts, prec=PREC_FP32)
        # one untimed step: the kept configuration's graphs are captured anew
        batch.rk_step(us, w0s, w1s, dts, nsteps=1, prec=PREC_FP32)
        # four steps in one call (a call converts the FP64 states to the FP32
        # stage vectors once, whatever its number of steps)
        reps = 4
        ms = _timed(torch, lambda: batch.rk_step(us, w0s, w1s, dts, nsteps=reps, prec=PREC_FP32), 1) / reps
        batch.check()
        st = ms / 5
        out["batched"] = {"workload": "64 instances, d in {3,4}, k in {2..5}, 8..24 cells/dir",
                          "dofs": batch.n_dofs, "tiles": batch.tiles, "ms_per_step": ms,
                          "GDoF/s_per_stage": batch.n_dofs / (st * 1e-3) / 1e9,
                          "frac_hbm": 24 * batch.n_dofs / (st * 1e-3) / 1e9 / hbm_peak,
                          "autotuned_ms_per_step": best}
        batch.close()
        for dg in dgs:
            dg.close()
        del us, w0s, w1s

    # adjoint: gradient of the final-time misfit over 200 steps, checkpoints every 20
    if want("adjoint"):
        w = W.config_adjoint()
        dg, zeta = make(w)
        dt, steps = W.time_step(w)
        u0 = torch.tensor(W.separable_state(w, zeta), device="cuda")
        tgt = u0 + torch.tensor(W.noise(w), device="cuda")
        dg.rk_step(tgt, dt, nsteps=steps, prec=PREC_FP32)
        every = w.extra["checkpoint_every"]
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # one untimed pass: graph captures and the checkpoints' memory
        misfit_gradient(u0, tgt, dg, dt, steps, prec=PREC_FP32, checkpoint_every=every)
        torch.cuda.synchronize()
        e0.record(stream)
        J, g = misfit_gradient(u0, tgt, dg, dt, steps, prec=PREC_FP32, checkpoint_every=every)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        # forward (200) + recomputation (200) + adjoint (200) steps
        out["adjoint"] = {"workload": w.name, "dofs": dg.n_dofs, "steps": steps,
                          "checkpoint_every": every, "ms_total": ms, "misfit": J,
                          "grad_norm": float(torch.linalg.vector_norm(g)),
                          "GDoF/s_per_stage": 3 * steps * 5 * dg.n_dofs / (ms * 1e-3) / 1e9}
        dg.close()

    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        reference_arm(args, world, rank)
        return
    import numpy as np
    import torch
    import workloads as W
    from paper_2002_08110_gb300 import DG, PREC_FP32, PREC_FP64, PREC_MIXED, reference_nodes

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = W.config_6d(cells=args.cells)
    from paper_2002_08110_gb300 import basis_nodes
    basis = {"gl": 0, "gll": 1, "gll_gauss": 2}[args.basis]
    zeta, qpts, _ = basis_nodes(basis, w.k)     # DoF nodes, quadrature points
    E = W.e_table(w, qpts)
    dg = DG(e_nodes=E, basis=basis, **W.dg_kwargs(w))
    if args.kernel_variant is not None:
        for prec in (PREC_FP32, PREC_MIXED):
            c = dg.get_launch(prec)
            dg.set_launch(prec, c["threads"], c["cells_per_block"], c["order"], args.kernel_variant)
    n = dg.n_dofs
    dt, _ = W.time_step(w)
    u0 = W.separable_state(w, zeta, xp=torch, device=dev)
    u = u0.clone()
    w0 = u0.float()
    w1 = torch.empty_like(w0)
    hbm_peak, peak_kind = peaks()

    # ---- the timed step: one fused LSRK stage (FP32 sweeps, FP32 w, FP64 u)
    kind = args.step_kind
    if kind == "apply_fp64" or kind == "apply_fp32_fp64io":
        d64 = torch.empty_like(u)

    def stage(i):
        if kind == "stage":
            a, b = (w0, w1) if i % 2 == 0 else (w1, w0)
            dg.rk_stage(a, b, u, i % 5, dt, prec=PREC_FP32)
        elif kind == "apply_fp32":
            dg.apply(w0, w1, prec=PREC_FP32)
        elif kind == "apply_fp32_fp64io":
            dg.apply(u, d64, prec=PREC_MIXED)
        else:
            dg.apply(u, d64, prec=PREC_FP64)

    for i in range(args.warmup):
        stage(i)
    dg.check()
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    torch.cuda.synchronize()
    barrier(world)
    ev[0].record(stream)
    for i in range(args.steps):
        stage(args.warmup + i)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    dg.check()
    per_launch = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    total_ms = reduce_max(total_ms, world)
    barrier(world)
    value = world * n * args.steps / (total_ms * 1e-3) / 1e9
    avg_launch = sum(per_launch) / len(per_launch)
    bpd = BYTES_PER_DOF["stage_fp32w_fp64u" if kind == "stage" else kind]
    achieved = bpd * n / (avg_launch * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "traffic": recorded_traffic(kind if args.basis == "gl" else f"{kind}_{args.basis}"),
            "peak_kind": peak_kind, "bytes_per_dof": bpd,
            "kernel": "fused LSRK stage (cell kernel, stage mode)" if kind == "stage" else "cell kernel, operator application"}
    # the FP32 arithmetic next to the bytes (the FP64 apply runs on the FP64 pipe)
    roof["flops"] = (flop_entry(n, avg_launch, w.dx + w.dv, w.k + 1, kind == "stage")
                     if kind != "apply_fp64" else None)

    # ---- stand-alone operator applications
    variants = {}
    if not args.no_variants:
        def time_fn(fn, reps, warm=1):
            for _ in range(warm):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        src32 = w0
        dst32 = torch.empty_like(src32)
        ms = time_fn(lambda: dg.apply(src32, dst32, prec=PREC_FP32), 10)
        variants["apply_fp32"] = ms
        src64 = u
        dst64 = torch.empty_like(u)
        ms = time_fn(lambda: dg.apply(src64, dst64, prec=PREC_MIXED), 10)
        variants["apply_fp32_fp64io"] = ms
        ms = time_fn(lambda: dg.apply(src64, dst64, prec=PREC_FP64), args.fp64_reps, warm=1)
        variants["apply_fp64"] = ms
        del dst32
        dg.check()
        for k in list(variants):
            ms = variants[k]
            gbs = BYTES_PER_DOF[k] * n / (ms * 1e-3) / 1e9
            variants[k] = {"ms": ms, "GDoF/s": n / (ms * 1e-3) / 1e9, "GB/s": gbs,
                           "frac_hbm": gbs / hbm_peak}
        del dst64

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        steps_e2e = 3
        h_w = torch.empty(n, dtype=torch.float32, pin_memory=True)
        h_u = torch.empty(n, dtype=torch.float64, pin_memory=True)
        h_w.copy_(w0)
        h_u.copy_(u)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h_w2 = torch.empty(n, dtype=torch.float32, pin_memory=True)
        # untimed first call: the library allocates its device staging once
        dg.rk_stage_host(h_w, h_w2, h_u, 0, 0.0, prec=PREC_FP32)
        h_u.copy_(u)
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(steps_e2e):
            # the public host-buffer call: copies in, fused stage, copies out
            src, dst = (h_w, h_w2) if i % 2 == 0 else (h_w2, h_w)
            dg.rk_stage_host(src, dst, h_u, i % 5, dt, prec=PREC_FP32)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps_e2e
        ms = reduce_max(ms, world)
        e2e = {"value": world * n / (ms * 1e-3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": n * (4 + 8), "d2h_bytes_per_step": n * (8 + 4),
               "ms_per_step": ms}
        del h_w, h_w2, h_u

    others = None
    if not args.no_configs:
        del u0, u, w0, w1
        torch.cuda.empty_cache()
        others = measure_configs(torch, hbm_peak,
                                 None if args.configs is None else set(args.configs.split(",")))

    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        # the whole mesh if the host has the memory (3 FP64 vectors), else one v3 slab
        whole = _mem_available_gb() >= 3 * 8 * n / 1e9 + 10
        res = cpu_oracle(args.cells, 1, slabs=None if whole else 1)
        sec = min(res["seconds"])
        cpu = _cpu_line(res, res["dofs"] / sec / 1e9)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": w.name if args.basis == "gl" else f"{w.name}_{args.basis}",
                       "basis": args.basis, "dofs": n, "cells": w.ncells, "degree": w.k,
                       "step": "fused LSRK(5,4) stage: FP32 sweeps, FP32 stage vector, FP64 state",
                       "l2": "inputs larger than L2 (vectors 4.3-8.6 GB)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "step_kind": kind,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps,
            "clocks": clk,
            "variants": variants,
            "configs": others,
            "launch": dg.get_launch(PREC_FP32),
        }
        print(json.dumps(line), flush=True)
    dg.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
