"""Benchmark of the two-stage block orthogonalization of s-step GMRES on GB300.

Workload (one step): the standalone block-orthogonalization pass of an
n x 61 FP64 basis, n = 4,194,304 (the 2048 x 2048 2D Laplace grid size):
column 0 plus 12 s-step blocks of s = 5 columns through stage 1 (one BCGS-PIP
each, against all accumulated columns), then stage 2 (BCGS-PIP = CholQR) on
the whole 61-column big panel (s^ = m = 60).  Each step re-orthogonalizes the
previous step's output, so every step does identical work on a 2 GB basis
(16x the 129 MB L2: no step reads another's data from L2).

value  = algorithmic HBM bytes of the step (8376 B per row)
         / device time of the step  [GB/s], inputs resident in HBM;
e2e    = the same bytes / time with the basis copied in from pinned host
         memory and Q, R copied back, every step;
roofline = the dominant kernel of the step, timed per launch with CUDA events
         inside the timed region.

The JSON line also reports the FP64 s-step GMRES solver on the same grid (one
timed restart cycle of m = 60) and the time to solution of the 64 x 64 case.

``--impl reference`` times the CPU oracle (numpy FP64) on a bounded row sample
of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_ROWS = 2048 * 2048
S = 5
NBLK = 12
NCOL = 1 + S * NBLK
K_BLOCKS = [1 + S * j for j in range(NBLK)]
BYTES_PER_ROW = (8 * sum(k + S for k in K_BLOCKS) + 8 * sum(k + 2 * S for k in K_BLOCKS)
                 + 8 * NCOL + 16 * NCOL)
METRIC = "time-to-solution @relres 1e-8 & ortho HBM GB/s vs plain FP64; solves/s, p99 lat"
WORKLOAD = (f"two-stage block orthogonalization of an n x {NCOL} FP64 basis, n={N_ROWS} (2048^2 grid): "
            f"q_1 + {NBLK} blocks of s={S} through stage 1 (BCGS-PIP), stage 2 (CholQR) on the {NCOL}-column big panel")


def flops_gram(n, k, nb):
    return 2.0 * n * (k * nb + nb * (nb + 1) / 2)


def flops_update(n, k, nb):
    return 2.0 * n * k * nb + 1.0 * n * nb * nb


def bytes_gram(n, k, nb):
    return 8.0 * n * (k + nb)


def bytes_update(n, k, nb):
    return 8.0 * n * (k + 2 * nb)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- reference arm / CPU baseline
def oracle_step(X):
    """One step of the workload on the CPU oracle (in place on X, n_s x 61)."""
    from oracle import blockortho as bo
    import numpy as np
    n = X.shape[0]
    for k in K_BLOCKS:
        Qh, P, T = bo.stage1(X[:, :k], X[:, k:k + S])
        X[:, k:k + S] = Qh
    Q, _, _ = bo.stage2(np.zeros((n, 0)), X)
    X[:, :] = Q


def cpu_oracle_rate(rows, steps, warmup=0):
    import numpy as np
    import synth
    X = np.asfortranarray(synth.tall_basis(rows, NCOL, seed=1))
    X[:, 0] /= np.linalg.norm(X[:, 0])
    for _ in range(warmup):
        oracle_step(X)
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle_step(X)
    dt = time.perf_counter() - t0
    return BYTES_PER_ROW * rows * steps / dt / 1e9, dt


def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    rows = args.ref_rows
    val, dt = cpu_oracle_rate(rows, args.steps, warmup=min(args.warmup, 1))
    cores = cpu_threads()
    line = {"impl": "reference", "metric": METRIC, "value": round(val, 3), "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * dt / args.steps, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_rows": rows, "parallelism": "replicas"},
            "cpu_baseline": {"value": round(val, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "sample": f"{rows} of {N_ROWS} rows per step (numpy FP64 oracle, BLAS threads = cores)"},
            "e2e": {"value": round(val, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU arm
def run_ours(args):
    import numpy as np
    import torch
    import synth
    from paper_2402_15033_gb300 import build as _build, capi

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    _build.build()
    capi.load()
    dev = torch.device("cuda", local)
    n = args.rows

    # basis: 61 columns, ld = n (n is a multiple of 32)
    host = synth.tall_basis(n, NCOL, seed=1 + rank)
    basis = torch.empty(NCOL, n, dtype=torch.float64, device=dev)
    basis.copy_(torch.from_numpy(host.T.copy()))
    B = basis.T
    B[:, 0] /= torch.linalg.norm(B[:, 0])
    Rh = torch.zeros(NCOL, NCOL, dtype=torch.float64, device=dev).T
    R2 = torch.zeros(NCOL, NCOL, dtype=torch.float64, device=dev).T
    work = torch.empty(capi.workspace_bytes(n, NCOL, NCOL), dtype=torch.uint8, device=dev)
    st = torch.zeros(NBLK + 1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream

    kinds = {"stage1_gram": [], "stage1_update": [], "stage2_gram": [], "stage2_update": []}

    def step(evs=None):
        for j, k in enumerate(K_BLOCKS):
            Q = B[:, :k]
            V = B[:, k:k + S]
            Rb = Rh[:k + S, k:k + S]
            if evs is not None:
                e0 = torch.cuda.Event(enable_timing=True); e0.record()
            capi.ortho_gram_chol(Q, V, Rb, work, st[j:j + 1], k=k, stream=stream)
            if evs is not None:
                e1 = torch.cuda.Event(enable_timing=True); e1.record()
            capi.ortho_update(Q, V, Rb, st[j:j + 1], k=k, stream=stream)
            if evs is not None:
                e2 = torch.cuda.Event(enable_timing=True); e2.record()
                evs.append(("stage1_gram", k, S, e0, e1))
                evs.append(("stage1_update", k, S, e1, e2))
        if evs is not None:
            e0 = torch.cuda.Event(enable_timing=True); e0.record()
        capi.ortho_gram_chol(None, B, R2, work, st[NBLK:], k=0, stream=stream)
        if evs is not None:
            e1 = torch.cuda.Event(enable_timing=True); e1.record()
        capi.ortho_update(None, B, R2, st[NBLK:], k=0, stream=stream)
        if evs is not None:
            e2 = torch.cuda.Event(enable_timing=True); e2.record()
            evs.append(("stage2_gram", 0, NCOL, e0, e1))
            evs.append(("stage2_update", 0, NCOL, e1, e2))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if int(st.abs().sum().item()) != 0:
        raise RuntimeError("Cholesky breakdown in the benchmark input")

    # ---- timed region (device-resident inputs)
    clocks = ClockSampler()
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    evs = []
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record()
    for _ in range(args.steps):
        step(evs)
    t_end.record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    for kind, k, nb, a, b in evs:
        kinds[kind].append((k, nb, a.elapsed_time(b)))
    ms_per_step = total_ms / args.steps
    bytes_step = BYTES_PER_ROW * n
    value = bytes_step / (ms_per_step * 1e-3) / 1e9 * world

    # per-kernel-family time; the dominant one carries the roofline
    fam = {}
    for kind, lst in kinds.items():
        tot = sum(x[2] for x in lst)
        fl = sum((flops_gram if "gram" in kind else flops_update)(n, k, nb) for k, nb, _ in lst)
        by = sum((bytes_gram if "gram" in kind else bytes_update)(n, k, nb) for k, nb, _ in lst)
        fam[kind] = {"ms_total": tot, "launches": len(lst), "flops": fl, "bytes": by}
    dom = max(fam, key=lambda k: fam[k]["ms_total"])
    d = fam[dom]
    peaks, src = load_peaks()
    fp64_peak_tflops = 152 * 2070e6 * 2 * 2 / 1e12   # see the design doc: 2 FP64 FMA/clk/SM x max clock
    achieved_tflops = d["flops"] / (d["ms_total"] * 1e-3) / 1e12
    achieved_gbs = d["bytes"] / (d["ms_total"] * 1e-3) / 1e9
    roofline = {"bound": "alu", "achieved": round(achieved_tflops, 4), "peak": round(fp64_peak_tflops, 4),
                "unit": "TFLOP/s", "frac": round(achieved_tflops / fp64_peak_tflops, 4),
                "traffic": None, "kernel": dom, "peak_source": "FP64 FMA pipe: 2/clk/SM x 152 SMs x 2070 MHz",
                "hbm": {"achieved_gbs": round(achieved_gbs, 1), "peak_gbs": peaks["hbm_gbs"],
                        "frac": round(achieved_gbs / peaks["hbm_gbs"], 4), "peak_source": src}}
    families = {k: {"ms_per_step": round(v["ms_total"] / args.steps, 4), "launches_per_step": v["launches"] // args.steps,
                    "gbs": round(v["bytes"] / (v["ms_total"] * 1e-3) / 1e9, 1),
                    "tflops": round(v["flops"] / (v["ms_total"] * 1e-3) / 1e12, 4)} for k, v in fam.items()}

    # ---- end to end: pinned host basis in, Q and R out, every step
    e2e = None
    if not args.no_e2e:
        hostin = torch.from_numpy(host.T.copy()).pin_memory()
        hostin[0] /= torch.linalg.norm(hostin[0])
        hostq = torch.empty_like(hostin).pin_memory()
        hostr = torch.empty(NCOL, NCOL, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        ke = max(1, min(args.steps, 3))
        a.record()
        for _ in range(ke):
            basis.copy_(hostin, non_blocking=True)
            step()
            hostq.copy_(basis, non_blocking=True)
            hostr.copy_(R2.T, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        ems = a.elapsed_time(b) / ke
        e2e = {"value": round(bytes_step / (ems * 1e-3) / 1e9 * world, 3), "unit": "GB/s",
               "h2d_bytes_per_step": int(hostin.numel() * 8),
               "d2h_bytes_per_step": int(hostq.numel() * 8 + hostr.numel() * 8),
               "ms_per_step": round(ems, 3)}

    # ---- the FP64 solver on the same grid: one restart cycle, and C1 to convergence
    solve = None
    if not args.no_solve and rank == 0:
        solve = solver_numbers(capi, dev, args)

    # ---- CPU oracle on a bounded sample of the same workload
    cpu = None
    if rank == 0 and not args.no_cpu:
        rows = 2 * args.ref_rows
        val, dt = cpu_oracle_rate(rows, 1)
        cpu = {"value": round(val, 3), "unit": "GB/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"one step on {rows} of {n} rows (numpy FP64 oracle), {dt:.1f} s"}

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "n": n, "cols": NCOL, "s": S, "panel": NCOL - 1,
                           "bytes_per_step": bytes_step, "l2": "basis 2 GB >> 129 MB L2, no flush needed",
                           "parallelism": "replicas" if world > 1 else "single"},
                "roofline": roofline, "kernels": families, "e2e": e2e, "cpu_baseline": cpu,
                "gpu_launches": (2 * NBLK + 2) * args.steps, "clocks": clk, "solver": solve}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def solver_numbers(capi, dev, args):
    import numpy as np
    import torch
    import synth
    from scipy.sparse import csr_matrix
    out = {}
    # C1: 64 x 64 Laplace, tol 1e-8, FP64 two-stage, to convergence (time to solution)
    A = synth.laplace2d(64)
    xt = synth.x_true(A.n, 0)
    b = csr_matrix((A.vals, A.colind, A.rowptr), shape=(A.n, A.n)) @ xt
    S1 = capi.Solver.from_csr(A, capi.default_opts(m=60, s=5, panel=60, tol=1e-8))
    bd = torch.tensor(b, device=dev)
    xd = torch.zeros(A.n, dtype=torch.float64, device=dev)
    S1.solve(bd, xd)
    times = []
    for _ in range(5):
        xd.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, res = S1.solve(bd, xd)
        times.append(time.perf_counter() - t0)
    S1.close()
    out["laplace64_fp64"] = {"time_to_solution_ms": round(1e3 * statistics.median(times), 3), "status": rc,
                             "iters": res["iters"], "relres": res["relres_true"]}
    # 2048 x 2048 Laplace: one restart cycle (60 iterations), per-phase times
    if args.rows == N_ROWS:
        A = synth.laplace2d(2048)
        xt = synth.x_true(A.n, 0)
        b = csr_matrix((A.vals, A.colind, A.rowptr), shape=(A.n, A.n)) @ xt
        opts = capi.default_opts(m=60, s=5, panel=60, tol=1e-14, max_restarts=1, timing=1)
        S2 = capi.Solver.from_csr(A, opts)
        bd = torch.tensor(b, device=dev)
        xd = torch.zeros(A.n, dtype=torch.float64, device=dev)
        S2.solve(bd, xd)
        xd.zero_()
        rc, res = S2.solve(bd, xd)
        S2.close()
        cyc = res["t_total_ms"]
        out["laplace2048_fp64_cycle"] = {"ms_per_restart_cycle": round(cyc, 3), "iters": res["iters"],
                                         "iters_per_s": round(res["iters"] / (cyc * 1e-3), 1),
                                         "t_mpk_ms": round(res["t_mpk_ms"], 3), "t_stage1_ms": round(res["t_stage1_ms"], 3),
                                         "t_stage2_ms": round(res["t_stage2_ms"], 3), "t_ls_ms": round(res["t_ls_ms"], 3),
                                         "relres_after_one_cycle": res["relres_true"], "status": rc}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rows", type=int, default=N_ROWS)
    ap.add_argument("--ref-rows", type=int, default=1 << 20)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
