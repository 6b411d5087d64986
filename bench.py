"""Benchmark of the two-stage block orthogonalization of s-step GMRES on GB300.

Workload (one step): the standalone block-orthogonalization pass of an
n x 61 FP64 basis, n = 4,194,304 (the 2048 x 2048 2D Laplace grid size):
column 0 plus 12 s-step blocks of s = 5 columns through stage 1 (one BCGS-PIP
each, against all accumulated columns), then stage 2 (BCGS-PIP = CholQR) on
the whole 61-column big panel (s^ = m = 60).  Each step re-orthogonalizes the
previous step's output, so every step does identical work on a 2 GB basis
(16x the 129 MB L2: no step reads another's data from L2).

value  = algorithmic HBM bytes of the step (8376 B per row: each stage-1 Gram reads
         its k + s columns once, each update reads k + s and writes s, stage 2
         reads the 61 columns twice and writes them once; 8 bytes per value)
         / device time of the step  [GB/s], inputs resident in HBM.  The
         headline step runs the exact-slice tensor-core arithmetic (FP64 in and
         out, FP64-quality Gram and update); the same step on the FP64 pipe and
         in double-float arithmetic is reported beside it (other_arith);
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


def tc_tile_count(k, nb):
    """16 x 8 output tiles of the tensor-core Gram (those not strictly below the G diagonal)."""
    return sum(1 for mt in range((k + nb + 15) // 16) for nt in range((nb + 7) // 8)
               if not (16 * mt - k > 8 * nt + 7))


def tc_mma_flops(n, k, nb):
    """f16 tensor FLOPs the exact-slice Gram executes: per 64-row chunk, 4
    k-steps x 28 digit-pair MMAs of 16 x 8 x 16 for every M-tile (narrow
    blocks, the streaming kernel) or every output tile not strictly below the
    G diagonal (wide blocks, the mma.sync kernel); for wide blocks whose
    columns are all in the digit basis (the stage-2 panel, as benchmarked) the
    tcgen05 kernel's 4 k-steps x six M = 128 MMAs of N = 1024 columns in all;
    k + nb > 64 runs FP64."""
    if k + nb > 64:
        return 0.0
    if nb >= 9:
        return math.ceil(n / 64) * 4 * 2 * 128 * 1024 * 16
    tiles = (k + nb + 15) // 16 if nb <= 8 else tc_tile_count(k, nb)
    return math.ceil(n / 64) * tiles * 4 * 28 * 2 * 16 * 8 * 16


def tc_update_mma_flops(n, k, nb):
    """f16 tensor FLOPs the exact-slice update executes: per 64-row chunk, 4
    M-tiles per N-tile of 8 columns, every k-step over k + nb (narrow blocks)
    or those up to the last nonzero row of the triangular W (wide blocks), 28
    digit-pair MMAs of 16 x 8 x 16 each."""
    kx = k + nb
    if kx > 64:
        return 0.0
    nks = (kx + 15) // 16
    if nb <= 8:
        steps = nks
    else:
        steps = sum(min(nks, (k + 8 * nt + 7) // 16 + 1) for nt in range((nb + 7) // 8))
    return math.ceil(n / 64) * 4 * steps * 28 * 2 * 16 * 8 * 16


ARITH_TEXT = {"fp64": "FP64 pipe (native FP64 FMA)",
              "tc": "Gram and update on f16 tensor cores by exact 8-bit slicing (FP64 quality); "
                    "resident digit basis of 7 bytes per value: each column sliced once",
              "dd": "double-float (hi+lo FP32), ~2^-48 relative, FP64 in/out"}

DTYPE_TEXT = {"fp64": "f64", "tc": "f64 in/out, products as exact f16 digit slices", "dd": "f32x2 (double-float)"}

FP64_PEAK_TFLOPS = 152 * 2070e6 * 2 * 2 / 1e12   # nominal: 2 FP64 FMA/clk/SM x 152 SMs x max clock (1.26)
FP64_PROBE_TFLOPS = 1.19                          # an FMA-chain probe on this GPU (not a driver measurement)


# DRAM bytes per launch from one ncu capture at n = 1,048,576 (profiles/),
# scaled by 4 to the benchmark's n (traffic grows with n): the last stage-1
# block (k = 56) and the stage-2 panel.  Entries are removed when the kernel
# changes after its capture.
NCU_TRAFFIC = {
    "tc": {"stage1_gram": 4 * (457.3 + 3.4) * 1e6},
    "fp64": {"stage1_gram": 4 * (511.8 + 3.2) * 1e6, "stage2_gram": 4 * (514.7 + 3.5) * 1e6},
}


def roofline_of(d, kernel, arith):
    """Roofline object of one kernel family: FP64-pipe bound for FP64 kernels,
    HBM-bound figure for the tensor-core Gram (its algorithmic bytes over the
    measured copy bandwidth), with the other bound attached."""
    peaks, src = load_peaks()
    t = d["ms_total"] * 1e-3
    gbs = d["bytes"] / t / 1e9
    tfl = d["flops"] / t / 1e12
    hbm = {"achieved_gbs": round(gbs, 1), "peak_gbs": peaks["hbm_gbs"], "frac": round(gbs / peaks["hbm_gbs"], 4),
           "peak_source": src}
    traffic = NCU_TRAFFIC.get(arith, {}).get(kernel)
    tnote = ("ncu DRAM read+write of the k=56 launch (stage 1) or the panel launch (stage 2), "
             "captured at n=1,048,576 and scaled x4") if traffic else None
    if arith == "dd":
        # double-float runs on the FP32 pipe (about 20 FP32 operations per FP64
        # product); its bytes are the FP64 algorithmic bytes, so it is reported
        # against the HBM roof like the tensor-core arithmetic
        return {"bound": "hbm", "achieved": round(gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(gbs / peaks["hbm_gbs"], 4), "traffic": None, "kernel": kernel, "peak_source": src}
    if arith == "tc" and d.get("tensor_flops"):
        tt = d["tensor_flops"] / t / 1e12
        return {"bound": "hbm", "achieved": round(gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(gbs / peaks["hbm_gbs"], 4), "traffic": traffic, "traffic_note": tnote,
                "kernel": kernel, "peak_source": src,
                "tensor": {"executed_tflops": round(tt, 2), "mma_sync_f16_peak_tflops": MMA_SYNC_PEAK,
                           "frac": round(tt / MMA_SYNC_PEAK, 4),
                           "peak_source": "mma.sync m16n8k16 throughput measured on this GPU (bf16; f16 "
                                          "issues at the same rate)"}}
    return {"bound": "alu", "achieved": round(tfl, 4), "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
            "frac": round(tfl / FP64_PEAK_TFLOPS, 4), "traffic": traffic, "traffic_note": tnote, "kernel": kernel,
            "peak_source": "nominal FP64 FMA pipe: 2/clk/SM x 152 SMs x 2070 MHz (no driver measurement of FP64)",
            "frac_of_probe": round(tfl / FP64_PROBE_TFLOPS, 4),
            "probe_tflops": FP64_PROBE_TFLOPS, "hbm": hbm}


MMA_SYNC_PEAK = 604.0


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


def max_over_ranks(x, world, device=None):
    """The slowest rank's x (a time in ms): an all-reduce MAX over the process
    group (NCCL on GPUs, gloo on CPUs); x itself at N = 1."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(bytes_per_rank, ms, world):
    """GB/s of the whole job: each of the world ranks moves bytes_per_rank, all
    within ms (the slowest rank's time)."""
    return bytes_per_rank / (ms * 1e-3) / 1e9 * world


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

    grams = {"fp64": capi.ortho_gram_chol, "dd": capi.ortho_gram_chol_dd, "tc": capi.ortho_gram_chol_tc}
    # digit basis of the tensor-core step: every column is sliced once (column 0
    # by a fill, each block by its update) and read back by the later Grams
    CAPC = 64
    digits = torch.empty(capi.digits_bytes(n, CAPC), dtype=torch.uint8, device=dev)

    def make_step(arith, B=B, Rh=Rh, R2=R2, stream=stream):
        """One step on the basis view B (and its factor blocks Rh, R2), on `stream`."""
        gram = grams[arith]
        dd = arith == "dd"
        tc = arith == "tc"
        tcd = tc and not args.no_digits

        def step(evs=None):
            def mark():
                if evs is None:
                    return None
                e = torch.cuda.Event(enable_timing=True)
                e.record()
                return e
            for j, k in enumerate(K_BLOCKS):
                Q = B[:, :k]
                V = B[:, k:k + S]
                Rb = Rh[:k + S, k:k + S]
                e0 = mark()
                if tcd:
                    if j == 0:
                        capi.digits_fill(B[:, :1], 0, digits, CAPC, stream=stream)
                    capi.ortho_gram_chol_tcd(Q, V, Rb, work, st[j:j + 1], digits, CAPC, k, k=k, stream=stream)
                else:
                    gram(Q, V, Rb, work, st[j:j + 1], k=k, stream=stream)
                e1 = mark()
                if tcd:
                    capi.ortho_update_tcd(Q, V, Rb, st[j:j + 1], digits, CAPC, k=k, stream=stream)
                else:
                    capi.ortho_update(Q, V, Rb, st[j:j + 1], k=k, stream=stream, dd=dd, tc=tc)
                e2 = mark()
                if evs is not None:
                    evs.append(("stage1_gram", k, S, e0, e1))
                    evs.append(("stage1_update", k, S, e1, e2))
            e0 = mark()
            if tcd:
                capi.ortho_gram_chol_tcd(None, B, R2, work, st[NBLK:], digits, CAPC, NCOL, k=0, stream=stream)
            else:
                gram(None, B, R2, work, st[NBLK:], k=0, stream=stream)
            e1 = mark()
            capi.ortho_update(None, B, R2, st[NBLK:], k=0, stream=stream, dd=dd, tc=tc)
            e2 = mark()
            if evs is not None:
                evs.append(("stage2_gram", 0, NCOL, e0, e1))
                evs.append(("stage2_update", 0, NCOL, e1, e2))
        return step

    def families_of(evs, arith, steps):
        kinds = {"stage1_gram": [], "stage1_update": [], "stage2_gram": [], "stage2_update": []}
        for kind, k, nb, a, b in evs:
            kinds[kind].append((k, nb, a.elapsed_time(b)))
        fam = {}
        for kind, lst in kinds.items():
            tot = sum(x[2] for x in lst)
            gram = "gram" in kind
            fl = sum((flops_gram if gram else flops_update)(n, k, nb) for k, nb, _ in lst)
            by = sum((bytes_gram if gram else bytes_update)(n, k, nb) for k, nb, _ in lst)
            tfl = (sum((tc_mma_flops if gram else tc_update_mma_flops)(n, k, nb) for k, nb, _ in lst)
                   if arith == "tc" else 0.0)
            fam[kind] = {"ms_total": tot, "launches": len(lst), "flops": fl, "bytes": by, "tensor_flops": tfl}
        out = {}
        for kk, v in fam.items():
            out[kk] = {"ms_per_step": round(v["ms_total"] / steps, 4), "launches_per_step": v["launches"] // steps,
                       "gbs": round(v["bytes"] / (v["ms_total"] * 1e-3) / 1e9, 1),
                       "tflops": round(v["flops"] / (v["ms_total"] * 1e-3) / 1e12, 4)}
            if v["tensor_flops"]:
                out[kk]["tensor_tflops_executed"] = round(v["tensor_flops"] / (v["ms_total"] * 1e-3) / 1e12, 2)
        return fam, out

    step = make_step(args.arith)
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
    total_ms = max_over_ranks(t_start.elapsed_time(t_end), world, dev)
    ms_per_step = total_ms / args.steps
    bytes_step = BYTES_PER_ROW * n
    value = whole_job_gbs(bytes_step, ms_per_step, world)

    # per-kernel-family time; the dominant one carries the roofline
    fam, families = families_of(evs, args.arith, args.steps)
    dom = max(fam, key=lambda k: fam[k]["ms_total"])
    roofline = roofline_of(fam[dom], dom, args.arith)

    # ---- the same step in the other arithmetics, reported beside the headline
    others = {}
    R2_main = R2.clone()
    for ar in ("fp64", "tc", "dd"):
        if ar == args.arith or (ar == "dd" and args.no_dd) or (ar == "tc" and args.no_tc):
            continue
        st_o = make_step(ar)
        for _ in range(2):
            st_o()
        torch.cuda.synchronize()
        ev_o = []
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            st_o(ev_o)
        b.record()
        torch.cuda.synchronize()
        if int(st.abs().sum().item()) != 0:
            raise RuntimeError(f"Cholesky breakdown in the benchmark input ({ar})")
        dms = a.elapsed_time(b) / args.steps
        fam_o, families_o = families_of(ev_o, ar, args.steps)
        dom_o = max(fam_o, key=lambda k: fam_o[k]["ms_total"])
        others[ar] = {"value": round(bytes_step / (dms * 1e-3) / 1e9, 3), "unit": "GB/s",
                      "ms_per_step": round(dms, 3), "arithmetic": ARITH_TEXT[ar], "kernels": families_o,
                      "roofline": roofline_of(fam_o[dom_o], dom_o, ar),
                      "max_abs_R_diff_vs_headline": float((R2 - R2_main).abs().max().item())}
    # leave the basis as the headline arithmetic produced it (e2e below re-copies it anyway)

    # ---- end to end through the library's own call on host buffers: every step
    # ortho_plan_run copies the page-locked host basis in (block by block, while
    # stage 1 runs), orthogonalizes it and copies Q and R back (in row ranges,
    # while the stage-2 update runs); the plan's device buffers are allocated
    # once, before the timed region
    e2e = None
    if not args.no_e2e and args.arith in ("tc", "fp64"):
        ar = capi.GMRES_ARITH_TC if args.arith == "tc" else capi.GMRES_ARITH_FP64
        plan = capi.OrthoPlan(n, S, NBLK, ar, stream)
        hostin = torch.from_numpy(host.T.copy()).pin_memory()
        hostin[0] /= torch.linalg.norm(hostin[0])
        hostq = torch.empty_like(hostin).pin_memory()
        hostrh = torch.zeros(NCOL, NCOL, dtype=torch.float64).pin_memory()
        hostr2 = torch.zeros(NCOL, NCOL, dtype=torch.float64).pin_memory()
        for _ in range(2):
            rc, _ = plan.run(hostin.T, hostq.T, hostrh.T, hostr2.T, on_device=False)
            if rc != 0:
                raise RuntimeError("Cholesky breakdown in the end-to-end steps")
        ke = max(3, min(args.steps, 10))
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for i in range(ke):
            rc, _ = plan.run(hostin.T, hostq.T, hostrh.T, hostr2.T, on_device=False)
            if rc != 0:
                raise RuntimeError("Cholesky breakdown in the end-to-end steps")
        b.record()
        torch.cuda.synchronize()
        plan.close()
        ems = max_over_ranks(a.elapsed_time(b) / ke, world, dev)
        e2e = {"value": round(whole_job_gbs(bytes_step, ems, world), 3), "unit": "GB/s",
               "h2d_bytes_per_step": int(hostin.numel() * 8),
               "d2h_bytes_per_step": int(hostq.numel() * 8 + hostrh.numel() * 8 + hostr2.numel() * 8),
               "ms_per_step": round(ems, 3), "steps": ke,
               "call": "ortho_plan_run on page-locked host buffers (one library call per step)",
               "overlap": "inside each call: columns in block by block during stage 1, Q out in row ranges "
                          "during the stage-2 update"}

    # ---- the FP64 solver on the same grid: one restart cycle, and C1 to convergence
    solve = None
    if not args.no_solve and rank == 0:
        solve = solver_numbers(capi, dev, args)

    # ---- the precision, batching and serving patterns
    patterns = None
    if not args.no_patterns and rank == 0:
        patterns = {"mixed_precision": mixed_numbers(capi, dev), "batched": batched_numbers(capi, args),
                    "serving": serving_numbers(capi, args)}

    # ---- CPU oracle on a bounded sample of the same workload
    cpu = None
    cpu_solver = None
    if rank == 0 and not args.no_cpu:
        rows, steps = n, 2
        val, dt = cpu_oracle_rate(rows, steps)
        cpu = {"value": round(val, 3), "unit": "GB/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"{steps} steps on all {rows} rows (numpy FP64 oracle), {dt:.1f} s"}
        cpu_solver = oracle_numbers(args)

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_TEXT[args.arith], "data": "synthetic",
                "config": {"workload": WORKLOAD, "n": n, "cols": NCOL, "s": S, "panel": NCOL - 1,
                           "bytes_per_step": bytes_step, "l2": "basis 2 GB >> 129 MB L2, no flush needed",
                           "parallelism": "replicas" if world > 1 else "single"},
                "arith": ARITH_TEXT[args.arith], "roofline": roofline, "kernels": families,
                "other_arith": others, "e2e": e2e, "cpu_baseline": cpu,
                "gpu_launches": (2 * NBLK + 2 + (1 if args.arith == "tc" and not args.no_digits else 0)) * args.steps,
                "clocks": clk,
                "solver": solve, "cpu_solver": cpu_solver,
                "patterns": patterns}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _time_solve(capi, A, bd, dev, opts, reps=3):
    """Median wall time of gmres_solve (device b and x) after one warm-up solve
    (the warm-up captures the cycle graphs); the result dict of the last solve."""
    import torch
    S = capi.Solver.from_csr(A, opts)
    xd = torch.zeros(A.n, dtype=torch.float64, device=dev)
    S.solve(bd, xd)
    times = []
    for _ in range(reps):
        xd.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, res = S.solve(bd, xd)
        times.append(time.perf_counter() - t0)
    S.close()
    return statistics.median(times), rc, res


def solver_numbers(capi, dev, args):
    """Time to solution of the s-step GMRES solver: the 64 x 64 case (C1) and
    the 2048 x 2048 case (C2) at tol 1e-8 for the two-stage scheme and the
    paper's comparisons (standard GMRES as s = 1, BCGS-PIP2 = two-stage with
    s^ = s, BCGS2-CholQR2), monomial and automatic Newton basis, FP64 and
    tensor-core arithmetic, with the Gauss-Seidel preconditioner and with
    shifted CholQR; one timed restart cycle per scheme and s^ in {5, 20, 40,
    60} with per-phase times (the layout of Table 2)."""
    import torch
    import synth
    from scipy.sparse import csr_matrix
    out = {}
    T, A = capi.GMRES_ARITH_TC, capi.GMRES_ARITH_FP64
    NA, MO = capi.GMRES_BASIS_NEWTON_AUTO, capi.GMRES_BASIS_MONOMIAL

    def tts_table(grid, variants, reps):
        Am = synth.laplace2d(grid)
        b = csr_matrix((Am.vals, Am.colind, Am.rowptr), shape=(Am.n, Am.n)) @ synth.x_true(Am.n, 0)
        bd = torch.tensor(b, device=dev)
        tab = {}
        for name, kw in variants:
            o = dict(m=60, s=5, panel=60, tol=1e-8, max_restarts=5000)
            o.update(kw)
            dt, rc, res = _time_solve(capi, Am, bd, dev, capi.default_opts(**o), reps)
            tab[name] = {"time_to_solution_ms": round(1e3 * dt, 3), "status": rc, "iters": res["iters"],
                         "restarts": res["restarts"], "relres": res["relres_true"]}
        return tab

    c1 = [("fp64", dict(arith=A)), ("tc", dict(arith=T)),
          ("s10_newton_auto_fp64", dict(s=10, basis=NA, arith=A)), ("s10_newton_auto_tc", dict(s=10, basis=NA, arith=T)),
          ("s10_monomial_shifted_fp64", dict(s=10, shift=1, arith=A)),
          ("bcgs2_cholqr2_fp64", dict(ortho=capi.GMRES_ORTHO_BCGS2_CHOLQR2, arith=A))]
    out["laplace64_time_to_solution"] = tts_table(64, c1, 5)
    if args.rows == N_ROWS:
        c2 = [("two_stage_fp64", dict(arith=A)), ("two_stage_tc", dict(arith=T)),
              ("two_stage_s10_newton_auto_fp64", dict(s=10, basis=NA, arith=A)),
              ("two_stage_s10_newton_auto_tc", dict(s=10, basis=NA, arith=T)),
              ("two_stage_gauss_seidel_newton_auto_tc", dict(basis=NA, arith=T, precond=1)),
              ("two_stage_monomial_shifted_tc", dict(basis=MO, arith=T, shift=1)),
              ("two_stage_s10_monomial_shifted_tc", dict(s=10, basis=MO, arith=T, shift=1)),
              ("bcgs_pip2_fp64", dict(ortho=capi.GMRES_ORTHO_BCGS_PIP2, arith=A)),
              ("bcgs2_cholqr2_fp64", dict(ortho=capi.GMRES_ORTHO_BCGS2_CHOLQR2, arith=A)),
              ("bcgs2_cholqr2_tc", dict(ortho=capi.GMRES_ORTHO_BCGS2_CHOLQR2, arith=T)),
              ("standard_gmres_s1_fp64", dict(s=1, panel=1, arith=A))]
        tab = tts_table(2048, c2, 1)
        base = tab["bcgs2_cholqr2_fp64"]["time_to_solution_ms"]
        for v in tab.values():
            v["speedup_vs_bcgs2_cholqr2_fp64"] = round(base / v["time_to_solution_ms"], 3) if v["status"] == 0 else None
        out["laplace2048_time_to_solution"] = tab

        # one restart cycle per scheme and s^, per phase (Table 2's columns)
        Am = synth.laplace2d(2048)
        b = csr_matrix((Am.vals, Am.colind, Am.rowptr), shape=(Am.n, Am.n)) @ synth.x_true(Am.n, 0)
        bd = torch.tensor(b, device=dev)
        xd = torch.zeros(Am.n, dtype=torch.float64, device=dev)
        rows = [(f"two_stage_shat{p}", capi.GMRES_ORTHO_TWO_STAGE, p) for p in (5, 20, 40, 60)]
        rows.append(("bcgs2_cholqr2", capi.GMRES_ORTHO_BCGS2_CHOLQR2, 5))
        cycles = {}
        for name, ortho, panel in rows:
            for aname, arith in (("fp64", A), ("tc", T)):
                opts = capi.default_opts(m=60, s=5, panel=panel, tol=1e-14, max_restarts=1, timing=1, ortho=ortho,
                                         arith=arith)
                S2 = capi.Solver.from_csr(Am, opts)
                S2.solve(bd, xd)
                xd.zero_()
                rc, res = S2.solve(bd, xd)
                S2.close()
                cyc = res["t_total_ms"]
                cycles[f"{name}_{aname}"] = {
                    "ms_per_restart_cycle": round(cyc, 3), "iters": res["iters"],
                    "t_mpk_ms": round(res["t_mpk_ms"], 3), "t_ortho_ms": round(res["t_stage1_ms"] + res["t_stage2_ms"], 3),
                    "t_stage1_ms": round(res["t_stage1_ms"], 3), "t_stage2_ms": round(res["t_stage2_ms"], 3),
                    "t_ls_ms": round(res["t_ls_ms"], 3), "relres_after_one_cycle": res["relres_true"], "status": rc}
        base = cycles["bcgs2_cholqr2_fp64"]
        for v in cycles.values():
            v["ortho_speedup_vs_bcgs2_cholqr2_fp64"] = round(base["t_ortho_ms"] / v["t_ortho_ms"], 3)
            v["cycle_speedup_vs_bcgs2_cholqr2_fp64"] = round(base["ms_per_restart_cycle"] / v["ms_per_restart_cycle"], 3)
        out["laplace2048_shat_sweep_cycle"] = cycles
    return out


def oracle_numbers(args):
    """The CPU oracle (numpy FP64, all host cores) on the solver workloads: the
    64 x 64 time to solution (C1) and one restart cycle of the 2048 x 2048 (C2)
    and 160^3 (C3, FP64) systems, m = 60, s = 5, s^ = 60 (a bounded sample: a
    full solve takes many cycles)."""
    import synth
    from oracle import krylov as kr
    out = {"cores": cpu_threads(), "kind": "oracle"}
    A = synth.laplace2d(64)
    b = kr.as_operator(A) @ synth.x_true(A.n, 0)
    t0 = time.perf_counter()
    _, info = kr.sstep_gmres(A, b, m=60, s=5, panel=60, tol=1e-8)
    out["laplace64_time_to_solution_ms"] = round(1e3 * (time.perf_counter() - t0), 1)
    out["laplace64_iters"] = info["iters"]
    if args.rows == N_ROWS and not args.no_oracle_cycles:
        for name, A in (("laplace2048", synth.laplace2d(2048)), ("laplace3d_160", synth.laplace3d(160))):
            b = kr.as_operator(A) @ synth.x_true(A.n, 0)
            t0 = time.perf_counter()
            _, info = kr.sstep_gmres(A, b, m=60, s=5, panel=60, tol=1e-30, max_restarts=1)
            dt = time.perf_counter() - t0
            out[name + "_one_cycle_ms"] = round(1e3 * dt, 1)
            out[name + "_ms_per_iteration"] = round(1e3 * dt / max(info["iters"], 1), 2)
            out[name + "_iters"] = info["iters"]
    return out


def mixed_numbers(capi, dev):
    """Mixed-precision configuration: 3D Laplace 7-point on 160^3, FP32 basis and
    MPK, FP64 Gram/Cholesky/Hessenberg and refinement, m=60, s=10, s^=60,
    tol 1e-8.  Time to solution, and the error against x_true and against the
    FP64 path on the same system."""
    import numpy as np
    import torch
    import synth
    from scipy.sparse import csr_matrix
    A = synth.laplace3d(160)
    xt = synth.x_true(A.n, 0)
    M = csr_matrix((A.vals, A.colind, A.rowptr), shape=(A.n, A.n))
    b = M @ xt
    bd = torch.tensor(b, device=dev)
    out = {"grid": "160^3", "n": A.n}
    xs = {}
    auto = capi.GMRES_BASIS_NEWTON_AUTO
    runs = (("mixed", capi.GMRES_PREC_MIXED, 0, 0), ("fp64", capi.GMRES_PREC_FP64, 0, 0),
            # the Newton basis with automatic Leja-ordered Ritz shifts, where the
            # monomial basis breaks down at s = 10
            ("mixed_newton_auto", capi.GMRES_PREC_MIXED, auto, 0),
            ("fp64_newton_auto", capi.GMRES_PREC_FP64, auto, capi.GMRES_ARITH_FP64),
            ("tc_newton_auto", capi.GMRES_PREC_FP64, auto, capi.GMRES_ARITH_TC),
            # mixed precision with the Gram accumulated in double-float on the FP32 pipe
            ("mixed_dd_newton_auto", capi.GMRES_PREC_MIXED, auto, capi.GMRES_ARITH_DD))
    for name, prec, basis, arith in runs:
        S = capi.Solver.from_csr(A, capi.default_opts(m=60, s=10, panel=60, tol=1e-8, precision=prec,
                                                      max_restarts=2000, basis=basis, arith=arith))
        xd = torch.zeros(A.n, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, res = S.solve(bd, xd)
        dt = time.perf_counter() - t0
        S.close()
        x = xd.cpu().numpy()
        xs[name] = (rc, x)
        out[name] = {"status": rc, "time_to_solution_s": round(dt, 3), "iters": res["iters"],
                     "restarts": res["restarts"], "ir_steps": res["ir_steps"], "relres": res["relres_true"],
                     "err_vs_x_true": float(np.linalg.norm(x - xt) / np.linalg.norm(xt)),
                     "breakdown_block": res["breakdown_block"]}
        if basis == auto:
            out[name]["sigma"] = res["sigma"]
            out[name]["theta"] = [round(t, 6) for t in res["theta"][:10]]
    ref = "fp64" if xs["fp64"][0] == 0 else ("fp64_newton_auto" if xs["fp64_newton_auto"][0] == 0 else None)
    if ref:
        for name in out:
            if isinstance(out[name], dict) and name != ref and xs.get(name, (1,))[0] == 0:
                out[name]["err_vs_" + ref] = float(np.linalg.norm(xs[name][1] - xs[ref][1]) /
                                                   np.linalg.norm(xs[ref][1]))
    return out


def batched_systems(nsys, seed, nmin, nmax):
    """Half 2D upwinded convection-diffusion (5-point, cell Peclet ~ U(0,10)),
    half random banded (27 nnz/row, bandwidth 1000, N(0,1) off-diagonals,
    diagonally dominant), n log-uniform in [nmin, nmax]."""
    import numpy as np
    import synth
    g = synth.rng(seed)
    mats = []
    for i in range(nsys):
        n = int(np.exp(g.uniform(np.log(nmin), np.log(nmax))))
        if i % 2 == 0:
            mats.append(synth.convdiff2d(int(np.ceil(np.sqrt(n))), seed * 100000 + i))
        else:
            mats.append(synth.banded_random(n, seed * 100000 + i))
    return mats


def _rate(systems, converged, wall):
    return {"systems": systems, "converged": int(converged), "wall_s": round(wall, 3),
            "raw_solves_per_s": round(systems / wall, 3), "converged_per_s": round(converged / wall, 3),
            "ms_per_converged": round(1e3 * wall / converged, 2) if converged else None}


def batched_numbers(capi, args):
    """Batched configuration: 256 nonsymmetric systems, n log-uniform in
    [1e4, 5e5], s=5, m=40, s^=40, tol 1e-8, one persistent launch per step
    under captured CUDA graphs, autotuned grids.  Like for like: the batched
    engine and the single-system solver one system at a time with the same
    algorithm (FP64, monomial: both see the same breakdowns), then the
    precision pattern batched (FP32 basis, explicit projected Gram) against
    FP64 one at a time with the basis that converges on every system (Newton,
    automatic shifts) and with shifted CholQR.  Every arm: raw and converged
    solves per second of wall time."""
    import numpy as np
    import synth
    from scipy.sparse import csr_matrix
    t0 = time.perf_counter()
    mats = batched_systems(args.batch_systems, 2, 1e4, args.batch_nmax)
    bs = [csr_matrix((A.vals, A.colind, A.rowptr), shape=(A.n, A.n)) @ synth.x_true(A.n, i)
          for i, A in enumerate(mats)]
    gen_s = time.perf_counter() - t0
    nsys = len(mats)
    out = {"systems": nsys, "rows": int(sum(A.n for A in mats)), "nnz": int(sum(A.nnz for A in mats)),
           "generate_s": round(gen_s, 1)}

    def batched(name, o):
        B = capi.Batch(mats, o)
        tune = B.autotune()
        B.solve(bs, [np.zeros(A.n) for A in mats])   # warm-up (graph capture)
        xs = [np.zeros(A.n) for A in mats]
        t0 = time.perf_counter()
        rc, res = B.solve(bs, xs)
        wall = time.perf_counter() - t0
        B.close()
        ok = [r for r in res if r["status"] == 0]
        out[name] = dict(_rate(nsys, len(ok), wall), max_relres=max(r["relres_true"] for r in ok) if ok else None,
                         iters_median=int(np.median([r["iters"] for r in res])), autotune=tune)

    def one_at_a_time(name, o, note):
        t0 = time.perf_counter()
        ok = 0
        for A, b in zip(mats, bs):
            S = capi.Solver.from_csr(A, o)
            x = np.zeros(A.n)
            rc1, r1 = S.solve(b, x)
            S.close()
            ok += rc1 == 0
        out[name] = dict(_rate(nsys, ok, time.perf_counter() - t0), note=note)

    common = dict(m=40, s=5, panel=40, tol=1e-8, max_restarts=500)
    batched("fp64_batched_monomial", capi.default_opts(**common))
    one_at_a_time("fp64_one_at_a_time_monomial", capi.default_opts(**common),
                  "the same algorithm as fp64_batched_monomial; includes per-system create/destroy")
    batched("mixed_batched", capi.default_opts(precision=capi.GMRES_PREC_MIXED, **common))
    batched("mixed_batched_dd_gram", capi.default_opts(precision=capi.GMRES_PREC_MIXED, arith=capi.GMRES_ARITH_DD,
                                                       **common))
    one_at_a_time("fp64_one_at_a_time_newton_auto",
                  capi.default_opts(basis=capi.GMRES_BASIS_NEWTON_AUTO, **common),
                  "FP64, automatic Newton shifts (the batched engine takes given shifts only)")
    one_at_a_time("fp64_one_at_a_time_shifted_cholqr",
                  capi.default_opts(shift=capi.GMRES_SHIFT_CHOLQR3, **common),
                  "FP64, monomial, shifted CholQR (stage 1 shifted, stage 2 shifted CholQR3)")
    return out


def serving_numbers(capi, args):
    """Serving configuration: Poisson arrivals (rate swept) of solves drawn from
    2D Laplace grids 128^2..1024^2 and 3D convection-diffusion grids
    32^3..128^3, s in {5,10}, m in {30,60}, s^ = m, mixed precision served with
    footprint admission; p50/p99 latency and solves/s, against the plain FP64
    path solving the same requests one at a time."""
    import numpy as np
    import synth
    from scipy.sparse import csr_matrix
    g = synth.rng(3)
    cache = {}

    def mat(kind, N):
        key = (kind, N)
        if key not in cache:
            cache[key] = synth.laplace2d(N) if kind == "lap2d" else synth.convdiff3d(N, 7000 + N)
        return cache[key]

    reqs = []
    for i in range(args.serve_requests):
        if g.random() < 0.5:
            A = mat("lap2d", int(g.choice([128, 256, 512, 1024])))
        else:
            A = mat("cd3d", int(g.choice([32, 64, 96, 128])))
        s = int(g.choice([5, 10]))
        m = int(g.choice([30, 60]))
        b = csr_matrix((A.vals, A.colind, A.rowptr), shape=(A.n, A.n)) @ synth.x_true(A.n, i)
        reqs.append((A, b, s, m))
    # served: FP32 basis and MPK, Gram accumulated in double-float (about 2^-48, on the
    # FP32 pipe), FP64 Cholesky / Hessenberg / refinement, Newton basis with automatic
    # shifts (s = 10 requests keep converging)
    def served_opts(s, m, **kw):
        o = dict(precision=capi.GMRES_PREC_MIXED, arith=capi.GMRES_ARITH_DD, basis=capi.GMRES_BASIS_NEWTON_AUTO)
        o.update(kw)
        return capi.default_opts(m=m, s=s, panel=m, tol=1e-8, max_restarts=args.serve_restarts, **o)

    out = {"requests": len(reqs), "max_restarts": args.serve_restarts,
           "served": "mixed precision (FP32 basis/MPK), double-float Gram accumulation, FP64 Cholesky, Hessenberg "
                     "and refinement, Newton basis with Leja-ordered Ritz shifts",
           "rates": []}

    def serve(rate, opts_of):
        # rate 0: every request arrives at t = 0 (saturated server, peak solves/s)
        arr = np.cumsum(g.exponential(1.0 / rate, size=len(reqs))) if rate > 0 else np.zeros(len(reqs))
        srv = capi.Server(max_active=32)
        ids = []
        t0 = time.perf_counter()
        for (A, b, s, m), ta in zip(reqs, arr):
            while time.perf_counter() - t0 < ta:
                time.sleep(0.001)
            ids.append(srv.submit(A, b, opts=opts_of(s, m)))
        res = [srv.wait(i) for i in ids]
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.stop()
        conv = sum(1 for _, r in res if r["status"] == 0)
        d = dict(_rate(len(reqs), conv, wall), p50_ms=round(st["p50_ms"], 2), p99_ms=round(st["p99_ms"], 2),
                 server_busy_s=round(st["busy_s"], 3), statuses=sorted(set(r["status"] for _, r in res)))
        return d

    for rate in list(args.serve_rates) + [0.0]:
        d = serve(rate, served_opts)
        d["rate_per_s"] = rate if rate > 0 else "saturated"
        out["rates"].append(d)
    # the same requests served in plain FP64 (FP64 basis and Gram) with the same basis
    out["served_fp64_newton_auto_saturated"] = serve(0.0, lambda s, m: served_opts(
        s, m, precision=capi.GMRES_PREC_FP64, arith=capi.GMRES_ARITH_FP64))

    def one_at_a_time(basis):
        t0 = time.perf_counter()
        conv = 0
        for A, b, s, m in reqs:
            S = capi.Solver.from_csr(A, capi.default_opts(m=m, s=s, panel=m, tol=1e-8, basis=basis,
                                                          max_restarts=args.serve_restarts))
            x = np.zeros(A.n)
            rc, r = S.solve(b, x)
            S.close()
            conv += rc == 0
        return _rate(len(reqs), conv, time.perf_counter() - t0)

    # like for like: plain FP64 one request at a time with the served basis, and
    # with the monomial basis (whose s = 10 requests break down)
    out["fp64_one_at_a_time_newton_auto"] = one_at_a_time(capi.GMRES_BASIS_NEWTON_AUTO)
    out["fp64_one_at_a_time_monomial"] = one_at_a_time(capi.GMRES_BASIS_MONOMIAL)
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
    ap.add_argument("--no-oracle-cycles", action="store_true",
                    help="skip the oracle's restart cycles on the 2048^2 and 160^3 systems (about 40 s of CPU)")
    ap.add_argument("--no-patterns", action="store_true", help="skip the mixed, batched and serving configurations")
    ap.add_argument("--no-dd", action="store_true", help="skip the double-float measurement")
    ap.add_argument("--no-tc", action="store_true", help="skip the tensor-core Gram measurement")
    ap.add_argument("--no-digits", action="store_true",
                    help="tensor-core step without the resident digit basis (every read re-slices)")
    ap.add_argument("--arith", default="tc", choices=["fp64", "tc", "dd"],
                    help="arithmetic of the headline step (the others are reported beside it)")
    ap.add_argument("--batch-systems", type=int, default=256)
    ap.add_argument("--batch-nmax", type=float, default=5e5)
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-restarts", type=int, default=100)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[2.0, 8.0])
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
