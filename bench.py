#!/usr/bin/env python
"""Benchmark of the wave-equation hot path on the batched 64-shot workload.

Workload (default): 400 x 1200 seeded layered-fault model, dx 12.5 m,
dt 1 ms, 20-cell sponge, 8 Hz Ricker, 64 surface shots with 200-600
receivers and 3000-4000 samples each, all shots in one batched pass.

One step = one deblurred FWI iteration, in the order of the paper:
  1. fwi_gradient: forward modelling + misfit + adjoint-state gradient
     (forward pass storing a^n of every step device memory holds -- all of
     them on one GB300 -- checkpoints and segment recomputation for any
     others, adjoint pass);
  2. born_demig of the gradient (background + scattered fields jointly);
  3. rtm_mig of those Born data -> the doubly migrated image (Eq. 15);
  4. deblur_train: warm-started U-Net training on the (doubly migrated
     image -> gradient) pair, 20 epochs of 108 patches of 128 x 128, batch 32
     (the 200-epoch cold start runs once before the timed region);
  5. deblur_apply to the full gradient, 6. fwi_update of the model.
value = algorithmic cell updates per second, Gcell-updates/s: per step
6 U (forward U + adjoint U for the gradient, 2 U for Born, forward U +
adjoint U for migration), U = sum over shots of nt_s x padded window cells.
Checkpoint recomputation (up to 2 U more per step) is overhead and not counted.

--impl reference times the FP64 CPU oracle (the only other implementation
of this path) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FD Gcell-updates/s & HBM roofline %; model error vs GPU-s, deblurred vs plain"
UNIT = "Gcell-updates/s"
# Algorithmic bytes per cell update (the three-level count: kappa and the
# sponge come from a model shared by every shot, L2-resident, so they are not
# counted).  A forward update reads u^n and u^{n-1} and writes u^{n+1}; the
# forward pass of a gradient or migration also stores a^n; an adjoint update
# moves the same 12 B plus the read of a^n; a Born cell-step advances two
# fields (24 B) and reads the perturbation (4 B), counted as two updates.
FWD_BYTES_PER_CELL = 12
HIST_BYTES_PER_CELL = 4
ADJ_BYTES_PER_CELL = 16
BORN_BYTES_PER_CELL_STEP = 28
# The bytes the summed form the kernels use must move (u and D = u - w u^{n-1}
# both change every step): 16 B per forward update.  Reported as an extra.
SUMMED_FWD_BYTES_PER_CELL = 16


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="config2", choices=["config2", "config1", "marmousi"],
                   help="config2: the 64-shot 400 x 1200 batch (the benchmark); config1: the small parity case; "
                        "marmousi: the 30-shot 221 x 601 case of the paper's Marmousi test's shape")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--only", default="", choices=["", "fwd", "grad", "born", "nn"],
                   help="fwd: time batched forward modelling (model_shots) alone; grad: the FWI gradient "
                        "(fwi_gradient: forward storing the history, adjoint) alone; born: Born demigration "
                        "(born_demig) alone; nn: the network's training and apply alone on seeded smooth images "
                        "of the workload's size; used for profiling")
    p.add_argument("--nn-epochs", type=int, default=20)
    p.add_argument("--net", default="workload", choices=["workload", "paper"],
                   help="with --only nn: workload = base 32 on 128 x 128 patches (the benchmark's network); "
                        "paper = the paper's network (base 128 doubling to 2048, four levels) trained on the "
                        "full image (one padded sample per step); --nn-epochs is then the number of steps")
    p.add_argument("--shots", type=int, default=0,
                   help="with --only fwd/grad/born: the first SHOTS shots of the batch (small profiling captures)")
    p.add_argument("--nt", type=int, default=0,
                   help="with --only fwd/grad/born: records truncated to NT samples (small profiling captures)")
    p.add_argument("--reuse", action="store_true",
                   help="turn on dhfwi_set_reuse (Born and migration take the background from the gradient's stored "
                        "forward pass); the value still counts the step's 6 U algorithmic updates, and "
                        "performed_cell_updates_per_step says how many ran")
    p.add_argument("--cold-epochs", type=int, default=COLD_EPOCHS,
                   help="epochs of the network's cold start before the timed region (setup only)")
    return p.parse_args()


def make_case(name, shots=0, nt=0):
    """The workload; shots > 0 keeps the first shots of the 64-shot batch,
    nt > 0 truncates the records (profiling modes only: small captures of
    the same kernels)."""
    import numpy as np
    import synth

    case = {"config2": synth.config2_case, "config1": synth.config1_case,
            "marmousi": synth.marmousi_shaped_case}[name]()
    if shots > 0 and shots < case.geom.n_shots:
        case.geom = case.geom.subset(list(range(shots)))
    if nt > 0:
        g = case.geom
        g.nt = np.minimum(g.nt, nt).astype(np.int32)
        g.wavelet = np.ascontiguousarray(g.wavelet[..., : int(g.nt.max())])
    return case


def algorithmic_cells(case) -> int:
    return 6 * case.geom.cell_updates(case.nz, case.nb)


NET = dict(base_channels=32, levels=4, patch=128, stride=64, batch=32, lr=1e-3, seed=29, mute_rows=5, warmup_frac=0.1)
NET_PAPER = dict(base_channels=128, levels=4, patch=0, stride=1, batch=1, lr=1e-4, seed=29, mute_rows=5,
                 warmup_frac=0.1)
WARM_EPOCHS, COLD_EPOCHS = 20, 200


def conv_flops(base, levels, H, W):
    """Multiply-add FLOPs (2 per MAC) of one forward pass of the U-Net on H x W."""
    f = 0
    C = lambda l: base << l
    f += 2 * H * W * 9 * (1 * C(0) + C(0) * C(0))
    for l in range(1, levels + 1):
        h, w = H >> l, W >> l
        f += 2 * h * w * 9 * (C(l - 1) * C(l) + C(l) * C(l))
    for l in range(1, levels + 1):
        r = levels - l
        h, w = H >> r, W >> r
        f += 2 * (h // 2) * (w // 2) * C(r + 1) * 4 * C(r)          # transposed conv
        f += 2 * h * w * 9 * (2 * C(r) * C(r) + C(r) * C(r))
    f += 2 * H * W * C(0)
    return f


def n_patches(n, p, s):
    o = list(range(0, n - p + 1, s))
    if o[-1] != n - p:
        o.append(n - p)
    return len(o)


# ---------------------------------------------------------------------------
# Distributed plumbing (replicas: every rank runs the whole workload)
# ---------------------------------------------------------------------------
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist

            backend = "nccl"
            try:
                import torch

                if not torch.cuda.is_available():
                    backend = "gloo"
            except Exception:
                backend = "gloo"
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            import torch

            if torch.cuda.is_available():
                self.pg.barrier(device_ids=[self.local])
            else:
                self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch

        dev = torch.device("cuda", self.local) if torch.cuda.is_available() else torch.device("cpu")
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# ncu traffic from the committed profile (null when the kernel has changed)
# ---------------------------------------------------------------------------
# Sources of each step kernel: its profile under profiles/ records their
# hash, and its DRAM figures are used only while the hash matches.
KERNEL_SOURCES = {
    "fwd_step_kernel": ["fd_kernels.cu", "fd_device.cuh"],
    "fwd_tma_kernel": ["fd_tma.cu", "fd_tma.cuh", "fd_device.cuh"],
    "fwd_pair_kernel": ["fd_tma2.cu", "fd_tma.cuh", "fd_device.cuh"],
    "adj_pair_kernel": ["fd_tma2.cu", "fd_tma.cuh", "fd_device.cuh"],
    "born_tma_kernel": ["fd_tma.cu", "fd_tma.cuh", "fd_device.cuh"],
}


def kernel_source_hash(kernel: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(ROOT, "paper_2403_17518_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def forward_kernel(variant: int) -> str:
    """Name of the forward step kernel a step-kernel variant launches."""
    return "fwd_tma_kernel" if variant >= 3 else "fwd_step_kernel"


def profiled_traffic(kernel: str, cells_per_launch: float):
    """DRAM bytes per launch of a step kernel from profiles/, scaled to this
    launch size by its cell updates, or None if absent or taken on another
    kernel source."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_config2.md")
    if not os.path.exists(path) or kernel not in KERNEL_SOURCES:
        return None
    txt = open(path).read()
    m_hash = re.search(r"kernel source sha256\[:16\]:\s*`?([0-9a-f]{16})", txt)
    m_bpc = re.search(r"DRAM bytes per cell update:\s*([0-9.]+)", txt)
    if not m_hash or not m_bpc or m_hash.group(1) != kernel_source_hash(kernel):
        return None
    return float(m_bpc.group(1)) * cells_per_launch


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(case, n_shots: int, nt: int):
    import numpy as np

    g = case.geom.subset(list(range(min(n_shots, case.geom.n_shots))))
    g.nt = np.minimum(g.nt, nt).astype(np.int32)
    g.wavelet = np.ascontiguousarray(g.wavelet[:nt])
    return g


def run_oracle_step(case, g, d_obs):
    import oracle

    J, grad, _ = oracle.fwi_gradient(case.v_init, g, d_obs, case.h, case.dt, case.nb)
    db = oracle.born_demig(case.v_init, g, grad, case.h, case.dt, case.nb)
    oracle.rtm_mig(case.v_init, g, db, case.h, case.dt, case.nb)


def oracle_measure(case, n_shots, nt, steps, warmup):
    import oracle

    oracle.build()
    g = oracle_sample(case, n_shots, nt)
    d_obs = oracle.model_shots(case.v_true, g, case.h, case.dt, case.nb)
    for _ in range(warmup):
        run_oracle_step(case, g, d_obs)
    t0 = time.perf_counter()
    for _ in range(steps):
        run_oracle_step(case, g, d_obs)
    el = time.perf_counter() - t0
    cells = 6 * g.cell_updates(case.nz, case.nb) * steps
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    cores = min(cores, os.cpu_count() or 1)
    sample = (f"{g.n_shots} of {case.geom.n_shots} shots (first ones), each truncated to nt={nt} "
              f"samples, full {case.nz}x{case.nx} grid; gradient + Born + migration, FP64, OpenMP over shots")
    return cells / el / 1e9, el / steps, cores, sample


def cpu_cores():
    return os.cpu_count() or 1


def run_reference(args, dist):
    if dist.rank != 0:
        return
    case = make_case(args.workload)
    cores = cpu_cores()
    n_shots = min(cores, case.geom.n_shots)
    val, sec, used, sample = oracle_measure(case, n_shots, 150, max(args.steps, 1), args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(val, 6), "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sec * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(case, args),
        "cpu_baseline": {"value": round(val, 6), "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(val, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(case, args):
    return {
        "workload": f"{case.name}: one deblurred FWI iteration (forward modelling + adjoint-state gradient + "
                    f"Born demigration + migration + warm-started U-Net training + apply + model update)",
        "grid": [case.nz, case.nx], "h_m": case.h, "dt_s": case.dt, "sponge": case.nb,
        "shots": case.geom.n_shots, "nt_range": [int(case.geom.nt.min()), int(case.geom.nt.max())],
        "receivers_range": [int(min(case.geom.nrec(s) for s in range(case.geom.n_shots))),
                            int(max(case.geom.nrec(s) for s in range(case.geom.n_shots)))],
        "cell_updates_per_step": algorithmic_cells(case),
        "l2": "inputs larger than L2 (72 MB wavefield pools; the a^n history, ~250 GB, is written and read "
              "once per gradient and migration call)",
        "parallelism": f"replicas x{args.gpus}" if args.gpus > 1 else "single GPU",
    }


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------
def run_network_only(args, dist, case):
    """Network training (warm, --nn-epochs) and full-image apply alone."""
    import numpy as np
    import torch

    import synth
    from paper_2403_17518_gb300.ops import Context

    ctx = Context(case.nz, case.nx, case.h, case.dt, case.nb, device=dist.local)
    dev = torch.device("cuda", dist.local)
    x = torch.tensor(synth.smooth_random_field(case.nz, case.nx, 1, 3.0), dtype=torch.float32, device=dev)
    y = torch.tensor(synth.smooth_random_field(case.nz, case.nx, 2, 1.5), dtype=torch.float32, device=dev)
    out = torch.empty_like(y)
    net = NET_PAPER if args.net == "paper" else NET
    ctx.deblur_train(x, y, warm_start=False, epochs=1, **net)
    for _ in range(args.warmup):
        ctx.deblur_train(x, y, warm_start=True, epochs=args.nn_epochs, **net)
        ctx.deblur_apply(y, out=out)
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record()
    for _ in range(args.steps):
        ctx.deblur_train(x, y, warm_start=True, epochs=args.nn_epochs, **net)
    e1.record()
    for _ in range(args.steps):
        ctx.deblur_apply(y, out=out)
    e2.record()
    torch.cuda.synchronize()
    mult = 1 << net["levels"]
    Hp, Wp = -(-case.nz // mult) * mult, -(-case.nx // mult) * mult
    if args.net == "paper":
        npatch = 1
        f_train = args.nn_epochs * 3 * conv_flops(net["base_channels"], net["levels"], Hp, Wp)
    else:
        npatch = n_patches(case.nz, net["patch"], net["stride"]) * n_patches(case.nx, net["patch"], net["stride"])
        f_train = args.nn_epochs * npatch * 3 * conv_flops(net["base_channels"], net["levels"], net["patch"],
                                                           net["patch"])
    f_apply = conv_flops(net["base_channels"], net["levels"], Hp, Wp)
    t_train = e0.elapsed_time(e1) / max(args.steps, 1)
    t_apply = e1.elapsed_time(e2) / max(args.steps, 1)
    if dist.rank == 0:
        print(json.dumps({"only": "nn", "net": args.net, "base_channels": net["base_channels"],
                          "full_image": net["patch"] == 0, "params": ctx.net_size(),
                          "epochs": args.nn_epochs, "patches": npatch,
                          "train_ms": round(t_train, 2), "train_tflops": round(f_train / t_train / 1e9, 2),
                          "apply_ms": round(t_apply, 2), "apply_tflops": round(f_apply / t_apply / 1e9, 2)}),
              flush=True)
    ctx.close()


def run_forward_only(args, dist, ctx, case, geom, v0, d_out):
    """Batched forward modelling alone (model_shots), for kernel profiling."""
    import torch

    for _ in range(args.warmup):
        ctx.model_shots(v0, geom, out=d_out)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        ctx.model_shots(v0, geom, out=d_out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    U = case.geom.cell_updates(case.nz, case.nb)
    st = ctx.stats()
    peak, peak_kind = peaks()
    alg = FWD_BYTES_PER_CELL * U / ms / 1e6
    if dist.rank == 0:
        print(json.dumps({"only": "fwd", "workload": case.name, "ms_per_pass": round(ms, 3),
                          "step_variants": st["step_variant"],
                          "gcell_per_s": round(U / ms / 1e6, 3), "launches_per_pass": st["kernel_launches"],
                          "algorithmic_bytes_per_cell": FWD_BYTES_PER_CELL, "algorithmic_GBps": round(alg, 1),
                          "frac": round(alg / peak, 4), "peak": peak, "peak_kind": f"{peak_kind} (hbm_gbs)",
                          "summed_form_GBps": round(SUMMED_FWD_BYTES_PER_CELL * U / ms / 1e6, 1)}), flush=True)


def run_gradient_only(args, dist, ctx, case, geom, v0, d_obs):
    """The FWI gradient alone (fwi_gradient), for kernel profiling."""
    import torch

    grad = ctx.new_model()
    ctx.set_timing(True)
    for _ in range(args.warmup):
        ctx.fwi_gradient(v0, geom, d_obs, grad=grad)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        ctx.fwi_gradient(v0, geom, d_obs, grad=grad)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    st = ctx.stats()
    U = case.geom.cell_updates(case.nz, case.nb)
    if dist.rank == 0:
        print(json.dumps({"only": "grad", "workload": case.name, "ms_per_call": round(ms, 3),
                          "forward_ms": round(st["phase_ms"][0], 3), "backward_ms": round(st["phase_ms"][1], 3),
                          "step_variants": st["step_variant"], "launches_per_call": st["kernel_launches"],
                          "history_steps": st["history_steps"], "workspace_gb": round(st["workspace_bytes"] / 1e9, 2),
                          "gcell_per_s": round(2 * U / ms / 1e6, 3)}), flush=True)


def run_born_only(args, dist, ctx, case, geom, v0, d_obs):
    """Born demigration alone (born_demig), for kernel profiling."""
    import torch

    import synth

    dv = torch.tensor(synth.smooth_random_field(case.nz, case.nx, 5) * 100.0, dtype=torch.float32,
                      device=v0.device)
    d = ctx.new_data(geom)
    ctx.set_timing(True)
    for _ in range(args.warmup):
        ctx.born_demig(v0, geom, dv, out=d)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        ctx.born_demig(v0, geom, dv, out=d)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    st = ctx.stats()
    U = case.geom.cell_updates(case.nz, case.nb)
    if dist.rank == 0:
        print(json.dumps({"only": "born", "workload": case.name, "ms_per_call": round(ms, 3),
                          "born_ms": round(st["phase_ms"][2], 3), "step_variants": st["step_variant"],
                          "launches_per_call": st["kernel_launches"], "gcell_per_s": round(2 * U / ms / 1e6, 3),
                          "GBps_at_28B_per_cell_step": round(BORN_BYTES_PER_CELL_STEP * U / ms / 1e6, 1)}),
              flush=True)


def main():
    args = parse()
    dist = Dist()
    if args.impl == "reference":
        run_reference(args, dist)
        dist.close()
        return
    import numpy as np
    import torch

    from paper_2403_17518_gb300 import build
    from paper_2403_17518_gb300.ops import Context, GeomArgs

    torch.cuda.set_device(dist.local)
    build()
    prof = args.only in ("fwd", "grad", "born")
    case = make_case(args.workload, args.shots if prof else 0, args.nt if prof else 0)
    if args.only == "nn":
        run_network_only(args, dist, case)
        dist.close()
        return
    dev = torch.device("cuda", dist.local)
    ctx = Context(case.nz, case.nx, case.h, case.dt, case.nb, device=dist.local)
    geom = GeomArgs(case.geom)
    v_true = torch.tensor(case.v_true, dtype=torch.float32, device=dev)
    v0 = torch.tensor(case.v_init, dtype=torch.float32, device=dev)
    d_obs = ctx.model_shots(v_true, geom)
    setup_launches = ctx.stats()["kernel_launches"]
    if args.only in ("fwd", "grad", "born"):
        {"fwd": run_forward_only, "grad": run_gradient_only, "born": run_born_only}[args.only](
            args, dist, ctx, case, geom, v0, d_obs)
        ctx.close()
        dist.close()
        return
    grad = ctx.new_model()
    dm1 = ctx.new_model()
    direction = ctx.new_model()
    v1 = ctx.new_model()
    d_born = ctx.new_data(geom)
    ctx.set_timing(True)
    ctx.set_reuse(args.reuse)
    performed = [0]
    alpha = 0.01 * float(np.mean(case.v_init))
    # Cold start of the network (first FWI iteration), outside the timed region.
    ctx.fwi_gradient(v0, geom, d_obs, grad=grad)
    setup_launches += ctx.stats()["kernel_launches"]
    ctx.born_demig(v0, geom, grad, out=d_born)
    setup_launches += ctx.stats()["kernel_launches"]
    ctx.rtm_mig(v0, geom, d_born, out=dm1)
    setup_launches += ctx.stats()["kernel_launches"]
    ctx.deblur_train(dm1, grad, warm_start=False, epochs=args.cold_epochs, **NET)
    setup_launches += ctx.stats()["kernel_launches"]
    nn_ev = []
    # Library phases (CUDA events on the call's stream): 0 forward passes,
    # 1 backward sweeps, 2 Born joint passes.
    ph = [{"ms": 0.0, "launches": 0, "cells": 0} for _ in range(3)]
    hist = {"cells": 0, "steps": 0, "fwd_steps": 0}
    nt_max = int(max(case.geom.nt))
    launches = [0]

    def step(collect=False):
        J, _ = ctx.fwi_gradient(v0, geom, d_obs, grad=grad)
        stats = [ctx.stats()]
        ctx.born_demig(v0, geom, grad, out=d_born)
        stats.append(ctx.stats())
        ctx.rtm_mig(v0, geom, d_born, out=dm1)
        stats.append(ctx.stats())
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        ctx.deblur_train(dm1, grad, warm_start=True, epochs=WARM_EPOCHS, **NET)
        launches[0] += ctx.stats()["kernel_launches"]
        ctx.deblur_apply(grad, out=direction)
        launches[0] += ctx.stats()["kernel_launches"]
        ev1.record()
        if collect:
            nn_ev.append((ev0, ev1))
        ctx.fwi_update(v0, direction, alpha, 1500.0, 4500.0, 5, out=v1)
        launches[0] += ctx.stats()["kernel_launches"]
        for st in stats:
            launches[0] += st["kernel_launches"]
            if collect:
                performed[0] += st["cell_updates"]
                for k in range(3):
                    ph[k]["ms"] += st["phase_ms"][k]
                    ph[k]["launches"] += st["phase_launches"][k]
                    ph[k]["cells"] += st["phase_cells"][k]
                hist["cells"] += st["history_cells"]
                hist["steps"] = max(hist["steps"], st["history_steps"])
                hist["fwd_steps"] += nt_max if st["phase_launches"][0] > 0 else 0
        return J

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches_before = setup_launches + launches[0]
    launches[0] = 0
    clocks = ClockSampler(dist.local) if dist.rank == 0 else None
    if clocks:
        clocks.start()
    dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step(collect=True)
    e1.record()
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop() if clocks else None
    ms = e0.elapsed_time(e1)
    ms_max = dist.max(ms)
    cells_step = algorithmic_cells(case)
    value = dist.world * cells_step * args.steps / (ms_max / 1e3) / 1e9

    # Rooflines of the stencil kernels: each library phase's algorithmic
    # bytes over its CUDA-event time inside the timed region.
    peak, peak_kind = peaks()
    variants = ctx.stats()["step_variant"]
    fwd_pair = hist["fwd_steps"] / max(ph[0]["launches"], 1) > 1.5  # two time steps per launch
    kernels = [
        ("fwd_pair_kernel" if fwd_pair else forward_kernel(variants[0]),
         "forward passes of fwi_gradient and rtm_mig, storing the a^n history",
         FWD_BYTES_PER_CELL * ph[0]["cells"] + HIST_BYTES_PER_CELL * hist["cells"],
         f"{FWD_BYTES_PER_CELL} B per update (read u^n, u^(n-1), write u^(n+1)) + {HIST_BYTES_PER_CELL} B per "
         f"update that stores a^n"),
        ("adj_pair_kernel" if fwd_pair else ("adj_tma_kernel" if variants[2] >= 3 else "adj_step_kernel"),
         "backward sweeps of fwi_gradient and rtm_mig (adjoint steps with imaging, a^n read from the history)",
         ADJ_BYTES_PER_CELL * ph[1]["cells"],
         f"{ADJ_BYTES_PER_CELL} B per update (12 B for the adjoint field + 4 B to read a^n)"),
        ("born_tma_kernel" if variants[3] >= 3 else "born_step_kernel",
         "Born joint passes of born_demig (background and scattered fields)",
         BORN_BYTES_PER_CELL_STEP * ph[2]["cells"] // 2,
         f"{BORN_BYTES_PER_CELL_STEP} B per cell-step (two fields, 24 B, + 4 B for dv)"),
    ]
    rooflines = []
    for k, (kern, what, alg, rule) in enumerate(kernels):
        p_ms, nl, cells = ph[k]["ms"], max(ph[k]["launches"], 1), ph[k]["cells"]
        ach = alg / (p_ms / 1e3) / 1e9 if p_ms > 0 else None
        traffic = profiled_traffic(kern, cells / nl)
        rooflines.append({
            "kernel": f"{kern} ({what})", "bound": "hbm", "achieved": round(ach, 2) if ach else None, "peak": peak,
            "unit": "GB/s", "frac": round(ach / peak, 4) if ach else None,
            "traffic": round(traffic) if traffic else None,
            "algorithmic_bytes_per_launch": round(alg / nl), "bytes_rule": rule,
            "avg_launch_ms": round(p_ms / nl, 6), "launches_per_step": nl // max(args.steps, 1),
            "ms_per_step": round(p_ms / max(args.steps, 1), 2),
            "gcell_per_s": round(cells / (p_ms / 1e3) / 1e9, 2) if p_ms > 0 else None,
            "peak_kind": f"{peak_kind} (hbm_gbs)"})
    if ph[0]["ms"] > 0:
        summed = SUMMED_FWD_BYTES_PER_CELL * ph[0]["cells"] + HIST_BYTES_PER_CELL * hist["cells"]
        rooflines[0]["summed_form_GBps"] = round(summed / (ph[0]["ms"] / 1e3) / 1e9, 2)
    dominant = max(range(3), key=lambda k: ph[k]["ms"])

    # End to end through the public API with host buffers.
    e2e = None
    if not args.no_e2e:
        h_v0 = torch.tensor(case.v_init, dtype=torch.float32).pin_memory()
        h_dobs = d_obs.cpu().pin_memory()
        h_grad = torch.empty((case.nz, case.nx), dtype=torch.float32).pin_memory()
        h_dm1 = torch.empty((case.nz, case.nx), dtype=torch.float32).pin_memory()
        dv0 = torch.empty_like(v0)
        ddobs = torch.empty_like(d_obs)

        def e2e_step():
            dv0.copy_(h_v0, non_blocking=True)
            ddobs.copy_(h_dobs, non_blocking=True)
            ctx.fwi_gradient(dv0, geom, ddobs, grad=grad)
            ctx.born_demig(dv0, geom, grad, out=d_born)
            ctx.rtm_mig(dv0, geom, d_born, out=dm1)
            ctx.deblur_train(dm1, grad, warm_start=True, epochs=WARM_EPOCHS, **NET)
            ctx.deblur_apply(grad, out=direction)
            ctx.fwi_update(dv0, direction, alpha, 1500.0, 4500.0, 5, out=v1)
            h_grad.copy_(v1, non_blocking=True)
            h_dm1.copy_(direction, non_blocking=True)
            torch.cuda.synchronize()

        e2e_step()
        dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        el = dist.max(time.perf_counter() - t0)
        e2e = {"value": round(dist.world * cells_step * args.e2e_steps / el / 1e9, 4), "unit": UNIT,
               "h2d_bytes_per_step": int(h_v0.numel() * 4 + h_dobs.numel() * 4),
               "d2h_bytes_per_step": int(h_grad.numel() * 4 + h_dm1.numel() * 4 + 8)}

    nn_ms = sum(a.elapsed_time(b) for a, b in nn_ev) / max(len(nn_ev), 1)
    npatch = n_patches(case.nz, NET["patch"], NET["stride"]) * n_patches(case.nx, NET["patch"], NET["stride"])
    f_patch = conv_flops(NET["base_channels"], NET["levels"], NET["patch"], NET["patch"])
    f_apply = conv_flops(NET["base_channels"], NET["levels"], case.nz, case.nx)
    nn_flops = WARM_EPOCHS * npatch * 3 * f_patch + f_apply  # training = forward + two gradient GEMMs
    bf16_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops_sustained"] \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1700.0
    nn_tflops = nn_flops / (nn_ms / 1e3) / 1e12 if nn_ms > 0 else None

    cpu = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        n_sh = min(cpu_cores(), case.geom.n_shots)
        val, sec, used, sample = oracle_measure(case, n_sh, 300, 1, 0)
        cpu = {"value": round(val, 6), "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample}

    if dist.rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(case, args),
            # The stencil kernel that takes the most time of the step.
            "roofline": rooflines[dominant],
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches[0]),
            "launches_before_timed_region": int(launches_before),
            "step_variants": ctx.stats()["step_variant"],
            "time_block_depth": {"forward": ctx.stats()["time_block"][0], "adjoint": ctx.stats()["time_block"][1]},
            "reuse": bool(args.reuse),
            "performed_cell_updates_per_step": int(performed[0] // max(args.steps, 1)),
            "history_steps": {"stored": hist["steps"], "of": nt_max,
                              "workspace_gb": round(ctx.stats()["workspace_bytes"] / 1e9, 2)},
            "phase_ms_per_step": {"forward_ms": round(ph[0]["ms"] / args.steps, 2),
                                  "backward_ms": round(ph[1]["ms"] / args.steps, 2),
                                  "born_ms": round(ph[2]["ms"] / args.steps, 2), "network_ms": round(nn_ms, 2)},
            "rooflines_stencil": rooflines,
            "roofline_network": {
                "kernel": "U-Net training (20 warm epochs, 108 patches, batch 32) + full-image apply",
                "bound": "tensor", "achieved": round(nn_tflops, 2) if nn_tflops else None, "peak": bf16_peak,
                "unit": "TFLOP/s", "frac": round(nn_tflops / bf16_peak, 4) if nn_tflops else None,
                "flops_per_step": nn_flops, "peak_kind": "measured (bf16_tflops_sustained)",
            },
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    dist.close()


if __name__ == "__main__":
    main()
