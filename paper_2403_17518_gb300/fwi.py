"""FWI driver: plain steepest descent vs deblurred-gradient FWI (Section 2.3).

Each iteration of either arm computes the misfit and gradient (Eq. 2, Eq.
13).  The deblurred arm then forms the doubly migrated image of the gradient
(Eq. 15), trains the network to map it back to the gradient (warm-started
from the previous iteration, re-initialised at each new frequency band) and
applies the network to the gradient to get the direction (Section 2.3.1).
Both arms take the same step rule: the direction normalised to unit max, a
two-trial parabolic line search on the misfit, velocity clamped to the model
range, the top rows muted.  GPU time is the sum of CUDA-event intervals
around every call of an iteration (line-search forwards and training
included), so the arms are compared at equal GPU-seconds.

All arithmetic runs in libdhfwi.so; this module only sequences the calls and
low-pass filters the observed data and the wavelet per band on the host.
"""
from __future__ import annotations

import argparse
import copy
import json
import math
import time

import numpy as np
import torch

from .ops import Context, GeomArgs


def lowpass(x: np.ndarray, dt: float, fc: float, axis: int = -1) -> np.ndarray:
    """Zero-phase low-pass: unit gain below fc, cosine taper to 0 at 1.25 fc."""
    n = x.shape[axis]
    nf = 1 << int(math.ceil(math.log2(2 * n)))
    X = np.fft.rfft(x, nf, axis=axis)
    f = np.fft.rfftfreq(nf, dt)
    H = np.where(f <= fc, 1.0, np.where(f >= 1.25 * fc, 0.0, 0.5 * (1 + np.cos(np.pi * (f - fc) / (0.25 * fc)))))
    shape = [1] * X.ndim
    shape[axis] = -1
    y = np.fft.irfft(X * H.reshape(shape), nf, axis=axis)
    return np.take(y, np.arange(n), axis=axis)


def band_data(d_obs: np.ndarray, geom, dt: float, fc: float) -> np.ndarray:
    """Low-pass each shot record [nt_s][nrec_s] along time."""
    out = np.empty_like(d_obs)
    off = geom.data_offsets()
    for s in range(geom.n_shots):
        nr = geom.nrec(s)
        blk = d_obs[off[s]:off[s + 1]].reshape(int(geom.nt[s]), nr)
        out[off[s]:off[s + 1]] = lowpass(blk, dt, fc, axis=0).ravel()
    return out


class Timer:
    """Sums CUDA-event intervals on the current stream."""

    def __init__(self):
        self.pairs = []

    def __enter__(self):
        self.e0 = torch.cuda.Event(enable_timing=True)
        self.e1 = torch.cuda.Event(enable_timing=True)
        self.e0.record()
        return self

    def __exit__(self, *a):
        self.e1.record()
        self.pairs.append((self.e0, self.e1))

    def seconds(self) -> float:
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in self.pairs) / 1e3


def model_rms(v: torch.Tensor, v_true: torch.Tensor) -> float:
    return float(torch.sqrt(torch.mean((v - v_true) ** 2)).item())


def parabolic_alpha(J0: float, J1: float, J2: float, a1: float):
    """Step from the misfits at 0, a1 and 2 a1 (the parabola through the three
    points, minimised on [0, 4 a1]); returns (alpha, whether a trial lowered
    the misfit).  No improvement: 0; no minimiser, or a clamped vertex at 0:
    the better trial."""
    curv = (J2 - 2 * J1 + J0) / (2 * a1 * a1)
    slope = (4 * J1 - 3 * J0 - J2) / (2 * a1)
    if curv > 0:
        a_best = -slope / (2 * curv)
    else:
        a_best = 2 * a1 if J2 < J1 else a1
    a_best = min(max(a_best, 0.0), 4 * a1)
    improved = min(J1, J2) < J0
    if improved and a_best == 0.0:
        a_best = a1 if J1 <= J2 else 2 * a1
    if not improved:
        a_best = 0.0
    return a_best, improved


BACKTRACK = 8.0  # the second round of trials is this many times shorter


def line_search(ctx, v, dirn, ga, d_obs, d_try, trial, J0, a1, vmin, vmax, mute_rows):
    """Two-trial parabolic line search on the misfit along -dirn, with one
    backtracking round: when neither a1 nor 2 a1 lowers the misfit, the
    trials a1 / BACKTRACK and 2 a1 / BACKTRACK are tried.  Returns (alpha,
    whether a trial lowered the misfit, forward solves spent)."""
    solves = 0
    for b1 in (a1, a1 / BACKTRACK):
        Js = []
        for a in (b1, 2 * b1):
            ctx.fwi_update(v, dirn, a, vmin, vmax, mute_rows, out=trial)
            ctx.model_shots(trial, ga, out=d_try)
            Js.append(ctx.data_misfit(d_try, d_obs))
        solves += 2
        alpha, ok = parabolic_alpha(J0, Js[0], Js[1], b1)
        if ok:
            return alpha, True, solves
    return 0.0, False, solves


class BandData:
    """Observed data of the true model and their band-limited versions (the
    wavelet low-passed identically), computed once and shared by the arms."""

    def __init__(self, ctx: Context, case):
        v_true = torch.tensor(case.v_true, dtype=torch.float32, device=ctx.device)
        self.d_full = ctx.model_shots(v_true, case.geom).cpu().numpy()
        self.case = case
        self.bands = {}

    def get(self, fc: float):
        if fc not in self.bands:
            g = copy.deepcopy(self.case.geom)
            g.wavelet = lowpass(np.asarray(g.wavelet, dtype=np.float64), self.case.dt, fc)
            d = band_data(self.d_full, self.case.geom, self.case.dt, fc).astype(np.float32)
            self.bands[fc] = (GeomArgs(g), d)
        return self.bands[fc]


def run_arm(ctx: Context, case, mode: str, bands, iters: int, net_cfg: dict, cold_epochs: int, warm_epochs: int,
            vmin: float, vmax: float, mute_rows: int = 5, log=None, hybrid_iters: int = 0, data: BandData = None,
            timer=None):
    """mode: "plain" (gradient, parabolic line search), "bb" (gradient with
    the Barzilai-Borwein short step of Eq. 17, the paper's baseline; the
    first iteration of each band takes the line search), "deblur" (network
    direction every iteration) or "hybrid" (network direction for the first
    hybrid_iters iterations of the run, the gradient after: the Hessian
    approximation steers the early iterations, then conventional FWI
    continues, Section 4)."""
    dev = ctx.device
    v_true = torch.tensor(case.v_true, dtype=torch.float32, device=dev)
    v = torch.tensor(case.v_init, dtype=torch.float32, device=dev)
    data = data if data is not None else BandData(ctx, case)
    hist = [{"band": None, "iter": 0, "gpu_s": 0.0, "solves": 0, "model_rms": model_rms(v, v_true), "misfit": None}]
    solves = 0
    timer = timer if timer is not None else Timer()
    grad = ctx.new_model()
    direction = ctx.new_model()
    dm1 = ctx.new_model()
    trial = ctx.new_model()
    done_iters = 0
    v_prev, g_prev = ctx.new_model(), ctx.new_model()
    for fc in bands:
        trained_in_band = False  # the network restarts from scratch in each band (Section 4)
        have_prev = False  # BB needs two models and gradients of the same band
        ga, d_band = data.get(fc)
        d_obs = torch.tensor(d_band, dtype=torch.float32, device=dev)
        d_born = ctx.new_data(ga)
        d_try = ctx.new_data(ga)
        for it in range(iters):
            use_net = mode == "deblur" or (mode == "hybrid" and done_iters < hybrid_iters)
            with timer:
                J0, _ = ctx.fwi_gradient(v, ga, d_obs, grad=grad)
                a1 = 0.01 * float(np.mean(case.v_init))
                fallback = False
                stalled = False
                loss = None
                solves += 2  # forward + adjoint of the gradient (checkpoint recomputation not counted)
                if use_net:
                    solves += 2  # Born modelling + its adjoint (Section 3.1: two more solves)
                    ctx.born_demig(v, ga, grad, out=d_born)
                    ctx.rtm_mig(v, ga, d_born, out=dm1)
                    warm = it > 0 and trained_in_band
                    h = ctx.deblur_train(dm1, grad, warm_start=warm, epochs=warm_epochs if warm else cold_epochs,
                                         mute_rows=mute_rows, warmup_frac=0.1, **net_cfg)
                    trained_in_band = True
                    loss = [float(h[0]), float(h[-1])]
                    ctx.deblur_apply(grad, out=direction)
                    a_best, ok, ns = line_search(ctx, v, direction, ga, d_obs, d_try, trial, J0, a1, vmin, vmax,
                                                 mute_rows)
                    solves += ns
                    dirn = direction
                    if not ok:
                        # The plain gradient is the fallback when the network's
                        # direction does not lower the misfit.
                        fallback = True
                        dirn = grad
                        a_best, ok, ns = line_search(ctx, v, grad, ga, d_obs, d_try, trial, J0, a1, vmin, vmax,
                                                     mute_rows)
                        solves += ns
                    stalled = not ok
                else:
                    dirn = grad
                    alpha_bb = 0.0
                    if mode == "bb" and have_prev:
                        # Eq. 17: x_{k+1} = x_k - alpha g_k; fwi_update divides by
                        # max|g_k|.  Safeguard: the largest model change is
                        # bounded as in the line search (4 a1).
                        alpha_bb, gmax = ctx.bb_step(v, v_prev, grad, g_prev, mute_rows)
                        a_best = min(alpha_bb * gmax, 4 * a1)
                    if alpha_bb <= 0.0:  # no curvature estimate yet (or a negative one): line search
                        a_best, ok, ns = line_search(ctx, v, grad, ga, d_obs, d_try, trial, J0, a1, vmin, vmax,
                                                     mute_rows)
                        solves += ns
                        stalled = not ok
                if mode == "bb":
                    v_prev.copy_(v)
                    g_prev.copy_(grad)
                    have_prev = True
                ctx.fwi_update(v, dirn, a_best, vmin, vmax, mute_rows, out=v)
            done_iters += 1
            rec = {"band": fc, "iter": it + 1, "gpu_s": timer.seconds(), "solves": solves,
                   "model_rms": model_rms(v, v_true), "net": use_net,
                   "misfit": J0, "alpha": a_best, "fallback": fallback, "train_loss": loss, "stalled": stalled}
            hist.append(rec)
            if log:
                log(mode, rec)
            if stalled:
                # No step lowers the misfit even after backtracking: the next
                # iteration would repeat this one exactly, so the band ends.
                break
    return hist


def error_at(hist, budget: float, key: str = "gpu_s") -> float:
    """Model RMS error reached within `budget` (of GPU seconds or solves)."""
    best = hist[0]["model_rms"]
    for r in hist:
        if r[key] <= budget:
            best = r["model_rms"]
    return best


def summarize(arms: dict):
    """Model RMS error of every arm at the GPU time (and solve count) all
    arms reached."""
    t = min(h[-1]["gpu_s"] for h in arms.values())
    n = min(h[-1]["solves"] for h in arms.values())
    out = {"equal_gpu_s": t, "equal_solves": n, "initial_model_rms": next(iter(arms.values()))[0]["model_rms"]}
    for name, h in arms.items():
        out[f"{name}_model_rms"] = error_at(h, t)
        out[f"{name}_model_rms_at_solves"] = error_at(h, n, "solves")
        out[f"{name}_final"] = h[-1]
    return out


def main():
    import synth

    p = argparse.ArgumentParser(description="plain vs deblurred FWI at equal GPU-seconds")
    p.add_argument("--nz", type=int, default=150)
    p.add_argument("--nx", type=int, default=500)
    p.add_argument("--h", type=float, default=20.0)
    p.add_argument("--dt", type=float, default=2e-3)
    p.add_argument("--shots", type=int, default=25)
    p.add_argument("--nt", type=int, default=1500)
    p.add_argument("--bands", default="3,5")
    p.add_argument("--iters", type=int, default=8, help="iterations per band, deblurred arm")
    p.add_argument("--iters-plain", type=int, default=0, help="iterations per band, plain arm (default --iters)")
    p.add_argument("--mute", type=int, default=5, help="top rows muted in the update and the network input")
    p.add_argument("--lr", type=float, default=2e-4, help="network learning rate")
    p.add_argument("--arms", default="plain,deblur", help="comma list of plain, bb, deblur, hybrid or hybridN")
    p.add_argument("--iters-hybrid", type=int, default=0, help="iterations per band, hybrid arm (default --iters)")
    p.add_argument("--hybrid-net-iters", type=int, default=5,
                   help="hybrid arm: iterations at the start of the run that use the network direction")
    p.add_argument("--case", default="custom", choices=["custom", "config5"],
                   help="config5: the 600 x 2000, 200-shot multiscale workload (dx 10 m, dt 0.8 ms, nt 6000, "
                        "uneven apertures and record lengths); custom: the --nz/--nx/... model")
    p.add_argument("--patch", type=int, default=64, help="network training patch (128 for config 5)")
    p.add_argument("--cold-epochs", type=int, default=200)
    p.add_argument("--warm-epochs", type=int, default=20)
    p.add_argument("--no-reuse", action="store_true", help="propagate the background again in Born and migration")
    p.add_argument("--out", default="")
    a = p.parse_args()
    if a.case == "config5":
        case = synth.config5_case()
        a.nz, a.nx, a.h, a.dt, a.shots, a.nt = case.nz, case.nx, case.h, case.dt, case.geom.n_shots, int(
            case.geom.nt.max())
    else:
        v = synth.layered_fault_model(a.nz, a.nx, a.h, seed=31)
        v0 = synth.smooth_model(v, 10.0)
        wav = synth.ricker(8.0, a.dt, a.nt)
        geom = synth.surface_geometry(a.nx, a.shots, seed=31, nrec_range=(a.nx // 3, a.nx // 2),
                                      nt_range=(int(a.nt * 0.8), a.nt), margin=a.nx // 10, src_lo=10,
                                      src_hi=a.nx - 11, wavelet=wav)
        case = synth.Case(a.nz, a.nx, a.h, a.dt, 20, v, v0, geom, name="fwi-loop")
    ctx = Context(case.nz, case.nx, case.h, case.dt, case.nb)
    # Born and migration at the gradient's model take its stored forward pass.
    ctx.set_reuse(not a.no_reuse)
    net = dict(base_channels=32, levels=4, patch=a.patch, stride=a.patch // 2, batch=32, lr=a.lr, seed=29)
    bands = [float(b) for b in a.bands.split(",")]
    out = {"config": vars(a), "net": net}
    t0 = time.time()
    data = BandData(ctx, case)
    arms = {}
    for name in a.arms.split(","):
        # "hybridN": hybrid arm with the network for the first N iterations.
        mode = "hybrid" if name.startswith("hybrid") else name
        hyb = int(name[6:]) if mode == "hybrid" and name[6:] else a.hybrid_net_iters
        iters = a.iters
        if mode in ("plain", "bb") and a.iters_plain > 0:
            iters = a.iters_plain
        if mode == "hybrid" and a.iters_hybrid > 0:
            iters = a.iters_hybrid
        arms[name] = run_arm(ctx, case, mode, bands, iters, net, a.cold_epochs, a.warm_epochs, 1500.0, 4500.0,
                             mute_rows=a.mute, log=lambda m, r, nm=name: print(nm, json.dumps(r), flush=True),
                             hybrid_iters=hyb, data=data)
        out[name] = arms[name]
        if a.out:  # partial results survive a run cut short
            with open(a.out, "w") as f:
                f.write(json.dumps(dict(out, summary=summarize(arms))))
    out["wall_s"] = time.time() - t0
    out["summary"] = summarize(arms)
    s = json.dumps(out)
    if a.out:
        with open(a.out, "w") as f:
            f.write(s)
    print(s)


if __name__ == "__main__":
    main()
