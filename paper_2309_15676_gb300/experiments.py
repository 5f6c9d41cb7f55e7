"""Statistical validation of the meta-estimator along prescribed parameter trajectories (Sec. 6,
"variance reduction without lag" and "approximation accuracy").

The parameters of the box scene (config 1: 64x64 image, 32x32 RGB albedo, depth 3, 1 FD + 1
proportional spp) move from the initial to the target texture along a fixed schedule, without an
optimiser: after every update step the library's parameters are replaced by the schedule's next
point (mer_params_force), so the gradient samples <F_i>, <dF_i>, the meta-estimate <F_i>_M and its
variance approximations are those of the method along that path. Many independent runs (problems
with their own Philox keys, batched in one context) give the ground truth: the expected gradient
and the actual variances are the across-run mean and variance. Adam's bias-corrected moments of
the same samples (beta1 = 0.9, beta2 = 0.999) are the comparison.

Everything the method computes runs in the library's kernels; this module only moves the
parameters along the schedule and accumulates across-run sums of what the kernels produced.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import synth
from .api import Context, HyperParams

_STATS = ("F", "F2", "D", "D2", "M", "M2", "VM", "A", "A2", "AV", "VF", "VD", "AL")


def _schedule(kind: str, iters: int, tau: float):
    """Fraction of the way from the initial to the target texture at iteration k = 0..iters."""
    k = np.arange(iters + 1, dtype=np.float64)
    if kind == "linear":
        return k / iters
    if kind == "exponential":
        return (1.0 - np.exp(-k / tau)) / (1.0 - math.exp(-iters / tau))
    raise ValueError(kind)


def trajectory_study(runs: int = 1000, iters: int = 100, schedule: str = "linear", tau: float = 15.0,
                     per_ctx: int = 250, beta1: float = 0.9, beta2: float = 0.999, device: int = 0) -> dict:
    w = synth.workload_box()
    dev = torch.device("cuda", device)
    init = torch.from_numpy(w.init_tex.astype(np.float32)).to(dev)
    tgt_tex = torch.from_numpy(w.target_tex.astype(np.float32)).to(dev)
    frac = _schedule(schedule, iters, tau)
    path = [init + (tgt_tex - init) * float(f) for f in frac]
    step2 = [0.0] + [float(((path[k].double() - path[k - 1].double()) ** 2).sum()) for k in range(1, iters + 1)]
    c0 = Context(device)
    p0 = c0.add_scene(w.scene, HyperParams())
    target = c0.render(p0, tgt_tex, spp=256, stream=4, iteration=0).clone()
    c0.close()
    n_par = init.numel()
    acc = {s: torch.zeros(iters, n_par, dtype=torch.float64, device=dev) for s in _STATS}
    alpha_hist = torch.zeros(iters, 10, dtype=torch.float64, device=dev)
    done = 0
    while done < runs:
        nb = min(per_ctx, runs - done)
        ctx = Context(device)
        ids = []
        for r in range(nb):
            sc = dict(w.scene)
            sc["key_id"] = 1 + done + r
            pid = ctx.add_scene(sc, HyperParams())
            ctx.set_target(pid, target)
            ctx.set_params(pid, init)
            ids.append(pid)
        am = torch.zeros(nb, n_par, dtype=torch.float64, device=dev)
        av = torch.zeros_like(am)
        for k in range(iters):
            ctx.gradient_step()
            gr = [ctx.grads(p) for p in ids]
            F = torch.stack([x[0].reshape(-1) for x in gr]).double()
            D = torch.stack([x[1].reshape(-1) for x in gr]).double()
            ctx.update_step()
            st = [ctx.state(p) for p in ids]
            M = torch.stack([s["mean"].reshape(-1) for s in st]).double()
            VM = torch.stack([s["var"].reshape(-1) for s in st]).double()
            VF = torch.stack([s["m2f"].reshape(-1) for s in st]).double()
            VD = torch.stack([s["m2d"].reshape(-1) for s in st]).double() * step2[k]
            AL = torch.stack([s["alpha_prev"].reshape(-1) for s in st]).double()
            am = beta1 * am + (1 - beta1) * F
            av = beta2 * av + (1 - beta2) * F * F
            A = am / (1 - beta1 ** (k + 1))
            AV = av / (1 - beta2 ** (k + 1))
            for name, x in (("F", F), ("D", D), ("M", M), ("A", A)):
                acc[name][k] += x.sum(0)
                acc[name + "2"][k] += (x * x).sum(0)
            for name, x in (("VM", VM), ("AV", AV), ("VF", VF), ("VD", VD), ("AL", AL)):
                acc[name][k] += x.sum(0)
            alpha_hist[k] += torch.histc(AL.clamp(0, 1 - 1e-9).flatten().float(), bins=10, min=0, max=1).double()
            if k < iters - 1:
                for p in ids:
                    ctx.force_params(p, path[k + 1])
        ctx.close()
        done += nb
    return _summarise(acc, alpha_hist, runs, iters, schedule, step2)


def _summarise(acc, alpha_hist, runs, iters, schedule, step2) -> dict:
    n = float(runs)
    mean = {s: (acc[s] / n).cpu().numpy() for s in _STATS}
    var = lambda a, a2: np.maximum(mean[a2] - mean[a] ** 2, 0.0) * n / (n - 1)
    g = mean["F"]                       # expected gradient per iteration and texel
    var_f, var_d = var("F", "F2"), var("D", "D2")
    var_m, var_a = var("M", "M2"), var("A", "A2")
    # texels that receive gradient; iterations past the first ten (start-up)
    live = var_f[10:].mean(0) > 1e-4 * var_f[10:].mean(0).max()
    ks = slice(10, iters)
    sd_f = np.sqrt(var_f[ks][:, live])
    rel = lambda x: float(np.median(x))
    out = {
        "schedule": schedule, "runs": runs, "iterations": iters, "texels": int(live.sum()),
        # lag: |E[estimate] - E[F]| in units of the sample standard deviation
        "lag_meta": rel(np.abs(mean["M"][ks][:, live] - g[ks][:, live]) / sd_f),
        "lag_adam": rel(np.abs(mean["A"][ks][:, live] - g[ks][:, live]) / sd_f),
        # actual variance of the estimate relative to one sample's variance
        "var_ratio_meta": rel(var_m[ks][:, live] / var_f[ks][:, live]),
        "var_ratio_adam": rel(var_a[ks][:, live] / var_f[ks][:, live]),
        # actual over predicted standard deviation of <F>_M (Sec. 6: within 0.5 to 2)
        "sd_actual_over_predicted_meta": rel(np.sqrt(var_m[ks][:, live] / np.maximum(mean["VM"][ks][:, live], 1e-300))),
        "frac_within_0p5_2": float(np.mean(np.abs(np.log2(np.sqrt(
            var_m[ks][:, live] / np.maximum(mean["VM"][ks][:, live], 1e-300)))) <= 1.0)),
        # the variance approximations against their ground truth
        "varF_estimate_over_true": rel(mean["VF"][ks][:, live] / var_f[ks][:, live]),
        "varD_estimate_over_true": rel(mean["VD"][ks][:, live] / np.maximum(var_d[ks][:, live], 1e-300)),
        "alpha_mean_by_iteration": [float(x) for x in mean["AL"][:, live].mean(1)[::10]],
        "alpha_histogram_last_iteration": [float(x) for x in (alpha_hist[-1] / alpha_hist[-1].sum()).cpu().numpy()],
    }
    # three texels by actual gradient variance: the noisiest, the 75th percentile, the median
    vf = var_f[ks].mean(0)
    order = np.argsort(np.where(live, vf, -1.0))[::-1][: int(live.sum())]
    picks = {"noisiest": int(order[0]), "p75": int(order[len(order) // 4]), "median": int(order[len(order) // 2])}
    curves = {}
    for name, e in picks.items():
        curves[name] = {
            "texel": e,
            "iteration": list(range(0, iters, 10)),
            "true_gradient": [float(x) for x in g[::10, e]],
            "meta_mean": [float(x) for x in mean["M"][::10, e]],
            "meta_sd_actual": [float(x) for x in np.sqrt(var_m[::10, e])],
            "meta_sd_predicted": [float(x) for x in np.sqrt(mean["VM"][::10, e])],
            "adam_mean": [float(x) for x in mean["A"][::10, e]],
            "adam_sd_actual": [float(x) for x in np.sqrt(var_a[::10, e])],
            "sample_sd": [float(x) for x in np.sqrt(var_f[::10, e])],
        }
    out["texel_curves"] = curves
    return out


# ------------------------------------------------------------------------------------------
# Optimisation runs: time to a loss threshold, meta-estimator against plain Adam
# ------------------------------------------------------------------------------------------
def _eval_loss(ctx, pid, target, spp=64):
    img = ctx.render(pid, None, spp=spp, stream=5, iteration=0)
    return float(((img - target) ** 2).mean())


def _diagnose(ctx, pid) -> dict:
    """The meta-estimator's state over the texels that received gradient (Var[<F>] > 0): histogram
    of alpha (10 bins on [0, 1]), its mean, and Var[<dF>] / Var[<F>] with Var[<dF>] taken as
    Var_D times the squared norm of the last step (Eq. vardiff)."""
    st = ctx.state(pid)
    n2 = ctx.stats(pid)["dpi_norm2"]
    m2f = st["m2f"].double().flatten()
    live = m2f > 0
    a = st["alpha_prev"].double().flatten()[live].clamp(0.0, 1.0 - 1e-12)
    ratio = (st["m2d"].double().flatten()[live] * n2) / m2f[live]
    hist = torch.histc(a.float(), bins=10, min=0.0, max=1.0)
    return {"texels": int(live.sum()), "alpha_mean": float(a.mean()) if a.numel() else None,
            "alpha_hist": [float(x) for x in (hist / max(float(hist.sum()), 1.0)).cpu()],
            "varD_over_varF_median": float(ratio.median()) if ratio.numel() else None,
            "varD_over_varF_mean": float(ratio.mean()) if ratio.numel() else None}


def optimise_run(scene: dict, init_tex, target_img, mode: int, spp_prop: int, spp_fd: int, lr: float,
                 max_iters: int, frac: float, flags: int = 0, precond_lambda: float = 0.0, beta_d: float = 0.9,
                 diag_at=(), device: int = 0) -> dict:
    """One optimisation run of a single problem with graph-launched iterations: iterations and GPU
    time (iterations only, evaluation excluded) until the 64-spp eval loss (stream EVAL) drops below
    `frac` and below 10% of its iteration-0 value; evaluated every 2 iterations for the first 50,
    then every 10. `diag_at`: iteration counts at which the meta-estimator's state is summarised
    (_diagnose); they must fall on the evaluation schedule."""
    from .api import MODE_META
    sc = dict(scene)
    sc["spp_prop"], sc["spp_fd"] = spp_prop, spp_fd
    ctx = Context(device)
    pid = ctx.add_scene(sc, HyperParams(mode=mode, lr=lr, flags=flags, precond_lambda=precond_lambda,
                                        beta_d=beta_d))
    ctx.set_target(pid, target_img)
    ctx.set_params(pid, init_tex)
    # capture the iteration graph outside the timed region: one iteration, then rewind the state
    blob = ctx.checkpoint_save()
    ctx.iterate(1, use_graph=True)
    ctx.checkpoint_load(blob)
    torch.cuda.synchronize()
    l0 = _eval_loss(ctx, pid, target_img)
    thr = frac * l0
    gpu_ms, it, reached, reached_ms, last, lmin = 0.0, 0, None, None, l0, l0
    r10, r10_ms = None, None
    diag = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    while it < max_iters:
        k = 2 if it < 50 else 10
        e0.record()
        ctx.iterate(k, use_graph=True)
        e1.record()
        e1.synchronize()
        gpu_ms += e0.elapsed_time(e1)
        it += k
        last = _eval_loss(ctx, pid, target_img)
        lmin = min(lmin, last)
        if reached is None and last <= thr:
            reached, reached_ms = it, gpu_ms
        if r10 is None and last <= 0.1 * l0:
            r10, r10_ms = it, gpu_ms
        if it in diag_at and mode == MODE_META:
            diag[it] = _diagnose(ctx, pid)
    ctx.close()
    out = {"lr": lr, "iters": reached, "gpu_s": reached_ms / 1e3 if reached else None, "loss0": l0,
           "iters_10pct": r10, "gpu_s_10pct": r10_ms / 1e3 if r10 else None,
           "final_loss_ratio": last / l0, "min_loss_ratio": lmin / l0, "iters_run": it,
           "gpu_s_total": gpu_ms / 1e3}
    if diag:
        out["diagnostics"] = diag
    return out


def pinned_spiral(metal: float = 0.5, rough: float = 0.35, **kw):
    """The spiral workload with metalness and roughness the same constant in the initial and the
    target texture and held there (clamp range of a single value): only the base colour is
    optimised, and since neither the lobe choice nor the GGX sample depends on base colour, an FD
    pair's two branches follow the same path at every bounce."""
    w = synth.workload_spiral(**kw)
    sc = dict(w.scene)
    lo, hi = list(sc["clamp_lo"]), list(sc["clamp_hi"])
    lo[3], hi[3], lo[4], hi[4] = metal, metal, rough, rough
    sc["clamp_lo"], sc["clamp_hi"] = lo, hi
    init, tgt = w.init_tex.copy(), w.target_tex.copy()
    for t in (init, tgt):
        t[..., 3] = metal
        t[..., 4] = rough
    return sc, init, tgt


def meta_vs_adam_study(iters: int = 300, lrs=(0.003, 0.01, 0.03, 0.1), beta_ds=(0.5, 0.9, 0.99),
                       frac: float = 0.05, diag_at=(10, 50, 100, 200), device: int = 0) -> dict:
    """Where the meta-estimator's advantage over Adam at equal samples per iteration comes from
    (Sec. 1 and Sec. 6: 1 FD + 2 proportional spp against Adam's fresh samples), on the 256^2 spiral
    (depth 5) in two forms: every texture channel free, and metalness / roughness pinned so that FP
    pairs stay coincident. Per form and method, the best learning rate of the grid by GPU time to
    `frac` of the initial loss (else by the lowest loss), with the meta-estimator's alpha histogram
    and Var[<dF>] / Var[<F>] at `diag_at`; the meta-estimator for every beta_D of `beta_ds`, with
    FD pairs by random-number replay and (beta_D 0.9) with the pi_{i-1} branch on the pi_i path."""
    from .api import META_FD_SHARED_PATH, MODE_ADAM, MODE_META
    w = synth.workload_spiral()
    forms = {"free": (dict(w.scene), w.init_tex, w.target_tex), "pinned": pinned_spiral()}
    out = {"workload": "spiral256: 256^2, 8,192 triangles, 256^2 x 5 textures, depth 5",
           "threshold": f"{frac:.0%} of the iteration-0 64-spp eval loss", "lr_grid": list(lrs),
           "iterations": iters, "forms": {}}
    for name, (sc, init, tgt) in forms.items():
        c = Context(device)
        p = c.add_scene(sc, HyperParams())
        target = c.render(p, torch.from_numpy(np.ascontiguousarray(tgt, np.float32)).cuda(device), spp=256,
                          stream=4, iteration=0).clone()
        c.close()
        methods = [(f"meta_betaD_{bd}", MODE_META, 2, 1, 0, bd) for bd in beta_ds]
        methods += [("meta_shared_path", MODE_META, 2, 1, META_FD_SHARED_PATH, 0.9), ("adam", MODE_ADAM, 3, 0, 0, 0.9)]
        res = {}
        for mname, mode, sp, sf, flags, bd in methods:
            best = None
            for lr in lrs:
                r = optimise_run(sc, init, target, mode, sp, sf, lr, iters, frac, flags=flags, beta_d=bd,
                                 diag_at=diag_at, device=device)
                key = (0 if r["iters"] else 1, r["gpu_s"] if r["iters"] else r["min_loss_ratio"])
                if best is None or key < best[0]:
                    best = (key, r)
            res[mname] = best[1]
        out["forms"][name] = res
    return out
