"""Host-side arithmetic of the trajectory study (the statistics it reports from the kernels'
outputs), fed simulated runs whose answers are known: the schedule's end points and shape, the
across-run mean and variance, the lag in units of the sample deviation, the variance ratios and
the actual-over-predicted deviation."""
import numpy as np
import torch

from paper_2309_15676_gb300 import experiments as ex


def test_schedules():
    lin = ex._schedule("linear", 10, 15.0)
    assert np.allclose(lin, np.arange(11) / 10.0, rtol=0, atol=1e-15)
    e = ex._schedule("exponential", 100, 15.0)
    assert e[0] == 0.0 and abs(e[-1] - 1.0) < 1e-15
    d = np.diff(e)
    assert np.all(d > 0) and np.all(np.diff(d) < 0)       # increasing, concave


def test_summary_statistics_of_simulated_runs():
    rng = np.random.default_rng(3)
    runs, iters, n_par = 4000, 20, 40
    g = rng.normal(size=(iters, n_par))                    # expected gradient per iteration, texel
    s = rng.uniform(0.5, 2.0, n_par)                        # per-texel sample deviation
    acc = {k: np.zeros((iters, n_par)) for k in ex._STATS}
    for _ in range(runs):
        F = g + s * rng.standard_normal((iters, n_par))
        D = 0.1 * s * rng.standard_normal((iters, n_par))
        M = F                                               # an estimate equal to the sample
        A = g                                               # an estimate equal to the expectation
        for name, x in (("F", F), ("D", D), ("M", M), ("A", A)):
            acc[name] += x
            acc[name + "2"] += x * x
        acc["VM"] += s * s                                  # predicted variance of M: exact
        acc["AV"] += 0.0
        acc["VF"] += 4.0 * s * s                            # Var[F] estimate four times too large
        acc["VD"] += (0.1 * s) ** 2
        acc["AL"] += 0.3
    acc = {k: torch.from_numpy(v) for k, v in acc.items()}
    hist = torch.zeros(iters, 10, dtype=torch.float64)
    hist[:, 3] = runs * n_par
    out = ex._summarise(acc, hist, runs, iters, "linear", [0.0] * (iters + 1))
    assert out["texels"] == n_par
    se = 1.0 / np.sqrt(runs)
    # the lag is measured against the across-run mean of F: an estimate equal to F has none, the
    # exact expectation differs from that mean by its sampling error (median |N(0, 1)| ~ 0.67 se)
    assert out["lag_meta"] < 1e-12 and 0.3 * se < out["lag_adam"] < 2 * se
    assert abs(out["var_ratio_meta"] - 1.0) < 0.1 and out["var_ratio_adam"] < 1e-9
    assert abs(out["sd_actual_over_predicted_meta"] - 1.0) < 0.05 and out["frac_within_0p5_2"] == 1.0
    assert abs(out["varF_estimate_over_true"] - 4.0) < 0.4
    assert abs(out["varD_estimate_over_true"] - 1.0) < 0.1
    assert all(abs(a - 0.3) < 1e-12 for a in out["alpha_mean_by_iteration"])
    assert abs(out["alpha_histogram_last_iteration"][3] - 1.0) < 1e-12
    c = out["texel_curves"]["noisiest"]
    assert c["texel"] == int(np.argmax(s))
    assert np.allclose(c["true_gradient"], g[::10, c["texel"]], atol=5 * 2.0 * se + 1e-12)


def test_pinned_spiral_holds_metal_and_roughness():
    """The pinned form of the spiral: metalness and roughness equal the same constants in the
    initial and target textures and their clamp ranges are that single value (the update cannot
    move them), base colour stays free and differs between the two textures."""
    import numpy as np
    from paper_2309_15676_gb300.experiments import pinned_spiral
    sc, init, tgt = pinned_spiral(0.5, 0.35, width=16, height=16, segments=16, sides=8, tex=8)
    for t in (init, tgt):
        assert np.all(t[..., 3] == np.float32(0.5)) and np.all(t[..., 4] == np.float32(0.35))
    assert sc["clamp_lo"][3] == sc["clamp_hi"][3] == 0.5 and sc["clamp_lo"][4] == sc["clamp_hi"][4] == 0.35
    assert sc["clamp_lo"][:3] == [0.0, 0.0, 0.0] and np.any(init[..., :3] != tgt[..., :3])
