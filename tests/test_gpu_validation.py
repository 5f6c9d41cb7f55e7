"""Statistical validation along a prescribed trajectory (Sec. 6, "variance reduction without lag"):
the box parameters move linearly from the initial to the target texture without an optimiser
(mer_params_force), 500 independent runs give the expected gradient and the actual variances.
Checked: the meta-estimate follows the moving expected gradient more closely than Adam's
bias-corrected EMA of the same samples (no lag), its actual variance is lower, its predicted
standard deviation is within a factor 2 of the actual one for most texels and iterations, and the
zero-centred Var[<F>] approximation does not underestimate."""
import pytest

from .gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def test_trajectory_study_linear():
    need_gpu()
    from paper_2309_15676_gb300.experiments import trajectory_study
    r = trajectory_study(runs=500, iters=40, schedule="linear", per_ctx=250)
    assert r["texels"] > 100
    assert r["lag_meta"] < r["lag_adam"], r
    assert r["var_ratio_meta"] < r["var_ratio_adam"] < 1.0, r
    assert r["frac_within_0p5_2"] > 0.5, r
    assert r["varF_estimate_over_true"] > 1.0, r
