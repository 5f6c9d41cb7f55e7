"""The iteration's replays from the hit store (each PRB radiance pass keeps its paths' closest hits
and NEE visibilities, the replays trace nothing) against replays that re-trace every ray: the
same hits, so the same gradients up to the order of the float reductions, on a glossy spiral
(FD pairs that split), with shared-path FD pairs, and on a batch that mixes depths and scene kinds."""
import numpy as np
import pytest

from paper_2309_15676_gb300 import synth

from .gpu_common import need_gpu, params_match, rel_l2

pytestmark = pytest.mark.gpu


def _run(ws, flags, hit_store, iters=3):
    from paper_2309_15676_gb300.api import Context, HyperParams
    ctx = Context(0, replay_hit_store=hit_store)
    rng = np.random.default_rng(3)
    ids = []
    for w in ws:
        p = ctx.add_scene(w.scene, HyperParams(lr=0.02, flags=flags))
        ctx.set_target(p, rng.uniform(0, 1, (w.scene["height"], w.scene["width"], 3)).astype(np.float32))
        ctx.set_params(p, w.init_tex)
        ids.append(p)
    ctx.iterate(iters, use_graph=True)
    launches = ctx.launch_count()       # per iteration, gradient part and update
    ctx.gradient_step()
    out = []
    for p in ids:
        F, dF = (x.cpu().numpy().astype(np.float64) for x in ctx.grads(p))
        out.append((F, dF, ctx.get_params(p).cpu().numpy(), ctx.stats(p)["loss"]))
    ctx.close()
    return out, launches


@pytest.mark.parametrize("case", ["spiral", "spiral_shared_fd", "batch"])
def test_stored_replay_equals_retrace(case):
    need_gpu()
    from paper_2309_15676_gb300.api import META_FD_SHARED_PATH
    if case == "batch":
        ws = [synth.workload_box(32, 32, 16, max_depth=3, key_id=5),
              synth.workload_spiral(40, 32, 64, 16, 32, max_depth=6, spp_prop=2, spp_fd=1, key_id=9)]
    else:
        ws = [synth.workload_spiral(48, 40, 64, 16, 32, max_depth=5, spp_prop=2, spp_fd=1)]
    flags = META_FD_SHARED_PATH if case == "spiral_shared_fd" else 0
    a, la = _run(ws, flags, hit_store=True)
    b, lb = _run(ws, flags, hit_store=False)
    assert la < lb          # the stored replays launch no traversal
    if case != "batch":     # depth 5: four passes of 2D+1 launches, replays of D (or 2D+1), 10 others
        assert (la, lb) == (4 * 11 + 2 * 5 + 10, 6 * 11 + 10), (la, lb)
    for (Fa, dFa, pa, lsa), (Fb, dFb, pb, lsb) in zip(a, b):
        assert np.abs(Fa).max() > 0 and np.abs(dFa).max() > 0
        assert rel_l2(Fa, Fb) < 1e-5 and rel_l2(dFa, dFb) < 1e-5, (rel_l2(Fa, Fb), rel_l2(dFa, dFb))
        assert params_match(pa, pb)
        assert abs(lsa - lsb) <= 1e-6 * abs(lsb)
