"""Scatter (step a10) under heavy warp aggregation: eight small problems alternating three- and
five-channel textures of 2x2 texels, so that nearly every warp merges coincident footprints,
clamps taps at the texture edge and, at problem boundaries, mixes channel counts. The gradient of
each problem scattered inside the batch must equal the one scattered alone."""
import numpy as np
import pytest

from paper_2309_15676_gb300 import synth

from .gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def _workloads():
    ws = []
    for k in range(8):
        if k % 2 == 0:
            ws.append(synth.workload_box(12, 8, 2, max_depth=3, key_id=k))
        else:
            ws.append(synth.workload_spiral(8, 12, 16, 6, 2, max_depth=4, key_id=k))
    return ws


def test_batched_scatter_equals_single_with_merges_and_mixed_channels():
    torch = need_gpu()
    from paper_2309_15676_gb300.api import Context, HyperParams
    ws = _workloads()
    rng = np.random.default_rng(3)
    targets = [rng.uniform(0.0, 1.0, (w.scene["height"], w.scene["width"], 3)).astype(np.float32) for w in ws]

    def grads(items):
        ctx = Context(0)
        ids = []
        for w, t in items:
            p = ctx.add_scene(w.scene, HyperParams(lr=0.02))
            ctx.set_target(p, t)
            ctx.set_params(p, w.init_tex)
            ids.append(p)
        ctx.gradient_step()
        out = [ctx.grads(p)[0].cpu().numpy() for p in ids]
        ctx.close()
        return out

    batched = grads(list(zip(ws, targets)))
    for k, (w, t) in enumerate(zip(ws, targets)):
        (alone,) = grads([(w, t)])
        assert np.abs(alone).max() > 0, k
        err = np.abs(batched[k] - alone).max()
        assert err <= 1e-5 * np.abs(alone).max(), (k, err)
