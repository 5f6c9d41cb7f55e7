"""The Python binding checks every array it hands to the library (which receives bare pointers)
before any copy or library call: element counts against the problem's texture and image sizes,
and dtype, contiguity and device of caller-supplied buffers. Checked on the CPU: every refusal
happens before device work."""
import numpy as np
import pytest
import torch

from paper_2309_15676_gb300 import api


def _ctx():
    """A Context with one 8x8x5-texture, 4x6-image problem registered (no device work happens:
    every call below is refused before it)."""
    c = object.__new__(api.Context)
    c.device = torch.device("cuda", 0)
    c.shapes = [(8, 8, 5)]
    c.images = [(4, 6)]
    return c


@pytest.mark.parametrize("call", [
    lambda c: c.set_params(0, np.zeros((8, 8, 3))),
    lambda c: c.force_params(0, np.zeros(8 * 8 * 5 - 1)),
    lambda c: c.render_target(0, np.zeros((4, 4, 5)), 4),
    lambda c: c.set_target(0, np.zeros((4, 6, 4))),
    lambda c: c.render(0, np.zeros((8, 8, 4))),
    lambda c: c.render(0, None, out=torch.zeros(4, 6, 3)),                      # host tensor as output
    lambda c: c.render_samples(0, np.zeros(3)),
    lambda c: c.render_pair(0, np.zeros((8, 8, 5)), np.zeros((8, 8, 3))),
    lambda c: c.adjoint(0, None, np.zeros((4, 6, 2))),
    lambda c: c.adjoint_pair(0, np.zeros((8, 8, 5)), np.zeros((8, 8, 5)), np.zeros((4, 6, 3)), np.zeros(5)),
    lambda c: c.set_target_host(0, torch.zeros(4, 6, 3, dtype=torch.float64)),   # wrong dtype
    lambda c: c.set_target_async(0, torch.zeros(4, 7, 3)),                       # wrong size
    lambda c: c.loss_async(0, torch.zeros(1, dtype=torch.float32)),              # wrong dtype
])
def test_context_refuses_wrong_sizes_and_buffers(call):
    with pytest.raises(ValueError):
        call(_ctx())


def test_right_sizes_pass_the_checks():
    """The same checks accept correctly sized inputs of any shape (here only the checks run)."""
    assert api._numel(np.zeros((8, 8, 5))) == 320
    api._host_buf(torch.zeros(4, 6, 3), torch.float32, 72, "target image")
    api._host_buf(torch.zeros(2, dtype=torch.float64)[1:2], torch.float64, 1, "loss")
    with pytest.raises(ValueError):
        api._host_buf(torch.zeros(6, 4, 3).transpose(0, 1), torch.float32, 72, "target image")    # not contiguous


def test_module_functions_refuse_host_or_mismatched_tensors():
    x = torch.zeros(12)
    with pytest.raises(ValueError):
        api.image_loss(x, x)                                                   # host tensors
    with pytest.raises(ValueError):
        api.philox(0, 0, torch.zeros(5, 4, dtype=torch.int32))                # host counters
    with pytest.raises(ValueError):
        api.meta_step_raw(api.HyperParams(), x, x, x, x, x, x, x, x, x, 3, [0] * 3, [1] * 3, 0, 0, 0, 0.0)
    with pytest.raises(ValueError):
        api.meta_step_raw_ex(api.HyperParams(), {"pi": x}, 3, [0] * 3, [1] * 3, 0, 0, 0, 0.0)


def test_volume_refuses_wrong_sizes():
    v = object.__new__(api.Volume)
    v.device = torch.device("cuda", 0)
    v.shape = (4, 4, 4, 4)
    v.image_shape = (2, 3, 5, 3)
    for call in (lambda: v.render(np.zeros((4, 4, 4, 3))),
                 lambda: v.adjoint(np.zeros((4, 4, 4, 4)), np.zeros((2, 3, 5, 2))),
                 lambda: v.adjoint(np.zeros((4, 4, 4, 4)), np.zeros((2, 3, 5, 3)), grad=torch.zeros(256)),
                 lambda: v.adjoint_pair(np.zeros(256), np.zeros(255), np.zeros(90), np.zeros(90))):
        with pytest.raises(ValueError):
            call()
