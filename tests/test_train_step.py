"""Config 5: end-to-end training steps through the renderer's autograd
Function (BF16 parameters, per-sample scales) reduce the L1 loss."""
import numpy as np
import pytest

import gs_synthetic as S


def test_image_function_sampling_convention():
    """The HR target at scale s samples the same function at (x/s, y/s):
    pixel (s*x, s*y) of an integer-scale target equals LR pixel (x, y)."""
    f = S.image_function(5)
    ys, xs = np.mgrid[0:48, 0:48]
    lr = f(xs, ys)
    Y, X = np.mgrid[0:96, 0:96] / 2.0
    hr = f(X, Y)
    np.testing.assert_allclose(hr[:, ::2, ::2], lr, rtol=0, atol=1e-12)


@pytest.mark.gpu
def test_training_steps_reduce_loss():
    import torch
    from paper_2501_06838_gb300.train_step import TrainStep
    step = TrainStep()
    losses = []
    lr, hrs, scales = S.config5_batch(0)
    lr_t = torch.from_numpy(lr).cuda()
    hr_t = [torch.from_numpy(h).cuda() for h in hrs]
    for it in range(30):
        losses.append(float(step(lr_t, hr_t, scales)))
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.8 * losses[0], losses
    # gradients reached the first encoder layer
    assert step.model.inp.weight.grad is not None
    assert float(step.model.inp.weight.grad.abs().sum()) > 0


@pytest.mark.gpu
def test_fused_head_matches_pytorch_activations():
    """The renderer's fused head and the same activations in PyTorch give the same
    first-step loss and encoder gradient (float32 parameters, same seed)."""
    import torch
    from paper_2501_06838_gb300.train_step import TrainStep
    lr, hrs, scales = S.config5_batch(0)
    lr_t = torch.from_numpy(lr).cuda()
    hr_t = [torch.from_numpy(h).cuda() for h in hrs]
    res = {}
    for fused in (True, False):
        step = TrainStep(param_dtype=torch.float32, fused_head=fused, lr=0.0)
        loss = float(step(lr_t, hr_t, scales))
        res[fused] = (loss, step.model.inp.weight.grad.detach().clone())
    assert abs(res[True][0] - res[False][0]) < 1e-5 * abs(res[False][0])
    ga, gb = res[True][1], res[False][1]
    assert float((ga - gb).abs().max()) < 1e-3 * float(gb.abs().max())
