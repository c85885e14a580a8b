"""Host-side checks of the binding (no GPU): every caller-supplied buffer is
checked for device, dtype, shape and contiguity before its pointer reaches the
library, which trusts the pointers and sizes it is given; parameters off the
GPU are refused before any library call."""
import importlib

import pytest
import torch

R = importlib.import_module("paper_2501_06838_gb300.render")


def test_buffer_checks():
    cpu = torch.device("cpu")
    t = torch.zeros(3, 4, 5)
    assert R._need(t, (3, 4, 5), torch.float32, cpu, "output") is t
    with pytest.raises(ValueError, match="shape"):
        R._need(t, (3, 5, 4), torch.float32, cpu, "output")
    with pytest.raises(ValueError, match="contiguous"):
        R._need(t.transpose(1, 2).contiguous().transpose(1, 2), (3, 4, 5), torch.float32, cpu,
                "output")
    with pytest.raises(TypeError, match="float32"):
        R._need(t.double(), (3, 4, 5), torch.float32, cpu, "output")
    with pytest.raises(ValueError, match="meta"):
        R._need(t, (3, 4, 5), torch.float32, torch.device("meta"), "output")


def test_parameters_must_be_on_the_gpu():
    n = 4
    g = R.Gaussians(torch.zeros(n, 2), torch.ones(n, 2), torch.zeros(n), torch.zeros(n, 3),
                    torch.zeros(n))
    with pytest.raises(ValueError, match="CUDA"):
        R._device([g])
    with pytest.raises(ValueError, match="CUDA"):
        R._struct_g(g)
    v = R.View(2, 2, 4, 4, 2.0)
    with pytest.raises(ValueError, match="CUDA"):
        R.render(g, v)
    with pytest.raises(ValueError, match="one view per image"):
        R.render_batched([g], [v, v])
