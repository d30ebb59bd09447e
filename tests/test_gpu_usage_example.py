"""The library's usage example (paper_2004_11658_gb300/example.py): it builds
the list, evaluates and runs MD through the binding on a GPU."""
import math

import pytest


@pytest.mark.gpu
def test_usage_example_runs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_11658_gb300 import example
    out, thermo, ctx = example.main()
    torch.cuda.synchronize()
    assert out["status"] == 0 and ctx.status() == 0
    assert math.isfinite(out["energy"].item())
    assert torch.isfinite(out["force"]).all()
    assert torch.isfinite(thermo).all()
    assert 200.0 < thermo[-1, 2].item() < 400.0   # a 300 K start stays near 300 K over 50 fs
