"""The Python example in README.md: its names exist (CPU) and it runs (GPU)."""
import ast
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _example():
    with open(os.path.join(ROOT, "README.md")) as f:
        text = f.read()
    blocks = re.findall(r"```python\n(.*?)```", text, re.S)
    assert len(blocks) == 1, "README.md has one Python example"
    return blocks[0]


def test_readme_example_names_exist():
    code = _example()
    tree = ast.parse(code)
    from paper_2004_11658_gb300 import dp, synth
    mods = {"dp": dp, "synth": synth}
    used = {(n.value.id, n.attr) for n in ast.walk(tree)
            if isinstance(n, ast.Attribute) and isinstance(n.value, ast.Name) and n.value.id in mods}
    assert used, "the example calls the binding"
    for mod, attr in sorted(used):
        assert hasattr(mods[mod], attr), f"{mod}.{attr}"


@pytest.mark.gpu
def test_readme_example_runs():
    import torch
    scope = {}
    exec(compile(_example(), "README.md", "exec"), scope)
    torch.cuda.synchronize()
    out, thermo, ctx = scope["out"], scope["thermo"], scope["ctx"]
    assert out["status"] == 0 and ctx.status() == 0
    assert math.isfinite(out["energy"].item())
    assert torch.isfinite(out["force"]).all()
    assert torch.isfinite(thermo).all()
    assert 200.0 < thermo[-1, 2].item() < 400.0   # a 300 K start stays near 300 K over 50 fs
