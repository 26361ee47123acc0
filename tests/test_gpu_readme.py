"""The usage example in README.md runs as written on the GPU (so the documented calls stay valid)."""
import os
import re

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_readme_example_runs():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "README.md"), encoding="utf-8").read()
    blocks = re.findall(r"```python\n(.*?)```", text, re.S)
    assert blocks, "README has no python example"
    scope = {}
    exec(compile(blocks[0], "README.md", "exec"), scope)
    torch.cuda.synchronize()
    assert scope["X"].grad.shape == scope["x"].shape
    assert torch.equal(scope["y2"], scope["y"])            # the fused pass's outputs are the forward's bits
