"""The README's Python example runs as written and gives finite results
(the library's documented first steps must keep working)."""
import os
import re

import pytest
import torch

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_example_runs():
    text = open(os.path.join(ROOT, "README.md"), encoding="utf-8").read()
    blocks = re.findall(r"```python\n(.*?)```", text, flags=re.S)
    assert blocks, "the README has a Python example"
    env = {}
    exec(compile(blocks[0], "README.md example", "exec"), env)
    torch.cuda.synchronize()
    assert torch.isfinite(env["out"]).all() and torch.isfinite(env["dUdt"]).all()
    assert torch.isfinite(env["amax"]).all() and bool((env["amax"] > 0).all())
    env["plan"].close()
    env["forest"].close()
