"""The README's Python example runs as written."""
import os
import re

import pytest
import torch

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_example_runs(capsys):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, flags=re.S)
    assert len(blocks) == 1
    exec(compile(blocks[0], "README.md", "exec"), {"__name__": "readme"})
    torch.cuda.synchronize()
    loss = float(capsys.readouterr().out.strip().splitlines()[-1])
    assert 0.0 < loss < 10.0
