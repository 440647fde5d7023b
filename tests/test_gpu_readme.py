"""The README's Python example runs as written (on the GPU)."""
import os
import re

import pytest

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_python_example_runs():
    require_gpu()
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, flags=re.S)
    assert blocks, "README has no python example"
    for code in blocks:
        exec(compile(code, "README.md", "exec"), {"__name__": "readme_example"})
