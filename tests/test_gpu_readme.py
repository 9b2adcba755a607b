"""The README's Python example runs and prints what it says."""
import os
import re

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_example(capsys):
    from paper_2606_15437_gb300 import build as mkbuild
    mkbuild.build()
    text = open(os.path.join(ROOT, "README.md")).read()
    code = re.search(r"```python\n(.*?)```", text, re.S).group(1)
    exec(compile(code, "README.md", "exec"), {})
    out = capsys.readouterr().out.split("\n")
    assert out[0].split() == ["[", "1", "23", "1609]"] or out[0].replace(" ", "") == "[1231609]"
    assert out[1] == "(6, 17335328, 0, 2)"
    assert out[2] == "[(6, 0, 0, 0)]"
