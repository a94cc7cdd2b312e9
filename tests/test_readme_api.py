"""The Python example in README.md names only calls the package has (no GPU:
names and signatures are checked, nothing is run)."""
import inspect
import os
import re

import paper_2208_08903_gb300 as gf
from paper_2208_08903_gb300 import train

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _example():
    with open(os.path.join(ROOT, "README.md")) as f:
        text = f.read()
    blocks = re.findall(r"```python\n(.*?)```", text, re.S)
    assert blocks, "README.md has no Python example"
    return blocks[0]


def test_readme_example_names_exist():
    code = _example()
    for name in set(re.findall(r"\bgf\.(\w+)", code)):
        assert hasattr(gf, name), name
    for name in set(re.findall(r"\btrain\.(\w+)", code)):
        assert hasattr(train, name), name
    for meth in set(re.findall(r"\b(?:flow|f32)\.(\w+)\(", code)):
        assert hasattr(gf.Flow, meth), meth


def _top_level(args: str) -> str:
    """The argument text without the contents of nested calls."""
    prev = None
    while prev != args:
        prev, args = args, re.sub(r"\([^()]*\)", "", args)
    return args


def test_readme_example_keywords_are_parameters():
    code = _example()
    calls = {"gf.Flow": gf.Flow.__init__, "flow.sample": gf.Flow.sample, "flow.logq": gf.Flow.logq,
             "gf.new_mh_state": gf.new_mh_state, "gf.autocorr": gf.autocorr, "train.train": train.train}
    for prefix, fn in calls.items():
        params = inspect.signature(fn).parameters
        for m in re.finditer(re.escape(prefix) + r"\((.*)\)", code):
            for kw in re.findall(r"\b(\w+)=", _top_level(m.group(1))):
                assert kw in params, (prefix, kw)
