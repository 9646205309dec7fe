import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def read_golden(name: str) -> dict:
    """Parse a tests/golden fixture: 'key: v1 v2 ...' lines, '#' comments.
    Repeated keys collect into a list of value lists."""
    path = os.path.join(ROOT, "tests", "golden", name)
    out: dict = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, val = line.partition(":")
            toks = val.split()
            if key in out:
                if not isinstance(out[key][0], list):
                    out[key] = [out[key]]
                out[key].append(toks)
            else:
                out[key] = toks
    return out


@pytest.fixture(scope="session")
def golden():
    return read_golden
