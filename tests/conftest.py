import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def paper_value(key: str) -> dict:
    """An entry of tests/golden/paper_printed_values.json (numbers the paper
    prints, each with its place)."""
    import json
    with open(os.path.join(ROOT, "tests", "golden", "paper_printed_values.json")) as f:
        return json.load(f)[key]


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU run (tens of seconds)")
