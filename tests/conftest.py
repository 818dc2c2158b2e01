import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    # name every skipped test and its reason in the closing summary, also
    # under -q (e.g. a property-test module whose hypothesis import is absent)
    chars = getattr(config.option, "reportchars", None)
    if isinstance(chars, str) and "s" not in chars and "a" not in chars.lower():
        config.option.reportchars = chars + "s"
