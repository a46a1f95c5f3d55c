"""The round-trip the entry module's smoke() makes (an L = 12 product and mixed-precision
solve on cuda:0, checked against the oracle and dense LAPACK), run as a GPU test."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_smoke_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sys.path.insert(0, ROOT)
    import __graft_entry__ as entry
    entry.smoke()
