"""The smoke entry point (one tiny wave and Z4c run on cuda:0, checked
against the oracle) runs clean."""
import os
import sys

import pytest

pytestmark = pytest.mark.gpu


def test_smoke_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import __graft_entry__ as g
    g.smoke()
