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


def test_measured_fp64_peaks_are_sane():
    """sc_measure_fp64_peak (the bench's roofline denominators): the measured
    DFMA issue rate lies between the DADD rate and the nominal SMs x clock x 2
    per SM per clock (with a few percent of timer slack)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_09629_gb300 as sc
    sc.build()
    pk = sc.sc_measure_fp64_peak()
    nominal = pk["sms"] * pk["sm_clock_mhz"] * 2 / 1e3  # G DFMA/s
    assert pk["sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    assert 0.5 * nominal < pk["dadd_g_per_s"] <= pk["dfma_g_per_s"] * 1.02 <= nominal * 1.05, (pk, nominal)
