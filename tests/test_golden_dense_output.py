"""The oracle against exact values of the paper's printed RK4 dense-output
weights and refinement-boundary stage formulas (Sec. II, Eqs. denseoutput1/2
and Y1-Y4), evaluated by hand in tests/golden/."""
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "rk4_dense_output_and_taylor_stages.txt")


def _rows(kind):
    for line in open(GOLDEN):
        parts = line.split()
        if parts and parts[0] == kind:
            yield [Fraction(p) for p in parts[1:]]


def test_dense_output_weights_match_the_printed_formulas(orc):
    n = 0
    for m, theta, *b in _rows("weights"):
        np.testing.assert_allclose(orc.dense_b(float(theta), int(m)), [float(v) for v in b], rtol=0, atol=1e-15)
        n += 1
    assert n == 11


def test_boundary_stage_values_worked_example(orc):
    n = 0
    for theta0, *vals in _rows("stages"):
        got = [orc.amr_value(1.0, [2.0, 3.0, 5.0, 7.0], 0.5, float(theta0), which) for which in (1, 2, 3, 4, 0)]
        np.testing.assert_allclose(got, [float(v) for v in vals], rtol=1e-15, atol=1e-15)
        n += 1
    assert n == 2
