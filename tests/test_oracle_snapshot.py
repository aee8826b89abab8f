"""Oracle regression snapshot (integration test in the style of Sec. 3.2).

The fixture was written by tests/golden/make_golden.py from the oracle only;
it guards the oracle's arithmetic against unintended change.
"""
import os

import numpy as np

from tests.golden.make_golden import run

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_stored_snapshot():
    path = os.path.join(HERE, "golden", "cavity_8x8x8_10steps.txt")
    ref = np.loadtxt(path)
    got = np.array(run(), dtype=np.float64)
    np.testing.assert_array_equal(got[:, :5], ref[:, :5])          # iteration counts
    np.testing.assert_allclose(got[:, 5:], ref[:, 5:], rtol=1e-12, atol=1e-15)
