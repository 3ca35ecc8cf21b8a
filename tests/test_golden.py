"""The oracle against its stored regression fixture (tests/golden/oracle_regression.json,
written by tests/golden/make_golden.py from the oracle itself): a change of the oracle's
arithmetic shows here and must be justified by the paper before the fixture is rewritten.
Layer ids, S^H and E exactly; values to 1e-12 (libm may differ in the last bit between
hosts)."""
import json
import os

import numpy as np
import pytest

from golden import make_golden

HERE = os.path.dirname(os.path.abspath(__file__))
FIXTURE = json.load(open(os.path.join(HERE, "golden", "oracle_regression.json")))


@pytest.mark.parametrize("name,scene,window", make_golden.scenes(), ids=lambda x: x if isinstance(x, str) else "")
def test_oracle_matches_its_regression_fixture(name, scene, window):
    want = FIXTURE["cases"][name]
    got = make_golden.compute(scene, window)
    for k in ("ids", "sh", "edge"):
        assert np.array_equal(np.asarray(got[k]), np.asarray(want[k])), k
    for k in ("rgba", "grad_pos", "grad_col"):
        np.testing.assert_allclose(np.asarray(got[k]), np.asarray(want[k]), rtol=1e-12, atol=1e-12, err_msg=k)
