"""The oracle against its stored values (tests/golden/small2d_oracle.json, written by
tests/golden/make_golden.py from the oracle alone): a change to the oracle's arithmetic
shows up here and has to be made on purpose.  The tolerances only absorb rounding-order
differences between machines; the Newton iteration count must match exactly."""
import importlib.util
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _make_golden():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_oracle_reproduces_its_stored_small2d_values():
    stored = json.load(open(os.path.join(HERE, "golden", "small2d_oracle.json")))
    now = _make_golden().compute()
    assert now["workload"] == stored["workload"]
    assert now["newton_converged"] and now["newton_iterations"] == stored["newton_iterations"]
    for key, tol in (("J_prior_mean", 1e-12), ("gradient_norm_prior_mean", 1e-12), ("J_map", 1e-10),
                     ("m_map_norm", 1e-9)):
        assert abs(now[key] - stored[key]) <= tol * abs(stored[key]), key
    assert now["m_map_nodes"] == stored["m_map_nodes"]
    np.testing.assert_allclose(now["m_map_at_nodes"], stored["m_map_at_nodes"], rtol=0, atol=1e-8)
    lam, lam0 = np.array(now["eigenvalues"]), np.array(stored["eigenvalues"])
    big = lam0 > 0.1
    np.testing.assert_allclose(lam[big], lam0[big], rtol=1e-9)
    assert np.all(np.abs(lam[~big] - lam0[~big]) <= 1e-9 * lam0[0])
