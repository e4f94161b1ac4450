"""The FP64 oracle reproduces tests/golden/oracle_snapshots.txt (written by
tests/golden/make_oracle_snapshots.py, which calls only oracle/): a regression guard, so that
any change of the oracle's arithmetic shows up and has to be justified."""
import importlib.util
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _load():
    spec = importlib.util.spec_from_file_location("make_oracle_snapshots",
                                                  os.path.join(HERE, "golden", "make_oracle_snapshots.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_oracle_reproduces_its_snapshots():
    stored = {}
    for ln in open(os.path.join(HERE, "golden", "oracle_snapshots.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        name, *vals = ln.split()
        stored[name] = np.array([float(v) for v in vals])
    got = dict(_load().cases())
    assert set(got) == set(stored)
    for name, vals in got.items():
        ref = stored[name]
        assert np.allclose(np.ravel(vals), ref, rtol=1e-12, atol=1e-15), name
