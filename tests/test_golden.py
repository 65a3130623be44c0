"""The paper's printed constants, read from tests/golden/paper_values.txt."""
import os

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def paper_values():
    out = {}
    with open(os.path.join(HERE, "golden", "paper_values.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def test_oracle_uses_the_papers_constants():
    pv = paper_values()
    assert oracle.GAMMA == pv["gamma"]
    assert oracle.BIN_SIZE == pv["bin_size"]
    assert pv["energy_drift_bound"] == 4e-4
