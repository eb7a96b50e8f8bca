"""The oracle reproduces the digests stored by tests/golden/make_golden.py
(guards against platform-dependent behaviour, e.g. x86 vs Arm hosts)."""
import os

import pytest

import oracle
from tests.golden.cases import REGRESSION_CASES, make_case
from tests.golden.make_golden import digest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_regression.txt")


def _stored():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        out[k] = v
    return out


@pytest.mark.parametrize("name", REGRESSION_CASES)
def test_oracle_regression_digest(name):
    c = make_case(name)
    out, a, lev = oracle.stylize(c["tgt"], c["src"], c["style"], c["key_bits"], c["levels"],
                                 c["threshold"], c["radius"], c["seed"], n_threads=2)
    assert digest(a, lev, out) == _stored()[name]
