"""Writes oracle_regression.txt: digests of the oracle's outputs on small
integer-only synthetic inputs.  Calls only the oracle and the integer input
generators, so the stored values never come from the CUDA library.

    python tests/golden/make_golden.py
"""
import hashlib
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from tests.golden.cases import REGRESSION_CASES, make_case  # noqa: E402


def digest(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(a.tobytes())
    return h.hexdigest()[:32]


def main():
    lines = ["# name sha256[:32] of (assign, level, rgba8) from the oracle",
             "# written by tests/golden/make_golden.py (oracle only)"]
    for name in REGRESSION_CASES:
        c = make_case(name)
        out, a, lev = oracle.stylize(c["tgt"], c["src"], c["style"], c["key_bits"], c["levels"],
                                     c["threshold"], c["radius"], c["seed"], n_threads=4)
        lines.append(f"{name} {digest(a, lev, out)}")
    with open(os.path.join(HERE, "oracle_regression.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
