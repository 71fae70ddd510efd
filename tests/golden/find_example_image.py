"""Recover the running example's image from its printed table of critical points.

The paper prints the table of classical and ordinary critical points and values of its
running example (Appendix A.1, Table 2) but not the image itself.  This script searches
all 2^16 binary 4 x 4 images (vertex construction) for those whose classical tables,
computed by the oracle, equal the printed ones, and prints them.  It found exactly one,
stored as "image" in worked_example.json.  Test infrastructure: it calls only oracle/.

    python tests/golden/find_example_image.py
"""
import json
import os
import sys
from itertools import product

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402


def _key(v, m0=4):
    # vertex (i0, i1) has cell key 2 i0 + 14 i1 on the 7 x 7 grid of the example
    return 2 * (v % m0) + 14 * (v // m0)


def _orthant(eps):
    return sum(1 << k for k, e in enumerate(eps) if e == -1)


def main():
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "worked_example.json")) as f:
        golden = json.load(f)
    want = {_orthant(r["eps"]): set(zip(r["lw_pts"], r["lw_vals"])) for r in golden["critical_table"]["rows"]}
    found = []
    for bits in product((0, 1), repeat=16):
        img = np.array(bits, dtype=np.int64).reshape(4, 4)
        tab = O.critical_tables(img)
        if all({(_key(v), int(x)) for v, x in zip(tab.lower_idx[o], tab.lower_val[o])} == want[o] for o in want):
            found.append(img.tolist())
    print(json.dumps(found))
    return found


if __name__ == "__main__":
    main()
