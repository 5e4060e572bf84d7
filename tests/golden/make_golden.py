"""Writes the golden fixtures of this folder.  Calls only ``oracle/`` (and the
seeded input generators); run from the repository root:

    python tests/golden/make_golden.py

nd_7x7_leaf4.json  grid nested-dissection order of a 7 x 7 grid with leaf
                   size 4 (hand-checkable: the first separator is x = 3, then
                   y = 3 in each half, ...), plus its elimination tree and
                   fundamental supernode boundaries.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import symbolic as S  # noqa: E402


def main():
    rp, ci, v = W.laplacian_csr((7, 7))
    perm = S.nd_grid_order((7, 7), leaf=4)
    prp, pci, _ = S.permute_csr(rp, ci, v, perm)
    sym = S.Symbolic(prp, pci)
    out = {"dims": [7, 7], "leaf": 4, "perm": perm.tolist(), "parent": sym.parent.tolist(),
           "colcount": sym.colcount.tolist(), "sn_start": sym.sn_start.tolist(),
           "sn_level": sym.sn_level.tolist()}
    with open(os.path.join(HERE, "nd_7x7_leaf4.json"), "w") as f:
        json.dump(out, f)
        f.write("\n")


if __name__ == "__main__":
    main()
