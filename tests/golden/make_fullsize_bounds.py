"""Write tests/golden/fullsize_bounds.json: certified upper bounds of the
stopping-rule constants for the full-size RC workloads.

Calls only the oracle (``oracle.bounds.certified_bounds``: a CG solve turned
into a verified M-matrix super-solution).  Run from the repository root:

    python tests/golden/make_fullsize_bounds.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import pgsynth  # noqa: E402
from oracle import bounds  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fullsize_bounds.json")


def main():
    res = {"_cite": "Section III-B (Lemma 1: M is an M-matrix) and Eq. 2 / Eq. 10 (backward Euler); "
                    "verified super-solutions bound ||M^-1 D||_inf and 1 + ||G^-1 (C/h) 1||_inf"}
    for cfg in (1, 4):
        net = pgsynth.CONFIGS[cfg]()
        t0 = time.time()
        b = bounds.certified_bounds(net, net.meta["h"])
        b["seconds"] = time.time() - t0
        b["workload"] = net.name
        b["h"] = net.meta["h"]
        res[f"config{cfg}"] = b
        print(cfg, b, flush=True)
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
