"""Writes the stored expected values of the inversion tests.  Calls only the
FP64 oracle (oracle/) on its own seeded records; nothing here comes from the
CUDA library.

    python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_1109_0334_gb300 import workloads as W  # noqa: E402
from common import oracle_record  # noqa: E402


def c2_invert():
    spec = W.get("c2")
    U32, U_m, xt = oracle_record(O, spec)
    c, pm = O.make_case(spec), O.make_pmap(spec)
    t = time.time()
    x, S, hist = O.invert(c, pm, U_m, spec["P"], spec["iters"], spec["w"], spec["c1"],
                          spec["c2"], spec["seed"])
    return dict(workload="c2", x=[float(v) for v in x], S_m2=float(S),
                sumU2_m2=float(np.sum(U_m ** 2)), truth_x=[float(v) for v in xt],
                hist_m2=[float(h) for h in hist], oracle_seconds=time.time() - t,
                threads=O.get_threads())


if __name__ == "__main__":
    O.build()
    O.set_threads(os.cpu_count() or 1)
    out = c2_invert()
    with open(os.path.join(HERE, "c2_invert.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: v for k, v in out.items() if k != "hist_m2"}))
