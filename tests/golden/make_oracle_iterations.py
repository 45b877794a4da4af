"""Write tests/golden/oracle_iterations.json: how many iterations the FP64
oracle's unpreconditioned BiCGStab needs to bring one Z4 source of each
benchmark workload to a true relative residual of 1e-10.

Calls only the oracle (and the seeded input generators). The benchmark's
CPU baseline times a bounded number of oracle iterations on the same
workload and scales by this count.
"""

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1405_4524_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_iterations.json")


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        spec, U, eta = inputs.workload(name, n_rhs=1)
        F = oracle.field_strength(U)
        t = time.time()
        x, it, res = oracle.solve(U, eta[0], spec["kappa"], spec["csw"], -1.0, tol=1e-10, F=F)
        data[name] = {"iterations": int(it), "true_residual": float(res), "tol": 1e-10,
                      "source": 0, "seconds": round(time.time() - t, 1)}
        print(name, data[name], flush=True)
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["4x4x4x8", "16x16x16x32"])
