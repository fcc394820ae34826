"""Write tests/golden/logistic_16x200_oracle.json from the FP64 oracle only.

The stored values are the oracle's outputs for the 16 x 200 coupled-logistic
workload (seed 1001): per-library optimal E over 1..10 by leave-one-out
simplex at Tp_sel = 1, the skills rho_E, and the 16 x 16 CCM matrix at Tp = 0,
tau = 1 with each library embedded at its optimal E.  They guard the oracle's
arithmetic against silent change; the paper prints no worked example.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2105_12301_gb300 import inputs  # noqa: E402


def main():
    X = inputs.logistic_16x200()
    E_opt, rho_E = oracle.optimal_E_many(X, 10, 1, 1)
    rho = oracle.ccm_matrix(X, X, E_opt, 1, 0)
    out = {
        "workload": "logistic_16x200: 16 coupled logistic maps, L=200, seed 1001",
        "E_max": 10, "tau": 1, "Tp_sel": 1, "Tp": 0,
        "E_opt": [int(e) for e in E_opt],
        "rho_E": [[float(v) for v in r] for r in rho_E],
        "rho": [[float(v) for v in r] for r in rho],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        "logistic_16x200_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
