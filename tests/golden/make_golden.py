"""Write the stored expected values under tests/golden/ (calls only oracle/).

schlogl_cme_t10.txt: law of X at t = 10 for the Schloegl model (bistable
parameter set of Sec. 4.2 in c-convention, X0 = 250, reservoirs A = 1e5 and
B = 2e5 held fixed), from the chemical master equation truncated at X <= 1500
(mass lost to the truncation < 1e-10).  Columns: x, P(X = x).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import cme  # noqa: E402
from paper_2605_00479_gb300 import presets  # noqa: E402


def schlogl_cme():
    m = presets.schlogl()
    x0 = presets.schlogl_x0(m)
    states, P = cme.transient(m, x0, [1500, int(x0[1]), int(x0[2])], [10.0])
    v, p = cme.marginal(states, P[0], 0)
    with open(os.path.join(HERE, "schlogl_cme_t10.txt"), "w") as f:
        f.write("# Schloegl X law at t=10 from the truncated CME (see make_golden.py)\n")
        for xv, pv in zip(v, p):
            f.write(f"{xv} {pv:.17e}\n")


if __name__ == "__main__":
    schlogl_cme()
