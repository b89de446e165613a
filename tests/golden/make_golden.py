"""Write tests/golden/oracle_values.json: reference values computed by the CPU
oracle alone (oracle/), for GPU parity tests at full workload sizes that the
oracle cannot re-run inside a test.

    python tests/golden/make_golden.py [sphere64] [ellipsoid_o0]

Each entry records the oracle's settings (FFT-convolution operator, BiCGSTAB
tolerance), its iterations and true residuals, Q_ext/Q_abs/Q_sca per
polarization and the forward amplitudes f_ml(0).
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from dda_inputs import workloads as W  # noqa: E402
from oracle import dda as O  # noqa: E402

OUT = os.path.join(HERE, "oracle_values.json")


def solve(w, inc=0, tol=1e-11):
    t0 = time.time()
    r = O.solve_target(w.occ, w.comp, w.m, w.kd, w.khat[inc], w.yhat[inc], w.e01[inc],
                       w.method, npol=2, tol=tol, operator="fft")
    f0 = r["famp"][0]
    return {
        "workload": w.name, "incidence": inc, "N": w.n_dipoles, "kd": w.kd,
        "method": w.method, "m": [[c.real, c.imag] for c in w.m],
        "oracle": "FFT-convolution operator, BiCGSTAB", "tol": tol,
        "iters": [int(i) for i in r["iters"]], "resid": [float(x) for x in r["resid"]],
        "Qext": [float(x) for x in r["Qext"]], "Qabs": [float(x) for x in r["Qabs"]],
        "Qsca": [float(x) for x in r["Qsca"]],
        "f_forward": [[[float(f0[mm, l].real), float(f0[mm, l].imag)] for l in range(2)]
                      for mm in range(2)],
        "cpu_seconds": time.time() - t0,
    }


def main(which):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    if "sphere64" in which:
        data["sphere64"] = solve(W.c2_sphere64())
        json.dump(data, open(OUT, "w"), indent=1)
    if "ellipsoid_o0" in which:
        data["ellipsoid_o0"] = solve(W.c3_ellipsoid(), 0, tol=1e-10)
        json.dump(data, open(OUT, "w"), indent=1)


if __name__ == "__main__":
    main(sys.argv[1:] or ["sphere64", "ellipsoid_o0"])
