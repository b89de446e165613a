"""Write tests/golden/oracle_values.json: reference values computed by the CPU
oracle alone (oracle/), for GPU parity tests at full workload sizes that the
oracle cannot re-run inside a test.

    python tests/golden/make_golden.py [sphere64] [ellipsoid_o0] [ellipsoid_more]
                                       [sphere256]

Each entry records the oracle's settings (FFT-convolution operator, BiCGSTAB
tolerance), its iterations and true residuals, Q_ext/Q_abs/Q_sca per
polarization and the forward amplitudes f_ml(0).

sphere256 (8.8 M dipoles, 512^3 grid) runs the oracle's low-memory FFT
operator (same arithmetic per element, ~26 GB of host memory) for the first
polarization only: the lattice sphere is invariant under the 90-degree rotation
about the propagation axis x that takes y to z, and LDR's alpha is the same for
both polarizations (S = 0 for khat = x, e = y or z), so the second
polarization's Q's and f_22(0) equal the first's and f_12(0) = f_21(0) = 0.
Progress lines go to stderr.
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

# C3 orientations (index = itheta * NBETA + ibeta) spread over Theta and beta
ELLIPSOID_MORE = (6, 13, 19, 28)


def solve(w, inc=0, tol=1e-11, npol=2, operator="fft", workers=None):
    t0 = time.time()
    count = [0]

    def progress():
        count[0] += 1
        if count[0] % 10 == 0:
            print(f"{w.name} inc {inc}: {count[0]} products, {time.time() - t0:.0f} s",
                  file=sys.stderr, flush=True)

    r = O.solve_target(w.occ, w.comp, w.m, w.kd, w.khat[inc], w.yhat[inc], w.e01[inc],
                       w.method, npol=npol, tol=tol, operator=operator, workers=workers,
                       on_matvec=progress)
    f0 = r["famp"][0]
    return {
        "workload": w.name, "incidence": inc, "N": w.n_dipoles, "kd": w.kd,
        "method": w.method, "m": [[c.real, c.imag] for c in w.m],
        "oracle": "FFT-convolution operator, BiCGSTAB", "tol": tol, "npol": npol,
        "iters": [int(i) for i in r["iters"]], "resid": [float(x) for x in r["resid"]],
        "Qext": [float(x) for x in r["Qext"]], "Qabs": [float(x) for x in r["Qabs"]],
        "Qsca": [float(x) for x in r["Qsca"]],
        "f_forward": [[[float(f0[mm, l].real), float(f0[mm, l].imag)] for l in range(npol)]
                      for mm in range(2)],
        "cpu_seconds": time.time() - t0,
    }


def store(key, value):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    data[key] = value
    json.dump(data, open(OUT, "w"), indent=1)


def main(which):
    workers = int(os.environ.get("ORACLE_WORKERS", "0")) or None
    if "sphere64" in which:
        store("sphere64", solve(W.c2_sphere64()))
    if "ellipsoid_o0" in which:
        store("ellipsoid_o0", solve(W.c3_ellipsoid(), 0, tol=1e-10))
    if "ellipsoid_more" in which:
        w = W.c3_ellipsoid()
        for i in ELLIPSOID_MORE:
            store(f"ellipsoid_o{i}", solve(w, i, tol=1e-10, operator="fft_lowmem",
                                           workers=workers))
    if "sphere256" in which:
        store("sphere256", solve(W.c5_sphere256(), 0, tol=1e-9, npol=1,
                                 operator="fft_lowmem", workers=workers))


if __name__ == "__main__":
    main(sys.argv[1:] or ["sphere64", "ellipsoid_o0"])
