"""GB300-native discrete dipole approximation (the DDSCAT 7.3 guide's method):
BiCGSTAB on A P = E_inc with the A.P product as a zero-padded 3-D FFT
convolution, in hand-written sm_103a CUDA kernels behind a C ABI
(include/dda.h).

    from paper_1305_6497_gb300 import binding
    t = binding.Target(occ, comp, [1.5 + 0.02j], method="LDR")
    out = t.solve(kd, khat, e01, precision="fp32_refined")

The binding loads libdda.so on first use and raises if it is missing.
"""


def __getattr__(name):
    if name == "binding":
        import importlib
        return importlib.import_module(".binding", __name__)
    raise AttributeError(name)
