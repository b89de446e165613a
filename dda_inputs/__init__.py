"""Seeded synthetic inputs (targets, orientations, workloads) shared by the
CUDA path's tests and bench and by the CPU oracle.  No DDA arithmetic lives
here."""
