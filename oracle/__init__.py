"""FP64 CPU oracle of the GEM-PIC step (Pukhov, Elkina, Wilson, arXiv 2509.16793).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or execute this
package: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline and
--impl reference legs use it.  It shares no code with the CUDA path; the only common input
is the seeded workload description in paper_2509_16793_gb300/workloads.py, which the caller
passes in (this package imports nothing from the product package).
"""
from .gempic_ref import RefSim  # noqa: F401
