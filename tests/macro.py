"""Macroscopic observables of long rollouts (the package's analysis functions, re-exported
for the tests)."""
from paper_2106_09576_gb300.observables import angle_of_repose, discharge_rate, packing_fraction  # noqa: F401
