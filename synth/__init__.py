"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benches.

This package generates inputs only: Haar-random SU(2) gauge fields, smeared
gauge fields with a chosen mean plaquette, Gaussian spinor sources and random
gauge transformations.  It contains none of the Dirac operator's or the
solver's arithmetic; both sides receive identical arrays from here.
"""

from .fields import (  # noqa: F401
    Rng,
    haar_quaternions,
    haar_links,
    identity_links,
    gaussian_spinor,
    ape_smear_to_plaquette,
    mean_plaquette,
    quat_mul,
    quat_conj,
    lattice_volume,
)
