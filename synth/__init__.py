"""Seeded synthetic star catalogues for the extinction-mapping hot path.

This package only draws inputs: sky positions, distances, a truth extinction
field and noisy observations.  It computes nothing that the mapper itself
computes (no covariance quadrature, no EP), so both the CPU oracle and the
CUDA path can take their inputs from here without sharing arithmetic.
"""
from .catalogue import (Workload, WORKLOADS, make_catalogue, make_fields,
                        catalogue_subset, make_disc_catalogue, DISC_TRUTH)

__all__ = ["Workload", "WORKLOADS", "make_catalogue", "make_fields",
           "catalogue_subset", "make_disc_catalogue", "DISC_TRUTH"]
