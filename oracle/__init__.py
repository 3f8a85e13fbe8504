"""FP64 CPU oracle of the gridless quasistatic wake model.

TEST INFRASTRUCTURE ONLY: used by tests/, by the smoke check and by the
benchmark's CPU-baseline and reference legs.  The product library never
imports it.
"""
from .oracle import (OracleResult, build, ring_init, slice_fields, bp_shooting, bp_solve,  # noqa: F401
                     run, run_wake, lib_path)
from . import beam_push  # noqa: F401
