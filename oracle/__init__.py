"""FP64 CPU oracle of the SOP-model overdamped Langevin step (Python side).

TEST INFRASTRUCTURE ONLY. This package is the plain, slow restatement of the
paper's method that the CUDA path is checked against. Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it. It shares no code with the CUDA library and never imports it; both sides
take their inputs from the seeded generator in ``paper_1003_1148_gb300.synth``.

The arithmetic lives in ``sop_oracle.c`` (compiled with gcc, FP64, no FMA
contraction, no fast-math). This module only marshals numpy arrays.

Parity pins (tests/test_oracle_*.py): closed-form values of each potential at
special distances, central finite differences of the energy against the
forces, zero net force and torque, brute-force against scipy KD-tree and cell
lists, Philox against ATen's independent implementation, the Hybrid Taus
components against their bit-level linear recurrences and the LCG against its
closed form, Box-Muller
invariants and moments, the exactly solvable Brownian particle (Eqs. 3-4) and
the free-diffusion law.
"""
from .oracle import (Model, Ramp, box_muller, box_muller4, build, bonds, kB, native_pairs, noise, philox,
                     taus_next, OracleError, model_from_workload)

__all__ = ["Model", "Ramp", "box_muller", "box_muller4", "build", "bonds", "kB", "native_pairs", "noise", "philox", "taus_next",
           "OracleError", "model_from_workload"]
