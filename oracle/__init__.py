"""CPU FP64 (long-double accumulating) oracle for the block-step Hermite N-body method.

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's
CPU baseline may import this package; the product path never does.  It shares
no code with the CUDA library.  See oracle.c for the formulas and their sources.

Parity status per function:
  force, energy, predict, correct, interp, dt_criterion, dt_quantise,
  dt_startup, next_block, integrate: pinned (tests/test_oracle_pins.py; the
  start-up step against the closed form eta_s / w on a circular binary).
"""
from .oracle import *  # noqa: F401,F403
