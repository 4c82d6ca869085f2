"""Seeded synthetic inputs for the KT viscous-hydro step.

This package only *generates inputs*: problem parameters, initial states, the equation-of-state
table (Sec. 2.3 style tabulation of a given c_s^2(T)) and the Gubser-flow state used as an
initial condition.  It holds none of the KT scheme's arithmetic, so both the CUDA path and the
CPU oracle may use it.  All quantities are in fm units (hbar = c = 1): e, P, pi, Pi in fm^-4,
T in fm^-1, tau and x in fm.
"""
from .problem import Problem, HBARC  # noqa: F401
