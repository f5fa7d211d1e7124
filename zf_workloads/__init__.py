"""Seeded synthetic column generators shared by the tests, the benchmark and the oracle checks.

This module only draws data.  It holds none of the codec arithmetic: no bit
widths, no references, no run detection, no match finding.  Every value comes
from a counter-based hash (splitmix64 of seed, stream and index), so any row
range can be regenerated on its own and the integer generators give the same
bytes on x86_64 and aarch64.

The shapes follow the workloads the paper evaluates on (TPC-H-like analytical
fact-table columns, Section 5.1): uniform small integers, sorted keys with
geometric gaps, run-heavy date columns, Zipf-distributed low-cardinality codes,
log-normal scaled decimals and space-separated word text.
"""
from .gen import *  # noqa: F401,F403
