"""Microbenchmarks that measure the ceilings the rooflines are reported
against (the integer-pipe peaks are not part of the measured peaks).

``python -m paper_2307_06554_gb300.probes`` compiles ``alu_peak.cu`` for
sm_103a, runs it on the current GPU and prints one JSON line with
operations per second per operation kind, plus the SM clock seen.
"""
