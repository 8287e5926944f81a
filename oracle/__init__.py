"""CPU oracle of the GPZ compressor -- test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this package.
"""
