"""FP64 CPU oracle for the FOT iteration: test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs
import this package.  The CUDA product path never imports it and shares no code
with it.
"""
