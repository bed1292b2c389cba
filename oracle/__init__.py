"""Plain CPU FP64 oracle for MACH.  Test infrastructure only: import it from
tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg, nowhere else."""
