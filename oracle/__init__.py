"""Plain, slow FP64 CPU oracle for Monte Carlo TRG (arXiv:1710.03757).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import, call or run anything in
this package; the product path (the CUDA library and its Python binding) must
never touch it.  It shares no code with the device path.

Modules: philox (uniform stream), ising (site tensor and exact Z),
network (TRG geometry, exact traces), sampler (stochastic truncation),
trg (trajectories), estimator (mean and error bars).
"""
