"""GB300-native CoRdE Cosserat-rod time stepper (sm_103a CUDA behind a C ABI).

``workloads`` generates seeded synthetic inputs; ``corde`` is the thin ctypes binding of
the C-ABI library ``libcorde.so`` (built from ``csrc/``).  Importing this package does
not load the library; the binding loads it on first use and raises if it is missing.
"""
