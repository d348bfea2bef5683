"""GB300-native Fourier pseudo-spectral stepper for the real cubic Klein-Gordon equation.

The compute path lives in the CUDA library ``libkg.so`` (C ABI declared in
``include/kg.h``); :mod:`paper_1501_04552_gb300.kg` is its thin ctypes binding and
:mod:`paper_1501_04552_gb300.inputs` holds the seeded synthetic input generators.
Importing the package does not load the library; importing ``kg`` does, and fails
loudly when it has not been built.
"""
