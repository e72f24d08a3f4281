"""GB300-native PEPS sampling hot path (log|psi|, E_loc, dln psi/dA, gradient).

The compute path is ``libpeps.so`` (CUDA, sm_103a) behind a C ABI; the
Python binding in :mod:`paper_1611_09467_gb300.peps` only marshals arguments.
Importing this package imports nothing else, so :mod:`.inputs` can be used
without the CUDA library.
"""
