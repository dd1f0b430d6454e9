"""GB300-native CP-ALS-QR (restructured dimension tree + customised Q0 extrapolation).

The compute path is the C-ABI library ``libcpqr.so`` built from ``csrc/``;
``binding`` marshals arguments to it.  Importing this package does not load
the library; the first call into ``binding`` does, and fails loudly if the
library is missing.
"""
