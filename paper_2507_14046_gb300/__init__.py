"""GB300-native D²IP fitting path (deep dynamic image prior for 3D time-sequence EIT).

Submodules:
  synth    -- seeded synthetic workloads (sensitivity matrix, phantoms, measurements,
              input noise, Kaiming initial weights); pure NumPy, no method arithmetic.
  binding  -- ctypes binding of the C-ABI library ``libd2ip.so`` (argument marshalling only).
  build    -- compiles the CUDA library for sm_103a.

Importing this package does not load the CUDA library; ``binding`` does, and fails loudly
when it is missing.
"""
