"""GB300-native split pressure-gradient projection (Poblador-Ibanez & Sirignano,
arXiv 2103.01874, Sec. 5.4, Eqs. (32)-(34)).

Submodules:
  fields  -- seeded synthetic two-phase inputs (no solver arithmetic)
  ppe     -- ctypes binding of the C-ABI library libppe.so (device kernels)
  build   -- in-tree nvcc build of libppe.so for sm_103a
  serve   -- continuous-batching request loop (HBM-budget admission, slot streams)
  autotune -- launch-shape and schedule search per grid class, cached in JSON
  split_study -- multi-step accuracy of the split pressure gradient

Importing the package loads nothing native; `ppe` loads the library on first use
and raises if it is missing.
"""
__all__ = ["fields", "ppe", "build"]
