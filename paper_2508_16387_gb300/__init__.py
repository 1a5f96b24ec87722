"""GB300-native multi-material finite-volume solver (MUSCL + HLLC + FIVER, RK2,
level set) after M2C (arXiv 2508.16387).

The solver is the CUDA C-ABI library ``libm2cgpu.so`` built from ``csrc/``;
``m2c`` is its thin ctypes binding. ``workloads`` holds the seeded synthetic
inputs. Importing the package loads nothing; ``m2c`` loads the library on
first use and fails loudly if it is missing.
"""
__all__ = ["m2c", "workloads"]
