"""GB300-native PLDS: batch-dynamic (2+eps)-approximate k-core (coreness) maintenance.

Importing the package loads nothing native; ``paper_2106_03824_gb300.plds`` holds the
C-ABI binding, ``paper_2106_03824_gb300.workloads`` the seeded input generators.
"""
__all__ = ["plds", "workloads"]
