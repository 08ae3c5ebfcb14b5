"""GB300-native coupled D2Q9 + D2Q5 central-moment lattice Boltzmann method (arXiv:1710.10569).

Importing the package loads nothing native; ``paper_1710_10569_gb300.clb`` loads libclb.so on first
use and raises if it has not been built (``paper_1710_10569_gb300.build.build()``).
"""
__all__ = ["clb", "workloads", "build"]
