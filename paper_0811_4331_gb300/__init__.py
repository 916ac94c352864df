"""GB300 adaptive-multigrid Wilson-Dirac solver (package stub)."""
