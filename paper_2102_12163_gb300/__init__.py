"""GB300 implementation of the MR-LBM adaptive step (arXiv 2102.12163)."""
