"""GB300-native Nystrom high-dimensional kernel filtering (Nair & Chaudhury, arXiv 1901.06112)."""
