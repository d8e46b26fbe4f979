"""adpar: tape-free reverse-mode adjoints of bulk-parallel operators on GB300 (arXiv 2202.10297)."""
