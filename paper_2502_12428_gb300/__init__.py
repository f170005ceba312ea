"""GB300-native engine for quasi-F-split (Artin-Mazur) heights of quartic K3 surfaces over F_p.

Importing this package loads nothing native; ``paper_2502_12428_gb300.qfs`` binds the CUDA library.
"""
__all__ = ["inputs", "qfs"]
