"""GB300-native CTF-MNMF-ISS: a C-ABI CUDA library and its Python binding.

Importing the package does not load the CUDA library; ``paper_2510_02382_gb300.api``
does, and raises if it has not been built.
"""
__all__ = ["synth"]
