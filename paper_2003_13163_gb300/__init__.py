"""GB300 noisy-MPO engine (arXiv:2003.13163, hot path).

Importing the package is cheap: the CUDA library is loaded on first use of
``paper_2003_13163_gb300.mpo`` (see ``load_library``).
"""
__all__ = ["circuits"]
