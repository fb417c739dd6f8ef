"""MACT on GB300: minimax-approximant colour-space transforms (RGB -> CIELAB,
HSI, SCT) and 3D-LUT interpolation as hand-written sm_103a CUDA kernels
behind a C ABI (``libmact.so``), with a thin ctypes binding in ``mact``."""
__all__ = ["synth"]
