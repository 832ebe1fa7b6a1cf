"""GB300-native (sm_103a) per-timestep short-range force evaluation of the Cr-film /
carbon-indenter nano-indentation MD of Pal et al. (arXiv:1507.07068): cell binning and
Verlet-list rebuild, two-pass EAM (+ M(P) term) for Cr-Cr, Morse for Cr-C, velocity
Verlet -- hand-written CUDA kernels behind the C ABI of include/md.h (libmd.so), with a
thin ctypes binding (md.py).  PyTorch provides the CUDA stream.
"""
from .build_lib import build  # noqa: F401

__all__ = ["build", "md"]
