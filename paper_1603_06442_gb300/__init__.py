"""GB300-native Dirac quantum walk (arXiv:1603.06442): CUDA kernels behind a C ABI.

``binding`` is the ctypes layer over libqw.so (include/qw.h); ``inputs`` holds
the seeded synthetic input generators; ``build`` compiles the library.
"""

from . import binding  # noqa: F401
from .binding import Plan, QwError  # noqa: F401
