"""GB300-native Monte-Carlo integration of sector-decomposed Feynman integrals.

The method is that of A. V. Smirnov, "FIESTA 4: optimized Feynman integral
calculations with GPU support" (arXiv:1511.03614): sector decomposition, pole
subtraction and eps expansion on the host (``preprocess``), then VEGAS
integration of every (sector, eps order) unit by a persistent CUDA interpreter
of register bytecode (``csrc/fiesta.cu``, C ABI in ``include/fiesta.h``).
"""
from .preprocess import prepare_feynman, prepare_direct, assemble, Prepared, Unit
from .textformat import parse as parse_text

__all__ = ["prepare_feynman", "prepare_direct", "assemble", "Prepared", "Unit", "parse_text", "Integrator"]


def __getattr__(name):
    if name == "Integrator":
        from .api import Integrator
        return Integrator
    raise AttributeError(name)
