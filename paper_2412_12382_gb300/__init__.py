"""GB300 (sm_103a) motif-based community detection (Chen & Tsourakakis,
arXiv 2412.12382): per-edge triangles and wedges, Tectonic / TW / Jaccard / K3 / K4 similarity,
exact-rational pruning and connected components, as hand-written CUDA
kernels behind the C ABI of include/tectonic.h."""
from .tectonic import (  # noqa: F401
    JACCARD, K3, K4, TECTONIC, TW, Graph, TectonicError, load_library, library_path,
)

__version__ = "0.1.0"
