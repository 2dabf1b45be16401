"""Seeded synthetic graph generators: the inputs shared by the oracle and the
CUDA path.  This package holds no step of the community-detection method."""
from .csr import csr_from_pairs, num_edges, upper_pairs, dense_adjacency  # noqa: F401
from .rmat import rmat_csr, rmat_samples, feistel, cut_points  # noqa: F401
from .sbm import sbm_csr, planted_partition, block_of  # noqa: F401
