"""GB300-native MapSQ: MapReduce-based join of SPARQL triple-pattern partial
matches (arXiv 1702.03484) in hand-written sm_103a CUDA kernels behind a C ABI
(``include/mapsq.h``); :mod:`.mapsq` is the Python binding."""
from .mapsq import (  # noqa: F401
    Context, TableRef, MapsqError, JoinOpts, torch_allocator, lib,
    VAR_S, VAR_P, VAR_O, JOIN_AUTO, JOIN_HASH, JOIN_SORTED,
)
