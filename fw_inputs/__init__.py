"""Seeded synthetic inputs for the random-walk library and its oracle.

This package holds only input generation: graphs (Chung-Lu, R-MAT), edge
attributes (weights, labels) and query start vertices.  It contains none of
the walk method's arithmetic (no transition weights, no sampling, no walk
random numbers), so both the CUDA path and the CPU oracle may consume what it
produces without sharing any of the method's code.

Every random choice is a counter-based hash of (seed, index), evaluated with
integer torch ops, so a graph comes out identical on CPU and on a GPU and does
not depend on chunking or thread count.
"""

from .graphs import (  # noqa: F401
    Graph,
    chung_lu,
    rmat,
    one_per_vertex,
    random_starts,
    uniform_lengths,
    mix32,
)
