"""Seeded synthetic genomes and reads shared by the oracle tests, the GPU tests and the bench.

This package holds input generation only: it draws random reference sequences and reads and
returns them as ASCII byte arrays.  It contains none of the read-mapping arithmetic.
"""
from .generate import (  # noqa: F401
    WORKLOADS,
    Reads,
    build,
    counter_u64,
    k_of_length,
    make_reads,
    make_reference,
    make_workload,
    request_stream,
    revcomp_ascii,
    uneven_batches,
    uniform_reference,
)
