"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This package only builds circuits (gate lists with their angles) and bit
strings from splitmix64 streams.  It holds none of the method's arithmetic:
no gate matrices, no propagation and no amplitudes.  Both the oracle and the
library convert these neutral records into their own representations.
"""
from .mlp_init import mlp_init_params  # noqa: F401
from .circuits import (  # noqa: F401
    Gate, Circuit, Workload, SplitMix64,
    qft, amplitude_amplification, qaoa_maxcut, quantum_walk,
    three_qubit_example, four_qubit_figure, placement_figure, random_small_circuit,
    qft_workload, qft_signal_workload, aa_workload, qaoa_workload, qw_workload,
    random_regular_graph, bits_to_int, int_to_bits,
)
