"""Seeded synthetic inputs shared by the tests, the benchmark and the CPU oracle's callers.

Holds no decoder arithmetic: base-graph generation, information bits, GF(2) encoding,
the AWGN channel with its demapper, and LLR quantisation/conversion only.
"""
from .philox import philox4x32, PhiloxStream, seed_key
from .graphs import SHAPES, generate_base_graph, rate_params, expand_H
from .encode import info_bits, encode_structured, encode_gaussian, core_matrix
from .channel import std_normals, modulate_llr, quantize_int8, to_fp16, noise_n0, uniform_ebn0
from .workload import Workload, make_workload

__all__ = [
    "philox4x32", "PhiloxStream", "seed_key", "SHAPES", "generate_base_graph",
    "rate_params", "expand_H", "info_bits", "encode_structured", "encode_gaussian",
    "core_matrix", "std_normals", "modulate_llr", "quantize_int8", "to_fp16", "noise_n0",
    "uniform_ebn0",
    "Workload", "make_workload",
]
