"""Seeded synthetic two-sided markets.

This package only draws random inputs: factor matrices, popularity biases and
capacities. It holds none of the IPFP arithmetic, so both the CPU oracle
(``oracle/``) and the CUDA path (``paper_2411_19214_gb300``) can be fed from it
without sharing any of the method's code.
"""

from .markets import (  # noqa: F401
    Market,
    make_market,
    round_to_bf16,
    round_to_e4m3,
    fp8_exponent,
    fp8_row_exponents,
    fp8_quantized,
    fp8_encoded,
    e4m3_bits,
    bf16_bits,
    dense_job_market,
    fused_market,
    plain_dense_market,
    paper_shaped_market,
    batched_market_sizes,
    batched_markets,
    serving_request_sizes,
    serving_workload,
    crowding_market,
)
