"""Seeded synthetic filterbanks for the dedispersion path.

This package makes inputs only: radiometer noise, dispersed and scatter-broadened
pulses averaged over Δt×Δν cells, seeded beam lists and per-channel weight factors.
It holds none of the dedisperser's arithmetic (no delay tables, tap counts, trial-DM
rule, sums or S/N); both the CUDA path's tests and the oracle's tests draw their
inputs from here.
"""
from .filterbank import (  # noqa: F401
    Band,
    MASTER_SEED,
    cell_average_pulse,
    rect_pulse_cells,
    noise_u8,
    noise_f32,
    make_plain,
    make_craft,
    make_diff,
    make_large,
    make_batched_beams,
    spectral_weights,
    sub_seed,
    add_cells,
    make_beam_data,
    gaussian_profile,
    scattered_boxcar_profile,
    PLAIN_BAND,
    CRAFT_BAND,
    LARGE_BAND,
)
