"""Seeded synthetic workloads for the world-cache / screen-probe hot path.

This package is input generation only: box scenes, a pinhole camera, the
G-buffer (normal + distance) it sees, and the probe-ray hit records that the
paper's hardware ray tracing would return (Section 4 lets any caster that
returns hit points stand in).  It holds none of the radiance-caching
arithmetic; the oracle and the CUDA path both read its output unchanged.
"""
from .scene import (  # noqa: F401
    CONFIGS,
    batched_views,
    Camera,
    Frame,
    build_tracer,
    halton_jitter,
    make_frame,
    make_frames,
    make_scene,
    records_random,
    REC_PLANES,
)
from . import surrogate_inputs  # noqa: F401,E402
