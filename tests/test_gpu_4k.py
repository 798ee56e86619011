"""The 4K stress workload at full size (3840x2160, 8.3 M records, 2^24 slots, FP16-packed
resolved radiance), in the launch configuration bench.py --config 5 times: keys, occupancy
and fixed-point sums bit-exact; resolved and interpolated radiance within the FP16 packing
bound; no dropped hits."""
import pytest

import workload as wl

from _gpu_util import require_gpu, run_frames
from test_gpu_cache import _frames_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def test_4k_cache_four_frames_fp16():
    # four frames of the moving camera: the EMA blends revisited cells at full size
    scene = wl.make_scene(5)
    frames = [wl.make_frame(5, f, scene) for f in (0, 1, 2, 3)]
    bound = 2.0 ** -11 * sum(0.9 ** j for j in range(len(frames))) + 1e-4
    _frames_parity(5, frames, resolved_format=1, value_rel=bound)


def test_4k_chain_one_frame_fp16():
    scene = wl.make_scene(5)
    # one rounding to half (2^-11) of every radiance the probes read, plus the float32 path
    run_frames(5, [wl.make_frame(5, 0, scene)], rel=2.0 ** -10, resolved_format=1)
