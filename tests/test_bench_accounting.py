"""Host-side accounting of bench.py (no GPU): how many separate diffusion
launches a Strang step makes and the algorithmic bytes they move."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def test_diffusion_launches_per_step():
    # l = 1 with the step-I sub-step inside the reaction launch: the one
    # separate launch is the synchronising sub-step of step III
    assert bench.diffusion_launch_work(1, True, 16.0, 17.0) == (1, 33.0)
    # l = 1 without fusion: step I's sub-step has its own launch
    assert bench.diffusion_launch_work(1, False, 16.0, 17.0) == (2, 49.0)
    # l = 3 (the sheet): 2 + 3 launches fused, 6 without; one synchronises
    assert bench.diffusion_launch_work(3, True, 16.0, 17.0) == (5, 97.0)
    assert bench.diffusion_launch_work(3, False, 16.0, 17.0) == (6, 113.0)
