import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


ALL_BCS = [(0, 0, 0, 0), (0, 1, 0, 0), (1, 1, 1, 1), (1, 0, 0, 1), (0, 0, 1, 0)]
# periodic axes (face type 2 on both faces of the axis), alone and with walls
PERIODIC_BCS = [(2, 2, 2, 2), (2, 2, 0, 0), (2, 2, 1, 0), (0, 1, 2, 2), (1, 1, 2, 2)]
