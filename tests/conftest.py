import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU-only oracle runs")


@pytest.fixture(scope="session")
def sphere8():
    """Oracle system of the sphere scene on an 8^3 grid."""
    import scenes
    from oracle.pipeline import build_system
    sc = scenes.config(0, 8)
    return build_system(sc)


@pytest.fixture(scope="session")
def empty4():
    import scenes
    from oracle.pipeline import build_system
    return build_system(scenes.empty_scene(4), L=2)
