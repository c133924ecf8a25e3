import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def water_weights():
    from paper_2410_22867_gb300 import synth
    return synth.water_weights(1001)


@pytest.fixture(scope="session")
def water_oracle(water_weights):
    import oracle
    return oracle.Model(water_weights.to_blob())


@pytest.fixture(scope="session")
def water64():
    from paper_2410_22867_gb300 import synth
    return synth.water_box(64, 0)
