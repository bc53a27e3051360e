import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU checks")


@pytest.fixture(scope="session")
def hsc_problem():
    """The HSC-shaped frame set (4096^2 x 33 exposures, 43 x 43 PSFs, 5%
    masked), drawn once per session: several GPU tests read it whole or crop
    it."""
    import synth
    return synth.make_problem("hsc")
