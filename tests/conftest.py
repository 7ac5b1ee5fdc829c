import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


def load_chi(name):
    """Solvent susceptibility table written by tests/golden/make_golden.py (oracle only)."""
    d = np.load(os.path.join(GOLDEN, "chi_%s.npz" % name))
    return d["chi"], float(d["dk"])


@pytest.fixture(scope="session")
def water3():
    from paper_2403_01039_gb300 import synth
    s = synth.water_3site()
    chi, dk = load_chi("water3")
    s.update(chi=chi, dk=dk)
    return s


@pytest.fixture(scope="session")
def water3_drism():
    """3-site water with X from the oracle's DRISM (the sphere_32 workload's solvent)."""
    from paper_2403_01039_gb300 import synth
    s = synth.water_3site()
    chi, dk = load_chi("water3_drism")
    s.update(chi=chi, dk=dk)
    return s


@pytest.fixture(scope="session")
def water_nacl():
    from paper_2403_01039_gb300 import synth
    s = synth.water_nacl_5site()
    chi, dk = load_chi("water_nacl")
    s.update(chi=chi, dk=dk)
    return s
