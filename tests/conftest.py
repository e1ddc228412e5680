import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running oracle case")


def pytest_sessionstart(session):
    # compile the library (and the oracle helper) once per session, so a fresh
    # checkout or a freshly provisioned machine can run the suite directly
    import __graft_entry__
    __graft_entry__.build()
