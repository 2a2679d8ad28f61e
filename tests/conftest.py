import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_finish(session):
    # the oracle results of the largest parity cases take minutes: start them
    # now, in the background, when those tests are part of the run
    if session.config.option.collectonly:
        return
    if any("test_gpu_large.py" in item.nodeid for item in session.items):
        import large_cases
        large_cases.start()
