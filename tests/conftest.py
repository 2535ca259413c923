import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    # temporary files of tests stay inside the repository's build folder
    if not config.option.basetemp:
        config.option.basetemp = os.path.join(ROOT, "_build", "pytest-tmp")
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU oracle runs")
