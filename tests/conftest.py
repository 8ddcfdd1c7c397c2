import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# every library context a test closes is first checked for corrupted guard
# bands (out-of-bounds writes by any kernel)
os.environ.setdefault("PRCG_CHECK_GUARDS", "1")
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
