import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    # the batch autotuner's cache goes to a file of this session, not $HOME
    import tempfile
    os.environ.setdefault("STARMAP_TUNE_CACHE", os.path.join(tempfile.gettempdir(), f"starmap_tune_{os.getpid()}.txt"))
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")
