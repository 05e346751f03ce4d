import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _ensure_library():
    # The tests call the library through its C ABI; (re)build it when the
    # sources changed (a no-op when liblbm.so is up to date).
    import __graft_entry__
    __graft_entry__._builder().build()


_ensure_library()


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")
