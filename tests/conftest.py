import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU test")


def _ensure_library():
    """Build the in-tree CUDA library (incremental: only stale objects are recompiled) so the
    ABI tests find it even when the suite runs before an explicit build step."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_mtp_build", os.path.join(ROOT, "paper_1906_11029_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build(verbose=False)


_ensure_library()
