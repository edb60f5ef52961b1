import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle

    return oracle.load()


@pytest.fixture(autouse=True)
def _nothing_out_of_bounds(request):
    """On the bounds-checked build (TRTR_BOUNDS_CHECK=1), every GPU test must leave the
    kernels' out-of-bounds record empty."""
    yield
    if os.environ.get("TRTR_BOUNDS_CHECK") != "1" or request.node.get_closest_marker("gpu") is None:
        return
    from paper_2312_10316_gb300 import trtr

    assert trtr.trtr_bounds_checked(), "TRTR_BOUNDS_CHECK=1 but the default library is loaded"
    count, kind, i, j = trtr.trtr_bounds_report()
    assert count == 0, f"{count} out-of-bounds accesses; the first of kind {kind} at ({i}, {j})"
