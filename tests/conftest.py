import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line('markers', 'gpu: needs a CUDA GPU (GB300, sm_103a)')
    config.addinivalue_line('markers', 'slow: long CPU or GPU case')


@pytest.fixture(scope='session')
def sq():
    """The CUDA library's Python binding with a context on cuda:0."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    from paper_1411_2223_gb300 import sq as sqmod
    ctx = sqmod.Context(device=0)
    yield ctx
    ctx.close()
