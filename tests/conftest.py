import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def custom_env(nx=7, ny=7, nt=5, K=1, N=64, L=5, vbar=None, modes=None, sigma=None, seed=1,
               obstacle=None, target=None, actions=None, gbar=None, Y=None, **kw):
    """A small hand-made environment for closed-form checks."""
    from paper_2109_00857_gb300 import inputs
    if vbar is None:
        vbar = np.zeros((nt, ny, nx, 2))
    if modes is None:
        modes = np.zeros((nt, K, ny, nx, 2))
    if sigma is None:
        sigma = np.zeros(K)
    if obstacle is None:
        obstacle = np.zeros((nt, ny, nx), np.uint8)
    if target is None:
        target = np.zeros((ny, nx), np.uint8)
    if actions is None:
        actions = inputs.action_table(16, 1, 1.0)
    return inputs.Environment(nx=nx, ny=ny, nt=nt, K=K, N=N, L=L, vbar=np.asarray(vbar, float),
                              modes=np.asarray(modes, float), sigma=np.asarray(sigma, float),
                              seed=seed, obstacle=np.asarray(obstacle, np.uint8),
                              target=np.asarray(target, np.uint8), actions=np.asarray(actions, float),
                              gbar=gbar, Y=Y, **kw)


@pytest.fixture
def make_env():
    return custom_env
