import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")


def pytest_collection_modifyitems(config, items):
    # GPU tests are skipped, not failed, when no GPU is present and the run
    # did not select them explicitly with -m gpu.
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    selected = config.getoption("-m") or ""
    if "gpu" in selected and "not gpu" not in selected:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(scope="session")
def tiny():
    """The small workload: 10k x 128 mixture, oracle rotation and k-means."""
    import synth
    from oracle import ivf, pca
    X, Q, T, cfg = synth.workload("tiny")
    mu, R, lam = pca.train_rotation(X)
    Xr = pca.rotate(X, mu, R)
    init = np.random.default_rng(7).choice(len(X), cfg["nlist"], replace=False)
    C, a, objs = ivf.kmeans(Xr, init, 8)
    return dict(X=X, Q=Q, T=T, cfg=cfg, mu=mu, R=R, lam=lam, C=C, assign=a, objs=objs)
