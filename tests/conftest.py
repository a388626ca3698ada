import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def c1_matrix():
    """The 2000-series x 512-step five-class set at w = 51 (the benchmark workload): the
    GPU matrix in the benchmark's launch configuration, and the oracle's float mirror and
    float64 value of every one of its 1,999,000 pairs (OpenMP over the host's cores)."""
    import numpy as np
    import torch

    import oracle
    from paper_2307_04904_gb300 import api, synth

    values, offsets, _ = synth.five_class_set(2000, 512, seed=1)
    D = api.dtw_pairwise(torch.from_numpy(values).cuda(), torch.from_numpy(offsets).cuda(), 51)
    torch.cuda.synchronize()
    a, b = np.triu_indices(2000, 1)
    return dict(values=values, offsets=offsets, D=D.cpu().numpy(), a=a, b=b,
                mirror=oracle.pairs_f32_mirror(values, offsets, a, b, 51),
                ref=oracle.pairs(values, offsets, a, b, 51))
