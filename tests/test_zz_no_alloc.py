"""bf_max_step_size_pairs_noalloc (the allocation-free MaxStepSize over
explicit pairs) against the allocating path: alpha must equal min(1, min of
bf_accd's TOIs) exactly, since both evaluate the same additive CCD in the
same operation order.  Collected last so that it also runs after every
other GPU test in the same process; it passes alone as well."""
import numpy as np
import pytest

from paper_2512_12151_b300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def _pairs(seed, n, spread):
    rng = np.random.default_rng(seed)
    x0 = rng.standard_normal((n, 12)) * 0.1
    x1 = x0 + rng.standard_normal((n, 12)) * spread
    return x0, x1


def _expected(torch, ptype, x0, x1, s):
    n = x0.shape[0]
    toi = torch.zeros(n, dtype=torch.float64, device="cuda")
    B.bf_accd(ptype, x0, x1, s, toi)
    return min(1.0, float(toi.min())) if n else 1.0


def test_noalloc_matches_accd_two_calls(torch_cuda):
    torch = torch_cuda
    alpha = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    B.bf_max_step_size_pairs_noalloc(0, 0, None, None, 0.1, alpha)  # first call: setup only
    assert float(alpha[0]) == 1.0
    # several tiles and a ragged tail; hits (alpha < 1) and no hits (alpha = 1)
    cases = [(0, 5000, 0.12, 1), (1, 4097, 0.12, 2), (0, 300, 1e-4, 3), (1, 129, 0.3, 4), (0, 1, 0.3, 5)]
    for ptype, n, spread, seed in cases:
        x0, x1 = _pairs(seed, n, spread)
        x0 = torch.tensor(x0, device="cuda")
        x1 = torch.tensor(x1, device="cuda")
        ref = _expected(torch, ptype, x0, x1, 0.1)
        for _ in range(2):  # two calls in a row: the shared scratch is reused
            alpha.fill_(-1.0)
            B.bf_max_step_size_pairs_noalloc(ptype, n, x0, x1, 0.1, alpha)
            assert float(alpha[0]) == ref, (ptype, n, float(alpha[0]), ref)
    # a no-hit case (tiny motion far apart) must give exactly 1
    x0 = torch.zeros((64, 12), dtype=torch.float64, device="cuda")
    x0[:, 3:6] = 1.0
    x0[:, 6:9] = torch.tensor([0.0, 1.0, 0.0], dtype=torch.float64)
    x0[:, 0:3] = torch.tensor([0.2, 0.2, 1.0], dtype=torch.float64)
    B.bf_max_step_size_pairs_noalloc(0, 64, x0, x0.clone(), 0.1, alpha)
    assert float(alpha[0]) == 1.0
    # a non-finite coordinate allows no step, wherever the pair sits
    x1 = x0.clone()
    x1[37, 4] = float("nan")
    for _ in range(2):
        alpha.fill_(-1.0)
        B.bf_max_step_size_pairs_noalloc(0, 64, x0, x1, 0.1, alpha)
        assert float(alpha[0]) == 0.0
    B.bf_max_step_size_pairs_noalloc(0, 64, x0, x0.clone(), 0.1, alpha)
    assert float(alpha[0]) == 1.0


def test_noalloc_limits(torch_cuda):
    torch = torch_cuda
    n_max = 1 << 20
    x0, x1 = _pairs(11, n_max + 1, 0.12)  # one pair more than a call may take
    x0 = torch.tensor(x0, device="cuda")
    x1 = torch.tensor(x1, device="cuda")
    alpha = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.bf_max_step_size_pairs_noalloc(1, n_max, x0, x1, 0.1, alpha)
    assert float(alpha[0]) == _expected(torch, 1, x0[:n_max], x1[:n_max], 0.1)
    with pytest.raises(B.BfError):
        B.bf_max_step_size_pairs_noalloc(1, n_max + 1, x0, x1, 0.1, alpha)
    with pytest.raises(B.BfError):
        B.bf_max_step_size_pairs_noalloc(2, 10, x0, x1, 0.1, alpha)
    with pytest.raises(B.BfError):
        B.bf_max_step_size_pairs_noalloc(0, 10, x0, x1, 1.5, alpha)
