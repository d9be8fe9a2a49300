"""The usage example of the README, as a test: the mixed-cell search on the
CPU (one cell, mixed volume 3) and, on the GPU, the track of its start
points (three converged solutions that solve the system to rounding)."""
import numpy as np
import pytest
import torch

N, M_SIZES = 2, [3, 3]
EXPONENTS = np.array([[2, 0], [0, 1], [0, 0],
                      [1, 1], [1, 0], [0, 0]])


def _data():
    rng = np.random.default_rng(0)
    coeffs = np.exp(2j * np.pi * rng.random(6))
    lifting = rng.integers(0, 1 << 20, size=6)
    return coeffs, lifting


@pytest.fixture(scope="module")
def hpt_host():
    from paper_2111_14317_gb300 import build
    build.build()
    from paper_2111_14317_gb300 import hpt
    return hpt


def test_readme_cells(hpt_host):
    coeffs, lifting = _data()
    cells, mv = hpt_host.mixed_cells(N, M_SIZES, EXPONENTS, lifting)
    assert len(cells) == 1 and mv == 3


@pytest.mark.gpu
def test_readme_track(hpt):
    coeffs, lifting = _data()
    cells, mv = hpt.mixed_cells(N, M_SIZES, EXPONENTS, lifting)
    sols = []
    for pairs in cells:
        h = hpt.System(N, M_SIZES, EXPONENTS, coeffs, lifting, {"kind": "pairs", "pairs": pairs}, hpt.HPT_MIXED)
        y0, count = hpt.binomial_start_device(N, M_SIZES, EXPONENTS, coeffs, pairs)
        x, status, steps = h.track(y0, hpt.Params(tol_accept=3e-3))
        sols.append(x[status == hpt.CONVERGED].cpu().numpy())
    x = np.concatenate(sols)
    assert x.shape[0] == mv
    F = np.stack([coeffs[0] * x[:, 0] ** 2 + coeffs[1] * x[:, 1] + coeffs[2],
                  coeffs[3] * x[:, 0] * x[:, 1] + coeffs[4] * x[:, 0] + coeffs[5]], 1)
    assert np.abs(F).max() < 1e-12
