"""Pins of the oracle's implicit-function adjoint (CPU only).

Convention: for a real loss L the gradient with respect to a complex
variable z is dL/dRe z + i dL/dIm z (PyTorch's convention).  Checked:
* on c1 y + c0 = 0 against the closed form and against torch.autograd
  differentiating y = -c0/c1 directly;
* on a tracked 3-variable system against central finite differences in the
  real and imaginary part of every coefficient, each perturbed solution
  re-polished by Newton's method from the unperturbed one.
"""
import numpy as np
import torch

import workloads as W
from oracle import cells


def test_linear_closed_form_and_autograd(oracle_mod):
    c1, c0 = 1.3 - 0.4j, -0.7 + 0.9j
    s = W.LaurentSystem(1, [2], np.array([[1], [0]]), np.array([c1, c0]), np.zeros(2, np.int64))
    osys = oracle_mod.System(s, np.zeros(2, np.int64), 1)
    x = np.array([[-c0 / c1]])
    gc = osys.adjoint(x, 2 * x)               # L = |x|^2 -> gx = 2x
    assert np.allclose(gc[1], 2 * c0 / abs(c1) ** 2, rtol=1e-14)
    assert np.allclose(gc[0], -2 * abs(c0) ** 2 / (abs(c1) ** 2 * np.conj(c1)), rtol=1e-14)
    t1 = torch.tensor(c1, dtype=torch.complex128, requires_grad=True)
    t0 = torch.tensor(c0, dtype=torch.complex128, requires_grad=True)
    L = (-t0 / t1).abs() ** 2
    L.backward()
    assert np.allclose(gc[0], t1.grad.numpy(), rtol=1e-14)
    assert np.allclose(gc[1], t0.grad.numpy(), rtol=1e-14)


def test_finite_differences_of_tracked_solutions(oracle_mod):
    for att in range(40):
        s = W.laurent_system(77, 3, 4, -1, 2, 32, attempt=att)
        try:
            cl, mv = cells.mixed_cells(s)
        except cells.NonGeneric:
            continue
        if mv >= 3:
            break
    P = oracle_mod.Params()
    xs = []
    for c in cl:
        te = cells.t_exponents(s, {"kind": "pairs", "pairs": c["pairs"]})
        osys = oracle_mod.System(s, te["e"], te["D"])
        x, st, _, _ = osys.track(P, cells.start_points(s, c["pairs"]), cells.tau0(te["e"], te["D"]))
        assert (st == oracle_mod.CONVERGED).all()
        xs.append(x)
    x = np.concatenate(xs)
    texp = np.zeros(s.M, np.int64)           # only t = 1 matters below
    base = oracle_mod.System(s, texp, 1)
    gc = base.adjoint(x, 2 * x)

    def loss(coeffs):
        sp = oracle_mod.System(s.with_coeffs(coeffs), texp, 1)
        xp, err = sp.polish(P, x)
        assert np.all(err < 1e-10)
        return float(np.sum(np.abs(xp) ** 2))

    h = 1e-6
    fd = np.zeros(s.M, complex)
    for i in range(s.M):
        for unit in (1.0, 1j):
            cp = s.coeffs.copy()
            cm = s.coeffs.copy()
            cp[i] += h * unit
            cm[i] -= h * unit
            d = (loss(cp) - loss(cm)) / (2 * h)
            fd[i] += d if unit == 1.0 else 1j * d
    assert np.max(np.abs(fd - gc)) < 1e-6 * max(1.0, np.abs(gc).max())
