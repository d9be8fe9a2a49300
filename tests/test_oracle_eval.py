"""Pins of the oracle's homotopy evaluation (CPU only).

Each check ties the oracle to something other than itself:
* central finite differences in y_j (along 1 and i: holomorphy) and in tau;
* the log-coordinate GEMM formulation of Section 5 (eqs. (6)-(8) and the
  extended Jacobian e^{Z A} B_k^T), written here with numpy -- a different
  algorithm from the oracle's repeated multiplication;
* H(y, t=1) = F(y) (Section 2, below eq. (1)) with numpy powers;
* numpy.polyval / numpy.polyder for a single variable;
* the t -> 0 limit: only a cell's two terms survive.
"""
import numpy as np
import pytest

import workloads as W
from oracle import cells


def _system(seed, n, m, lo=-2, hi=2, lift=16):
    s = W.laurent_system(seed, n, m, lo, hi, lift)
    texp = np.random.default_rng(seed).integers(0, 9, size=s.M)
    return s, texp


def _rel(a, b, scale):
    return float(np.max(np.abs(a - b) / np.maximum(scale, 1e-300)))


@pytest.mark.parametrize("n,m,D", [(1, 4, 1), (3, 4, 1), (4, 5, 3), (6, 7, 2)])
def test_finite_differences(oracle_mod, n, m, D):
    s, texp = _system(10 + n, n, m)
    osys = oracle_mod.System(s, texp, D)
    y, _ = W.random_points(3, 5, n)
    tau = np.linspace(-1.5, -0.1, 5)
    H, Hy, Ht = osys.eval(y, tau)
    SH, SHy, SHt = osys.scale(y, tau)
    for j in range(n):
        for direction in (1.0, 1j):
            h = 1e-5 * np.abs(y[:, j])
            e = np.zeros((5, n), complex)
            e[:, j] = h * direction
            Hp, _, _ = osys.eval(y + e, tau)
            Hm, _, _ = osys.eval(y - e, tau)
            fd = (Hp - Hm) / (2 * h[:, None] * direction)
            assert _rel(fd, Hy[:, :, j], SHy[:, :, j] + 1e-3 * SH) < 1e-7
    h = 1e-5
    Hp, _, _ = osys.eval(y, tau + h)
    Hm, _, _ = osys.eval(y, tau - h)
    assert _rel((Hp - Hm) / (2 * h), Ht, SHt + 1e-3 * SH) < 1e-7


def _log_form(s, texp, D, y, tau):
    """Section 5: z = log y, W = [z, tau] A_hat, E = exp(W),
    [D_z h_k | D_tau h_k | h_k] = E[:, S_k] B_k^T with
    B_k = [A_hat diag(c_k); c_k^T]."""
    p, n = y.shape
    Z = np.concatenate([np.log(y), tau[:, None]], axis=1)           # p x (n+1)
    Ahat = np.concatenate([s.exponents.T.astype(float), (np.asarray(texp) / D)[None, :]], 0)
    E = np.exp(Z @ Ahat)                                             # p x M
    out = np.zeros((p, n, n + 2), complex)
    for k in range(n):
        o, mk = s.offsets[k], s.m[k]
        ck = s.coeffs[o:o + mk]
        Bk = np.concatenate([Ahat[:, o:o + mk] * ck[None, :], ck[None, :]], 0)  # (n+2) x mk
        out[:, k, :] = E[:, o:o + mk] @ Bk.T
    return out


@pytest.mark.parametrize("n,m,D", [(2, 3, 1), (4, 5, 1), (5, 6, 4), (16, 32, 1)])
def test_log_coordinate_gemm_identity(oracle_mod, n, m, D):
    s, texp = _system(20 + n, n, m, -3, 3)
    osys = oracle_mod.System(s, texp, D)
    y, t = W.random_points(4, 64, n)
    tau = np.log(t)
    H, Hy, Ht = osys.eval(y, tau)
    SH, SHy, SHt = osys.scale(y, tau)
    ext = _log_form(s, texp, D, y, tau)
    # d h / d z_j = y_j d h / d y_j
    assert _rel(ext[:, :, :n], Hy * y[:, None, :], SHy * np.abs(y)[:, None, :] + 1e-12) < 1e-12
    assert _rel(ext[:, :, n], Ht, SHt + 1e-300) < 1e-12
    assert _rel(ext[:, :, n + 1], H, SH) < 1e-12


def test_target_system_at_t_equal_one(oracle_mod):
    s, texp = _system(7, 3, 5)
    osys = oracle_mod.System(s, texp, 1)
    y, _ = W.random_points(8, 10, 3)
    H, _, _ = osys.eval(y, np.zeros(10))
    SH, _, _ = osys.scale(y, np.zeros(10))
    F = np.zeros((10, 3), complex)
    for k in range(3):
        o = s.offsets[k]
        for i in range(s.m[k]):
            a = s.exponents[o + i]
            F[:, k] += s.coeffs[o + i] * np.prod(y ** a[None, :], axis=1)
    assert _rel(F, H, SH) < 1e-13


def test_single_variable_polyval(oracle_mod):
    rng = np.random.default_rng(5)
    deg = np.array([0, 1, 3, 4, 6])
    c = np.exp(2j * np.pi * rng.uniform(size=5))
    texp = np.array([5, 0, 2, 0, 7])
    s = W.LaurentSystem(1, [5], deg[:, None], c, np.zeros(5, np.int64))
    osys = oracle_mod.System(s, texp, 2)
    y = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    tau = -rng.uniform(0, 2, 7)
    H, Hy, Ht = osys.eval(y[:, None], tau)
    for q in range(7):
        poly = np.zeros(7, complex)
        dpoly = np.zeros(7, complex)
        for i in range(5):
            ts = np.exp(texp[i] / 2 * tau[q])
            poly[6 - deg[i]] += c[i] * ts
            dpoly[6 - deg[i]] += c[i] * ts * texp[i] / 2
        assert abs(H[q, 0] - np.polyval(poly, y[q])) < 1e-12 * (1 + abs(H[q, 0]))
        assert abs(Hy[q, 0, 0] - np.polyval(np.polyder(poly), y[q])) < 1e-11 * (1 + abs(Hy[q, 0, 0]))
        assert abs(Ht[q, 0] - np.polyval(dpoly, y[q])) < 1e-12 * (1 + abs(Ht[q, 0]))


def test_t_to_zero_leaves_the_cell(oracle_mod):
    s = W.config1(0)
    cl, _ = cells.mixed_cells(s)
    pairs = cl[0]["pairs"]
    te = cells.t_exponents(s, {"kind": "pairs", "pairs": pairs})
    osys = oracle_mod.System(s, te["e"], te["D"])
    y, _ = W.random_points(9, 6, 2)
    H, _, _ = osys.eval(y, np.full(6, -400.0))
    for k in range(2):
        o = s.offsets[k]
        a0, a1 = s.exponents[o + pairs[k][0]], s.exponents[o + pairs[k][1]]
        b = (s.coeffs[o + pairs[k][0]] * np.prod(y ** a0, axis=1)
             + s.coeffs[o + pairs[k][1]] * np.prod(y ** a1, axis=1))
        assert np.allclose(H[:, k], b, rtol=1e-13, atol=1e-13)


def _scale_numpy(s, texp, D, y, tau):
    """The componentwise tolerance scales written out term by term with numpy
    powers (no repeated multiplication, no logarithms): for every term
    c y^a t^s of h_k, |c| |y^a| t^s for H, |c a_j| |y^(a - e_j)| t^s for
    dH/dy_j and |c s| |y^a| t^s for dH/dtau (t = e^tau is real and positive)."""
    p, n = y.shape
    SH = np.zeros((p, n))
    SHy = np.zeros((p, n, n))
    SHt = np.zeros((p, n))
    for k in range(n):
        o = s.offsets[k]
        for i in range(s.m[k]):
            a = s.exponents[o + i].astype(float)
            sx = texp[o + i] / D
            c = abs(s.coeffs[o + i])
            mono = np.abs(np.prod(y ** a[None, :], axis=1))
            ts = np.exp(sx * tau)
            SH[:, k] += c * mono * ts
            SHt[:, k] += c * abs(sx) * mono * ts
            for j in range(n):
                if a[j] != 0:
                    SHy[:, k, j] += c * abs(a[j]) * mono / np.abs(y[:, j]) * ts
    return SH, SHy, SHt


def _signed_system(seed, n, m):
    """A system whose t-exponents take both signs, so that every |.| of the
    scales matters."""
    s = W.laurent_system(seed, n, m, -3, 3, 16)
    rng = np.random.default_rng(seed + 1)
    texp = rng.integers(-8, 9, size=s.M)
    # coefficient magnitudes other than 1, so that |c| matters too
    s = W.LaurentSystem(s.n, s.m, s.exponents, s.coeffs * rng.uniform(0.25, 4.0, s.M), s.lifting)
    return s, texp


def _check_scale(osys, s, texp, D, n, seed):
    y, t = W.random_points(seed, 48, n)
    tau = np.log(t)
    SH, SHy, SHt = osys.scale(y, tau)
    RH, RHy, RHt = _scale_numpy(s, texp, D, y, tau)
    for got, ref in ((SH, RH), (SHy, RHy), (SHt, RHt)):
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref) / np.maximum(ref, 1e-300)) < 1e-12


@pytest.mark.parametrize("n,m,D", [(2, 3, 1), (4, 5, 3), (7, 9, 2), (16, 32, 1)])
def test_scale_is_the_sum_of_term_magnitudes(oracle_mod, n, m, D):
    """ora_scale (the denominator of every parity tolerance: the sums of term
    magnitudes of Section 5's extended Jacobian entries) against numpy."""
    s, texp = _signed_system(30 + n, n, m)
    _check_scale(oracle_mod.System(s, texp, D), s, texp, D, n, 5 + n)


# Mistakes planted in a copy of the oracle's C core, each in the scale sums:
# the pin above must reject every one of them.
_SCALE_MUTANTS = [
    ("dropped |s|", "ht += c * fabs(sexp) * mono * ts;", "ht += c * sexp * mono * ts;"),
    ("dropped t^s", "h += c * mono * ts;\n            ht += c * fabs", "h += c * mono;\n            ht += c * fabs"),
    ("dropped |a_j|", "SHy[k * n + j] += c * fabs((double)a[j])", "SHy[k * n + j] += c * ((double)a[j])"),
    ("y^a for y^(a - e_j)", "cabs(powprod(n, y, yinv, a, j)) * ts;", "cabs(powprod(n, y, yinv, a, -1)) * ts;"),
    ("|c| dropped", "const double c = cabs(coef_at(s, idx));", "const double c = 1.0;"),
]


@pytest.mark.parametrize("name,old,new", _SCALE_MUTANTS, ids=[m[0] for m in _SCALE_MUTANTS])
def test_scale_pin_rejects_planted_mistakes(oracle_mod, tmp_path, name, old, new):
    import ctypes
    import subprocess
    src = open(oracle_mod._SRC).read()
    assert src.count(old) == 1, name
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(lib),
                    str(mut), "-lm"], check=True)
    mlib = ctypes.CDLL(str(lib))
    mlib.ora_scale.restype = ctypes.c_int
    saved = oracle_mod._lib
    oracle_mod._lib = mlib
    try:
        s, texp = _signed_system(34, 4, 5)
        with pytest.raises(AssertionError):
            _check_scale(oracle_mod.System(s, texp, 3), s, texp, 3, 4, 9)
    finally:
        oracle_mod._lib = saved
