"""Pins for the oracle's real spherical harmonics, coupling tensors, Bessel
basis and cutoff envelope (Sec. 2.1 irreducible-representation reading)."""
import math

import numpy as np
import pytest
import torch
from scipy.special import eval_legendre, sph_harm_y
from sympy.physics.quantum.cg import CG

from oracle.model import bessel, envelope
from oracle.sph import coupling_paths, real_cg, sh_real

RNG = np.random.default_rng(123)


def _unit(n):
    v = RNG.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _Y(v, lmax=2):
    return [t.numpy() for t in sh_real(torch.tensor(v), lmax)]


def test_sh_component_normalisation():
    Y = _Y(_unit(50))
    for l, Yl in enumerate(Y):
        np.testing.assert_allclose((Yl ** 2).sum(-1), 2 * l + 1, rtol=1e-13)


def test_sh_addition_theorem():
    a, b = _unit(40), _unit(40)
    Ya, Yb = _Y(a), _Y(b)
    cos = (a * b).sum(-1)
    for l in range(3):
        np.testing.assert_allclose((Ya[l] * Yb[l]).sum(-1),
                                   (2 * l + 1) * eval_legendre(l, cos), atol=1e-12)


def test_sh_matches_scipy_complex_harmonics():
    """Real Y_lm = sqrt(4 pi) * {sqrt2 (-1)^m Im Y_l^|m| (m<0); Y_l^0; sqrt2 (-1)^m Re Y_l^m (m>0)}."""
    v = _unit(30)
    theta = np.arccos(np.clip(v[:, 2], -1, 1))
    phi = np.arctan2(v[:, 1], v[:, 0])
    Y = _Y(v)
    for l in range(3):
        for m in range(-l, l + 1):
            c = sph_harm_y(l, abs(m), theta, phi)
            if m < 0:
                ref = math.sqrt(2) * (-1) ** m * c.imag
            elif m == 0:
                ref = c.real
            else:
                ref = math.sqrt(2) * (-1) ** m * c.real
            np.testing.assert_allclose(Y[l][:, m + l], math.sqrt(4 * math.pi) * ref, atol=1e-12)


def test_paths_and_nonzeros():
    p2 = coupling_paths(2)
    assert p2 == [(0, 0, 0), (0, 1, 1), (0, 2, 2), (1, 0, 1), (1, 1, 0), (1, 1, 2),
                  (1, 2, 1), (2, 0, 2), (2, 1, 1), (2, 2, 0), (2, 2, 2)]
    assert coupling_paths(1) == [(0, 0, 0), (0, 1, 1), (1, 0, 1), (1, 1, 0)]
    nnz = sum(int((np.abs(real_cg(*p)) > 1e-12).sum()) for p in p2)
    assert nnz == 83
    assert sum(int((np.abs(real_cg(*p)) > 1e-12).sum()) for p in coupling_paths(1)) == 10


def _wigner_D(R, l, npts=64):
    """D_l(R) from the SH themselves by least squares: Y_l(R x) = D Y_l(x)."""
    x = _unit(npts)
    A = _Y(x)[l]
    Bm = _Y(x @ R.T)[l]
    D, *_ = np.linalg.lstsq(A, Bm, rcond=None)
    return D.T


def _rand_rot():
    q = RNG.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


@pytest.mark.parametrize("path", coupling_paths(2))
def test_cg_equivariance(path):
    l1, l2, l3 = path
    C = real_cg(*path)
    for _ in range(5):
        R = _rand_rot()
        if RNG.random() < 0.5:
            R = -R                                   # improper: inversion included
        D1, D2, D3 = (_wigner_D(R, l) for l in (l1, l2, l3))
        a = RNG.normal(size=2 * l1 + 1)
        b = RNG.normal(size=2 * l2 + 1)
        lhs = D3 @ np.einsum("abc,a,b->c", C, a, b)
        rhs = np.einsum("abc,a,b->c", C, D1 @ a, D2 @ b)
        np.testing.assert_allclose(lhs, rhs, atol=1e-11)


@pytest.mark.parametrize("path", coupling_paths(2))
def test_cg_norm_sign_and_sympy_centre(path):
    l1, l2, l3 = path
    C = real_cg(*path)
    assert abs(np.linalg.norm(C) - 1.0) < 1e-13
    ref = abs(float(CG(l1, 0, l2, 0, l3, 0).doit())) / math.sqrt(2 * l3 + 1)
    assert ref > 0
    np.testing.assert_allclose(C[l1, l2, l3], ref, rtol=1e-12)


def test_cg_special_cases():
    for l in range(3):
        np.testing.assert_allclose(real_cg(0, l, l)[0], np.eye(2 * l + 1) / math.sqrt(2 * l + 1), atol=1e-14)
        np.testing.assert_allclose(real_cg(l, 0, l)[:, 0, :], np.eye(2 * l + 1) / math.sqrt(2 * l + 1), atol=1e-14)
    np.testing.assert_allclose(real_cg(1, 1, 0)[:, :, 0], np.eye(3) / math.sqrt(3), atol=1e-14)


# ---- parity-odd coupling paths (full O(3)) ----

def test_odd_paths():
    assert coupling_paths(2, parity="odd") == [(1, 1, 1), (1, 2, 2), (2, 1, 2), (2, 2, 1)]
    assert coupling_paths(1, parity="odd") == [(1, 1, 1)]
    assert coupling_paths(0, parity="odd") == []
    assert sorted(coupling_paths(2, parity="all")) == sorted(coupling_paths(2) + coupling_paths(2, parity="odd"))
    assert not [p for p in coupling_paths(2, parity="odd") if p[2] == 0]   # no odd path into l = 0


def _yzx(v):
    """Cartesian vector -> the l = 1 component order (y, z, x)."""
    return np.array([v[1], v[2], v[0]])


def test_odd_cg_cross_product_closed_form():
    """C^{111}(a, b) = (a x b) / sqrt(6) in the (y, z, x) order (Levi-Civita,
    Frobenius norm 1, first nonzero entry C[y, z, x] = +1/sqrt(6))."""
    C = real_cg(1, 1, 1)
    for _ in range(5):
        a, b = RNG.normal(size=3), RNG.normal(size=3)
        got = np.einsum("abc,a,b->c", C, _yzx(a), _yzx(b))
        np.testing.assert_allclose(got, _yzx(np.cross(a, b)) / math.sqrt(6.0), atol=1e-14)


def test_odd_cg_221_closed_form():
    """Y_2(u), Y_2(v) are the traceless parts of u u^T, v v^T; the only vector
    bilinear in two such tensors, odd under inversion, is the axial vector of
    the antisymmetric part of their product, eps_ijk (A B)_jk = (u . v) (u x v):
    C^{221}(Y_2(u), Y_2(v)) = kappa (u . v) (u x v) with one constant kappa."""
    C = real_cg(2, 2, 1)
    ratios = []
    for _ in range(6):
        u, v = _unit(2)
        Yu, Yv = _Y(u[None], 2)[2][0], _Y(v[None], 2)[2][0]
        got = np.einsum("abc,a,b->c", C, Yu, Yv)
        ref = _yzx(np.dot(u, v) * np.cross(u, v))
        k = np.dot(got, ref) / np.dot(ref, ref)
        np.testing.assert_allclose(got, k * ref, atol=1e-12)
        ratios.append(k)
    assert np.ptp(ratios) < 1e-12 and abs(ratios[0]) > 0.1


@pytest.mark.parametrize("path", coupling_paths(2, parity="odd"))
def test_odd_cg_pseudotensor_sign_norm_and_sign_rule(path):
    """Proper rotations: D3 C(a, b) = C(D1 a, D2 b); improper ones (with the
    D_l taken from the harmonics, D_l(-R) = (-1)^l D_l(R)): the opposite sign,
    since (-1)^(l1 + l2) = -(-1)^l3 on an odd path.  Together with Frobenius
    norm 1 and the first-nonzero sign rule this fixes the tensor (the
    equivariant bilinear map of a triple (l1, l2, l3) is unique up to scale)."""
    l1, l2, l3 = path
    C = real_cg(*path)
    assert abs(np.linalg.norm(C) - 1.0) < 1e-13
    assert C.ravel()[np.flatnonzero(np.abs(C.ravel()) > 1e-12)[0]] > 0
    for k in range(6):
        R = _rand_rot()
        sign = 1.0
        if k % 2:
            R, sign = -R, -1.0
        D1, D2, D3 = (_wigner_D(R, l) for l in (l1, l2, l3))
        a = RNG.normal(size=2 * l1 + 1)
        b = RNG.normal(size=2 * l2 + 1)
        lhs = D3 @ np.einsum("abc,a,b->c", C, a, b)
        rhs = np.einsum("abc,a,b->c", C, D1 @ a, D2 @ b)
        np.testing.assert_allclose(lhs, sign * rhs, atol=1e-11)
        assert np.abs(rhs).max() > 1e-3


def test_bessel_closed_form():
    d = torch.tensor([0.3, 1.7, 3.9], dtype=torch.float64)
    B = bessel(d, 4.0, 8).numpy()
    for a, dv in enumerate(d.numpy()):
        for n in range(1, 9):
            ref = math.sqrt(2 / 4.0) * math.sin(n * math.pi * dv / 4.0) / dv
            assert abs(B[a, n - 1] - ref) < 1e-14


def test_envelope_closed_form_and_c2_at_cutoff():
    d = torch.tensor([0.0, 2.0, 5.0], dtype=torch.float64, requires_grad=True)
    u = envelope(d, 5.0, 6)
    x = 0.4
    assert abs(float(u[0]) - 1.0) < 1e-15
    assert abs(float(u[1]) - (1 - 28 * x ** 6 + 48 * x ** 7 - 21 * x ** 8)) < 1e-15
    (g,) = torch.autograd.grad(u.sum(), d, create_graph=True)
    (h,) = torch.autograd.grad(g.sum(), d)
    assert abs(float(u[2])) < 1e-13 and abs(float(g[2])) < 1e-12 and abs(float(h[2])) < 1e-11
