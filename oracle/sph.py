"""Real spherical harmonics and real-basis Clebsch-Gordan coupling tensors.

Sec. 2.1 of the paper builds the energy from "tensors up to rank l and tensor
products using their irreducible representations" without fixing a basis; the
reading used here:

  * Real spherical harmonics in component normalisation (sum_m Y_lm^2 = 2l+1),
    ordered m = -l .. l:
        Y_0 = 1
        Y_1 = sqrt(3) (y, z, x)
        Y_2 = (sqrt(15) xy, sqrt(15) yz, sqrt(5)/2 (3z^2 - 1), sqrt(15) xz,
               sqrt(15)/2 (x^2 - y^2))
  * Coupling tensors C^{l1 l2 l3}[m1, m2, m3] are the complex Clebsch-Gordan
    coefficients (Racah's closed formula) carried into this real basis by the
    unitary complex-to-real change of basis, normalised to Frobenius norm 1,
    with the sign chosen so that contracting Y_l1(z) and Y_l2(z) gives a
    positive multiple of Y_l3(z).  For l1 + l2 + l3 odd that contraction is
    zero (the coupling is odd under inversion: 1 x 1 -> 1 is the cross
    product), and the sign is chosen instead so that the first nonzero entry
    in (m1, m2, m3) order is positive.
  * Paths: every (l1, l2, l3) with l1, l2 <= l_max,
    |l1 - l2| <= l3 <= min(l1 + l2, l_max) and l1 + l2 + l3 even, in
    lexicographic order (the natural-parity paths); with parity="odd" the
    ones with l1 + l2 + l3 odd, with parity="all" both.
"""
import math
from functools import lru_cache

import numpy as np
import torch

SQ3 = math.sqrt(3.0)
SQ5 = math.sqrt(5.0)
SQ15 = math.sqrt(15.0)


def sh_real(u, l_max):
    """Real SH of unit vectors u (..., 3) -> list [Y_0, ..., Y_lmax], Y_l (..., 2l+1)."""
    x, y, z = u[..., 0], u[..., 1], u[..., 2]
    out = [torch.ones_like(x)[..., None]]
    if l_max >= 1:
        out.append(torch.stack([SQ3 * y, SQ3 * z, SQ3 * x], dim=-1))
    if l_max >= 2:
        out.append(torch.stack([
            SQ15 * x * y,
            SQ15 * y * z,
            0.5 * SQ5 * (3.0 * z * z - 1.0),
            SQ15 * x * z,
            0.5 * SQ15 * (x * x - y * y),
        ], dim=-1))
    if l_max > 2:
        raise ValueError("l_max <= 2 supported")
    return out


def coupling_paths(l_max, scalar_only=False, parity="even"):
    want = {"even": (0,), "odd": (1,), "all": (0, 1)}[parity]
    paths = []
    for l1 in range(l_max + 1):
        for l2 in range(l_max + 1):
            for l3 in range(abs(l1 - l2), min(l1 + l2, l_max) + 1):
                if (l1 + l2 + l3) % 2 not in want:
                    continue
                if scalar_only and l3 != 0:
                    continue
                paths.append((l1, l2, l3))
    return paths


def _f(n):
    return math.factorial(n)


def cg_complex(j1, m1, j2, m2, J, M):
    """<j1 m1 j2 m2 | J M> by Racah's closed formula (integer spins)."""
    if m1 + m2 != M or not (abs(j1 - j2) <= J <= j1 + j2):
        return 0.0
    if abs(m1) > j1 or abs(m2) > j2 or abs(M) > J:
        return 0.0
    pre = (2 * J + 1) * _f(J + j1 - j2) * _f(J - j1 + j2) * _f(j1 + j2 - J) / _f(j1 + j2 + J + 1)
    pre *= _f(J + M) * _f(J - M) * _f(j1 - m1) * _f(j1 + m1) * _f(j2 - m2) * _f(j2 + m2)
    s = 0.0
    for k in range(0, j1 + j2 + J + 1):
        args = [k, j1 + j2 - J - k, j1 - m1 - k, j2 + m2 - k, J - j2 + m1 + k, J - j1 - m2 + k]
        if min(args) < 0:
            continue
        den = 1
        for a in args:
            den *= _f(a)
        s += (-1) ** k / den
    return math.sqrt(pre) * s


def complex_to_real(l):
    """Q_l with Y_real = Q_l Y_complex (Condon-Shortley complex harmonics).

    m < 0: Y_lm = i/sqrt2 (Y_l^m - (-1)^m Y_l^-m);  m = 0: Y_l0 = Y_l^0;
    m > 0: Y_lm = 1/sqrt2 (Y_l^-m + (-1)^m Y_l^m).  Rows/cols ordered m = -l..l.
    """
    Q = np.zeros((2 * l + 1, 2 * l + 1), dtype=np.complex128)
    r = 1.0 / math.sqrt(2.0)
    for m in range(-l, l + 1):
        row = m + l
        if m < 0:
            Q[row, m + l] = 1j * r
            Q[row, -m + l] = -1j * r * (-1) ** m
        elif m == 0:
            Q[row, l] = 1.0
        else:
            Q[row, -m + l] = r
            Q[row, m + l] = r * (-1) ** m
    return Q


@lru_cache(maxsize=None)
def real_cg(l1, l2, l3):
    """Real coupling tensor C[m1, m2, m3] (float64 ndarray), Frobenius norm 1."""
    cg = np.zeros((2 * l1 + 1, 2 * l2 + 1, 2 * l3 + 1))
    for m1 in range(-l1, l1 + 1):
        for m2 in range(-l2, l2 + 1):
            M = m1 + m2
            if abs(M) <= l3:
                cg[m1 + l1, m2 + l2, M + l3] = cg_complex(l1, m1, l2, m2, l3, M)
    Q1, Q2, Q3 = complex_to_real(l1), complex_to_real(l2), complex_to_real(l3)
    # real components a_r = Q a_c  =>  c_r = Q3 CG(Q1^H a_r, Q2^H b_r)
    C = np.einsum("ai,bj,ck,ijk->abc", Q1.conj(), Q2.conj(), Q3, cg)
    re, im = np.abs(C.real).max(), np.abs(C.imag).max()
    C = C.real if re >= im else C.imag
    assert min(re, im) < 1e-12, (l1, l2, l3)
    C = C / np.linalg.norm(C)
    if (l1 + l2 + l3) % 2 == 0:
        # sign rule: C(Y_l1(z), Y_l2(z)) must be a positive multiple of Y_l3(z)
        zhat = torch.tensor([[0.0, 0.0, 1.0]], dtype=torch.float64)
        Y = [t[0].numpy() for t in sh_real(zhat, max(l1, l2, l3))]
        c = np.einsum("abc,a,b,c->", C, Y[l1], Y[l2], Y[l3])
    else:
        # odd path: the first nonzero entry in (m1, m2, m3) order is positive
        c = C.ravel()[np.flatnonzero(np.abs(C.ravel()) > 1e-12)[0]]
    if c < 0:
        C = -C
    return np.ascontiguousarray(C)
