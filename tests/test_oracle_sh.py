"""Pins for the oracle's spherical-harmonic basis (Sec. 3.1, Eq. 4).

The paper fixes only that the colour is a linear combination of SH up to
l_max; the basis is pinned here to mathematics that does not depend on the
oracle: orthonormality by exact quadrature, the addition theorem against
scipy's Legendre polynomials, scipy's complex SH, the printed table of real SH
constants in tests/golden/sh_constants.txt, and parity under v -> -v.
"""
import math
import os

import numpy as np
import pytest
import scipy.special as sp

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sh_constants.txt")


def _sphere_quadrature(n_theta, n_phi):
    x, w = np.polynomial.legendre.leggauss(n_theta)  # exact in cos(theta) up to 2n-1
    phi = (np.arange(n_phi) + 0.5) * 2 * math.pi / n_phi  # exact in phi up to n-1
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    wts = (w[:, None] * np.full(n_phi, 2 * math.pi / n_phi)[None, :]).reshape(-1)
    return dirs, wts


@pytest.mark.parametrize("deg", [0, 1, 2, 3, 5])
def test_gram_matrix_is_identity(deg):
    dirs, w = _sphere_quadrature(deg + 2, 2 * deg + 2)
    Y = O.sh_basis(deg, dirs)
    G = (Y * w[:, None]).T @ Y
    assert np.abs(G - np.eye(G.shape[0])).max() < 1e-12


@pytest.mark.parametrize("deg", [1, 2, 3, 4])
def test_addition_theorem(deg):
    rng = np.random.default_rng(3)
    u = rng.normal(size=(20, 3))
    v = rng.normal(size=(20, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    Yu, Yv = O.sh_basis(deg, u), O.sh_basis(deg, v)
    for l in range(deg + 1):
        sl = slice(l * l, (l + 1) * (l + 1))
        lhs = (Yu[:, sl] * Yv[:, sl]).sum(1)
        rhs = (2 * l + 1) / (4 * math.pi) * sp.eval_legendre(l, (u * v).sum(1))
        assert np.abs(lhs - rhs).max() < 1e-12


def test_matches_scipy_complex_sh_without_condon_shortley():
    rng = np.random.default_rng(5)
    d = rng.normal(size=(30, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(d[:, 2])
    phi = np.arctan2(d[:, 1], d[:, 0])
    Y = O.sh_basis(3, d)
    for l in range(4):
        for m in range(-l, l + 1):
            # scipy's complex SH carry the (-1)^m phase; the real basis
            # without that phase is sqrt(2) (-1)^m Re/Im of Y_l^|m|.
            Yc = sp.sph_harm_y(l, abs(m), theta, phi)
            if m == 0:
                ref = Yc.real
            elif m > 0:
                ref = math.sqrt(2) * (-1) ** m * Yc.real
            else:
                ref = math.sqrt(2) * (-1) ** m * Yc.imag
            assert np.abs(Y[:, l * l + l + m] - ref).max() < 1e-12, (l, m)


def _golden():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                l, m, x, y, z, val = line.split()
                rows.append((int(l), int(m), float(x), float(y), float(z), float(val)))
    return rows


def test_printed_constants():
    rows = _golden()
    assert len(rows) >= 16
    for l, m, x, y, z, val in rows:
        d = np.array([x, y, z])
        d /= np.linalg.norm(d)
        Y = O.sh_basis(3, d[None])[0]
        assert abs(Y[l * l + l + m] - val) < 5e-9, (l, m, Y[l * l + l + m], val)


def test_parity():
    rng = np.random.default_rng(9)
    d = rng.normal(size=(10, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Yp, Ym = O.sh_basis(3, d), O.sh_basis(3, -d)
    for l in range(4):
        sl = slice(l * l, (l + 1) * (l + 1))
        assert np.abs(Ym[:, sl] - (-1) ** l * Yp[:, sl]).max() < 1e-13


def test_cartesian_gradient_by_central_differences():
    rng = np.random.default_rng(11)
    pts = rng.normal(size=(8, 3))  # the polynomial form is defined off the sphere too
    _, dY = O.sh_basis(3, pts, grad=True)
    h = 1e-6
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd = (O.sh_basis(3, pts + e) - O.sh_basis(3, pts - e)) / (2 * h)
        assert np.abs(fd - dY[:, :, a]).max() < 1e-7
