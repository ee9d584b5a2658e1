"""Pins for the Ewald oracle: textbook lattice constants, alpha independence,
phi = dE/dq, F = -dE/dx, symmetry, and the spherical-order image sum."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


def _random_system(seed, n, L, neutral=True):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, L, (n, 3))
    q = rng.uniform(-1, 1, n)
    if neutral:
        q -= q.mean()
    return x, q


def test_wigner_self_term():
    g = _gold("lattice_constants.json")["wigner_simple_cubic"]["value"]
    for L in (1.0, 3.2, 21.5):
        assert oracle.xi(L) * L == pytest.approx(g, abs=2e-12)
        # a single charge in its box: E = 1/2 q^2 xi
        _, _, e = oracle.ewald(np.array([[0.1 * L, 0.7 * L, 0.3 * L]]), np.array([0.8]), L)
        assert e == pytest.approx(0.5 * 0.64 * g / L, rel=1e-12)


def test_madelung_rock_salt():
    M = _gold("lattice_constants.json")["madelung_rock_salt"]["value"]
    a = 0.5640
    pos, q = [], []
    for i, j, k in itertools.product(range(2), repeat=3):
        pos.append([i * a / 2, j * a / 2, k * a / 2])
        q.append((-1.0) ** (i + j + k))
    _, g, e = oracle.ewald(np.array(pos), np.array(q), a)
    # 4 ion pairs per cubic cell, r0 = a/2
    assert -e / 4 * (a / 2) == pytest.approx(M, rel=1e-11)
    assert np.abs(g).max() < 1e-10


def test_madelung_cesium_chloride():
    M = _gold("lattice_constants.json")["madelung_cesium_chloride"]["value"]
    a = 0.4123
    _, _, e = oracle.ewald(np.array([[0, 0, 0], [a / 2, a / 2, a / 2]]), np.array([1.0, -1.0]), a)
    r0 = a * np.sqrt(3) / 2
    assert -e * r0 == pytest.approx(M, rel=1e-11)


@pytest.mark.parametrize("neutral", [True, False])
def test_alpha_independence(neutral):
    x, q = _random_system(3, 200, 2.1, neutral)
    p1, g1, e1 = oracle.ewald(x, q, 2.1, rc=0.55)
    p2, g2, e2 = oracle.ewald(x, q, 2.1, rc=1.05)
    assert e1 == pytest.approx(e2, rel=1e-12, abs=1e-12)
    assert np.abs(p1 - p2).max() < 1e-11
    assert np.abs(g1 - g2).max() < 1e-10


def test_targets_subset_matches_full():
    x, q = _random_system(4, 300, 2.5, neutral=False)
    p, g, _ = oracle.ewald(x, q, 2.5)
    t = np.array([5, 17, 123, 299])
    pt, gt, et = oracle.ewald(x, q, 2.5, targets=t)
    assert et is None
    np.testing.assert_allclose(pt, p[t], rtol=0, atol=1e-13)
    np.testing.assert_allclose(gt, g[t], rtol=0, atol=1e-12)


def test_potential_is_charge_derivative_of_energy():
    # E is quadratic in q (background included), so central differences are exact
    x, q = _random_system(5, 40, 1.7, neutral=False)
    p, _, _ = oracle.ewald(x, q, 1.7)
    h = 1e-3
    for k in (0, 11, 39):
        qp = q.copy(); qp[k] += h
        qm = q.copy(); qm[k] -= h
        d = (oracle.ewald(x, qp, 1.7)[2] - oracle.ewald(x, qm, 1.7)[2]) / (2 * h)
        assert d == pytest.approx(p[k], rel=1e-9, abs=1e-10)


def test_force_is_position_derivative_of_energy():
    x, q = _random_system(6, 30, 1.5, neutral=False)
    _, g, _ = oracle.ewald(x, q, 1.5)
    h = 1e-5
    for k in (0, 7, 29):
        for ax in range(3):
            xp = x.copy(); xp[k, ax] += h
            xm = x.copy(); xm[k, ax] -= h
            d = (oracle.ewald(xp, q, 1.5)[2] - oracle.ewald(xm, q, 1.5)[2]) / (2 * h)
            # dE/dx_k = q_k grad phi_k
            assert d == pytest.approx(q[k] * g[k, ax], rel=1e-6, abs=1e-8)


def test_translation_and_cubic_symmetry():
    L = 1.9
    x, q = _random_system(7, 50, L, neutral=False)
    _, _, e = oracle.ewald(x, q, L)
    _, _, et = oracle.ewald(np.mod(x + np.array([0.31, -0.77, 1.23]), L), q, L)
    # 90 degree rotation about z maps the cubic lattice onto itself
    xr = np.stack([L - x[:, 1], x[:, 0], x[:, 2]], 1)
    _, _, er = oracle.ewald(np.mod(xr, L), q, L)
    assert et == pytest.approx(e, rel=1e-12)
    assert er == pytest.approx(e, rel=1e-12)


def test_spherical_image_sum_is_ewald_plus_dipole_term():
    """de Leeuw-Perram-Smith: whole image cells summed in spherical order (vacuum
    boundary) converge to the tin-foil Ewald energy + (2 pi / 3V)|D|^2 for a
    neutral cell.  The image sum is a plain Coulomb sum, independent of Ewald."""
    L, n = 1.3, 6
    x, q = _random_system(2, n, L, neutral=True)
    _, _, e = oracle.ewald(x, q, L)
    D = (q[:, None] * x).sum(0)
    target = e + 2 * np.pi / (3 * L ** 3) * (D @ D)
    R = 30
    ns = np.array([m for m in itertools.product(range(-R, R + 1), repeat=3)
                   if m[0] ** 2 + m[1] ** 2 + m[2] ** 2 <= R * R], float)
    src = (x[None, :, :] + ns[:, None, :] * L).reshape(-1, 3)
    es = 0.5 * (q * oracle.direct(x, src, np.tile(q, len(ns)))).sum()
    assert es == pytest.approx(target, rel=1e-6)
    # the dipole term is not negligible here, so a dropped or mis-signed term fails
    assert abs(2 * np.pi / (3 * L ** 3) * (D @ D)) > 1e-3 * abs(target)


def test_pair_kernel_consistent_with_ewald():
    L = 2.2
    x, q = _random_system(8, 12, L, neutral=False)
    p, g, _ = oracle.ewald(x, q, L)
    for i in (0, 5):
        s = sum(q[j] * oracle.pair_A(x[i] - x[j], L)[0] for j in range(12))
        gs = sum(q[j] * oracle.pair_A(x[i] - x[j], L)[1] for j in range(12) if j != i)
        assert s == pytest.approx(p[i], rel=1e-12, abs=1e-12)
        np.testing.assert_allclose(gs, g[i], atol=1e-11)


@pytest.mark.parametrize("neutral", [True, False])
def test_energy_only_route_matches_potential_route(neutral):
    x, q = _random_system(9, 500, 2.4, neutral)
    _, _, e = oracle.ewald(x, q, 2.4, rc=0.7)
    assert oracle.ewald_energy(x, q, 2.4, rc=0.7) == pytest.approx(e, rel=1e-12)
    assert oracle.ewald_energy(x, q, 2.4, rc=1.1) == pytest.approx(e, rel=1e-12)


def test_real_and_reciprocal_parts_add_up():
    x, q = _random_system(10, 300, 2.2, neutral=False)
    p, g, _ = oracle.ewald(x, q, 2.2)
    p1, g1, _ = oracle.ewald(x, q, 2.2, parts=1)
    p2, g2, _ = oracle.ewald(x, q, 2.2, parts=2)
    np.testing.assert_allclose(p1 + p2, p, atol=1e-12)
    np.testing.assert_allclose(g1 + g2, g, atol=1e-11)
