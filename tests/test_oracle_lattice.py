"""Pins of the oracle's lattice tables and pointwise formulas against what the lattice
definitions and the mathematics fix (not against a retyped copy of the same formula)."""
import itertools

import numpy as np
import pytest


def _velocity_set(e):
    return {tuple(int(v) for v in e[:, i]) for i in range(e.shape[1])}


def test_d3q19_velocity_set(orc):
    """Eq. 19: the rest vector, the 6 axis vectors and the 12 face diagonals."""
    e = orc.tables()["e19"]
    want = {(0, 0, 0)}
    want |= {tuple(s * (a == k) for a in range(3)) for k in range(3) for s in (1, -1)}
    for a, b in itertools.combinations(range(3), 2):
        for sa, sb in itertools.product((1, -1), repeat=2):
            v = [0, 0, 0]
            v[a], v[b] = sa, sb
            want.add(tuple(v))
    assert len(_velocity_set(e)) == 19 and _velocity_set(e) == want


def test_d3q19_weights_isotropy(orc):
    """Weights under Eq. 24 reproduce the lattice tensors of an isotropic c_s^2 = 1/3
    lattice up to fourth order."""
    t = orc.tables()
    e, w = t["e19"], t["w19"]
    d = np.eye(3)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(e @ w, 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ai,bi->ab", w, e, e), d / 3, atol=1e-15)
    assert np.allclose(np.einsum("i,ai,bi,ci->abc", w, e, e, e), 0, atol=1e-15)
    four = np.einsum("i,ai,bi,ci,di->abcd", w, e, e, e, e)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(four, iso, atol=1e-15)


def _dhumieres_basis(e):
    """The D3Q19 moment polynomials (d'Humieres et al. 2002) evaluated on the velocities,
    in the moment order of Eq. 20."""
    ex, ey, ez = e
    e2 = ex * ex + ey * ey + ez * ez
    rows = [
        np.ones_like(ex),
        19 * e2 - 30,
        (21 * e2 * e2 - 53 * e2 + 24) / 2,
        ex, (5 * e2 - 9) * ex,
        ey, (5 * e2 - 9) * ey,
        ez, (5 * e2 - 9) * ez,
        3 * ex * ex - e2, (3 * e2 - 5) * (3 * ex * ex - e2),
        ey * ey - ez * ez, (3 * e2 - 5) * (ey * ey - ez * ez),
        ex * ey, ey * ez, ez * ex,
        ex * (ey * ey - ez * ez), ey * (ez * ez - ex * ex), ez * (ex * ex - ey * ey),
    ]
    return np.array(rows, dtype=np.float64)


def test_M_rows_are_moment_polynomials(orc):
    """Eq. A2 equals the polynomial basis of Eq. 20 evaluated on Eq. 19."""
    t = orc.tables()
    assert np.array_equal(t["M"], _dhumieres_basis(t["e19"]))


def test_M_orthogonal_and_inverse(orc):
    t = orc.tables()
    M, Minv = t["M"], t["Minv"]
    G = M @ M.T
    assert np.allclose(G - np.diag(np.diag(G)), 0, atol=0)
    assert np.allclose(M @ Minv, np.eye(19), atol=1e-14)
    assert np.allclose(Minv @ M, np.eye(19), atol=1e-14)


def test_N_rows_are_basis_vectors(orc):
    """Eq. 36 is built from |1>, |e_x>, |e_y>, |e_z>, |e^2>, |e_x^2 - e_y^2>, |e_x^2 - e_z^2>
    on the D3Q7 velocities (first seven columns of Eq. 12)."""
    t = orc.tables()
    ex, ey, ez = t["e7"]
    assert _velocity_set(t["e7"]) == {(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0),
                                      (0, -1, 0), (0, 0, 1), (0, 0, -1)}
    rows = np.array([np.ones(7), ex, ey, ez, ex * ex + ey * ey + ez * ez,
                     ex * ex - ey * ey, ex * ex - ez * ez])
    assert np.array_equal(t["N"], rows)


def test_Ninv_as_printed_is_the_inverse(orc):
    """Eq. 43 (typed from the paper) is the inverse of Eq. 36."""
    t = orc.tables()
    assert np.allclose(t["N"] @ t["Ninv"], np.eye(7), atol=1e-15)
    assert np.allclose(t["Ninv"] @ t["N"], np.eye(7), atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_feq_moments(orc, seed):
    """Eq. 24: zeroth, first and second velocity moments of the porous incompressible
    equilibrium are rho, rho0 u and c_s^2 rho I + rho0 u u / phi."""
    rng = np.random.default_rng(seed)
    rho, rho0 = 1 + 0.05 * rng.uniform(-1, 1), 1.0
    u = 0.05 * rng.uniform(-1, 1, 3)
    phi = rng.uniform(0.3, 1.0)
    e = orc.tables()["e19"]
    f = orc.feq19(rho, u, phi, rho0)
    assert f.sum() == pytest.approx(rho, abs=1e-15)
    assert np.allclose(e @ f, rho0 * u, atol=1e-16)
    P = np.einsum("ai,bi,i->ab", e, e, f)
    assert np.allclose(P, rho / 3 * np.eye(3) + rho0 * np.outer(u, u) / phi, atol=1e-15)


def test_feq_phi1_is_incompressible_d3q19(orc):
    """phi = 1 reduces Eq. 24 to He & Luo's incompressible equilibrium
    w_i [rho + rho0 (3 e.u + 4.5 (e.u)^2 - 1.5 u^2)]."""
    t = orc.tables()
    u = np.array([0.03, -0.02, 0.01])
    eu = t["e19"].T @ u
    want = t["w19"] * (1.01 + (3 * eu + 4.5 * eu * eu - 1.5 * u @ u))
    assert np.allclose(orc.feq19(1.01, u, 1.0), want, atol=1e-16)


@pytest.mark.parametrize("seed", range(5))
def test_M_feq_equals_eq21(orc, seed):
    """Eq. 11 (m_eq = M f_eq) agrees with the closed form of Eq. 21 for beta1 = 3,
    beta2 = -5.5, beta3 = -0.5."""
    rng = np.random.default_rng(100 + seed)
    rho, u, phi = 1 + 0.02 * rng.uniform(-1, 1), 0.05 * rng.uniform(-1, 1, 3), rng.uniform(0.3, 1)
    M = orc.tables()["M"]
    assert np.allclose(M @ orc.feq19(rho, u, phi), orc.meq19_eq21(rho, u, phi), atol=2e-15)


@pytest.mark.parametrize("seed", range(5))
def test_stilde_is_velocity_derivative_of_meq(orc, seed):
    """Eq. 23 is the directional derivative of m_eq(u) (Eq. 21) along F: the forcing
    moments of Guo's scheme.  m_eq is quadratic in u, so a central difference is exact."""
    rng = np.random.default_rng(200 + seed)
    rho, u, phi = 1.0, 0.05 * rng.uniform(-1, 1, 3), rng.uniform(0.3, 1)
    F = 1e-3 * rng.uniform(-1, 1, 3)
    h = 0.5
    M = orc.tables()["M"]
    dm = (M @ orc.feq19(rho, u + h * F, phi) - M @ orc.feq19(rho, u - h * F, phi)) / (2 * h)
    assert np.allclose(orc.stilde19(u, F, phi), dm, atol=1e-15)


@pytest.mark.parametrize("seed", range(3))
def test_geq_moments_and_neq(orc, seed):
    """Eq. 42: sum g = sigma T, sum e g = T u, sum e e g = c_sT^2 sigma T I, and
    N g_eq = n_eq of Eq. 37."""
    rng = np.random.default_rng(300 + seed)
    T, u = rng.uniform(0, 1), 0.05 * rng.uniform(-1, 1, 3)
    sigma, varpi = rng.uniform(0.5, 2), rng.uniform(0.2, 0.8)
    t = orc.tables()
    g = orc.geq7(T, u, sigma, varpi)
    e = t["e7"]
    assert g.sum() == pytest.approx(sigma * T, abs=1e-15)
    assert np.allclose(e @ g, T * u, atol=1e-16)
    assert np.allclose(np.einsum("ai,bi,i->ab", e, e, g), varpi / 3 * sigma * T * np.eye(3),
                       atol=1e-15)
    assert np.allclose(t["N"] @ g, orc.neq7(T, u, sigma, varpi), atol=1e-15)


@pytest.mark.parametrize("seed", range(6))
def test_velocity_solves_eq26(orc, seed):
    """Eq. 27-28 solve the nonlinear Eq. 26: rho0 u = sum e f + rho0 F(u)/2, F from Eq. 4."""
    rng = np.random.default_rng(400 + seed)
    phi = rng.uniform(0.3, 1)
    K = 10 ** rng.uniform(-1, 2)
    Fphi = rng.uniform(0, 0.6)
    nu = rng.uniform(0.01, 0.2)
    G = 1e-3 * rng.uniform(-1, 1, 3)
    f = orc.feq19(1.0, 0.05 * rng.uniform(-1, 1, 3), phi) + 1e-3 * rng.uniform(-1, 1, 19)
    u = orc.velocity(f, G, phi, nu, K, Fphi)
    F = orc.force(u, G, phi, nu, K, Fphi)
    e = orc.tables()["e19"]
    assert np.allclose(u, e @ f + 0.5 * F, atol=1e-16)
