"""Pins of the seeded input generator's one piece of arithmetic shared by the
oracle and the GPU path: the isotropic conversion (E, nu) -> (mu, lambda)
that several tests feed to both sides.  A mistake there would pass every
parity test, so it is checked against what elasticity fixes independently:
the inverse relations and textbook values."""
import numpy as np
import pytest

import fe_inputs as fi


@pytest.mark.parametrize("E,nu", [(1e4, 0.45), (3.2e4, 0.3), (5e3, 0.49), (2e11, 0.0)])
def test_lame_from_young_inverse_relations(E, nu):
    mu, lam = fi.lame_from_young(E, nu)
    # Poisson's ratio and Young's modulus recovered from the Lame pair
    assert abs(lam / (2.0 * (lam + mu)) - nu) <= 1e-14
    assert abs(mu * (3.0 * lam + 2.0 * mu) / (lam + mu) - E) <= 1e-13 * E
    # bulk modulus two ways: lambda + 2 mu / 3 = E / (3 (1 - 2 nu))
    assert abs((lam + 2.0 * mu / 3.0) - E / (3.0 * (1.0 - 2.0 * nu))) <= 1e-12 * E / (1.0 - 2.0 * nu)


def test_lame_from_young_textbook_values():
    """Structural steel, E = 200 GPa, nu = 0.3: G = 76.923 GPa and
    lambda = 115.385 GPa (the values tabulated in elasticity texts)."""
    mu, lam = fi.lame_from_young(200e9, 0.3)
    assert abs(mu / 1e9 - 76.923) < 5e-4
    assert abs(lam / 1e9 - 115.385) < 5e-4
    mu0, lam0 = fi.lame_from_young(1.0, 0.0)          # no lateral coupling
    assert mu0 == 0.5 and lam0 == 0.0


def test_lame_from_young_is_linear_in_E():
    """The per-element scale s_e of the adjoint multiplies E at fixed nu, so
    the pair must scale with E."""
    E = fi.lognormal_modulus(50, seed=11)
    mu, lam = fi.lame_from_young(E, 0.4506)
    mu1, lam1 = fi.lame_from_young(1.0, 0.4506)
    np.testing.assert_allclose(mu, E * mu1, rtol=1e-15)
    np.testing.assert_allclose(lam, E * lam1, rtol=1e-15)
