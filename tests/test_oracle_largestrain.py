"""Large-strain pins of the oracle's material laws (Section 3.1's hyperelastic
energies) against classical closed forms that the small-strain and derivative
pins do not reach.

Incompressible uniaxial tension, F = diag(s, s^-1/2, s^-1/2) (J = 1):
  * Mooney-Rivlin W = c10 (I1bar - 3) + c01 (I2bar - 3) + volumetric(J):
    I1 = s^2 + 2/s, I2 = 2 s + 1/s^2, and the true-stress difference
    sigma_11 - sigma_22 = 2 (s^2 - 1/s) (c10 + c01 / s)  (Rivlin's uniaxial
    result; the c01 term decays as 1/s, so a wrong weight or a swapped
    invariant in the I2 part changes the curve's shape, not only its slope);
  * neo-Hookean: sigma_11 - sigma_22 = mu (s^2 - 1/s) (Treloar's curve).
The volumetric terms vanish at J = 1 (ln J = 0, J - 1 = 0), so neither the
bulk modulus nor lambda enters; lateral stresses are equal and shear-free.
"""
import numpy as np
import pytest

from oracle import fe_oracle as O

STRETCHES = (0.55, 0.8, 1.0, 1.35, 2.0, 3.0)


def _uniaxial(s):
    return np.diag([s, s ** -0.5, s ** -0.5])[None]


def _cauchy(P, F):
    J = np.linalg.det(F)
    return (P @ np.swapaxes(F, -1, -2)) / J[..., None, None]


@pytest.mark.parametrize("s", STRETCHES)
@pytest.mark.parametrize("c10,c01", [(1.5e3, 5e2), (1.0, 0.0), (0.0, 1.0), (2.0e3, -3.0e2)])
def test_mooney_rivlin_incompressible_uniaxial(s, c10, c01):
    kappa = 5e4
    F = _uniaxial(s)
    sig = _cauchy(O.mr_pk1(F, c10, c01, kappa), F)[0]
    want = 2.0 * (s * s - 1.0 / s) * (c10 + c01 / s)
    scale = max(abs(c10), abs(c01)) * (s * s + 1.0 / s) + 1e-300
    assert abs((sig[0, 0] - sig[1, 1]) - want) <= 1e-12 * scale
    assert abs(sig[1, 1] - sig[2, 2]) <= 1e-12 * scale
    off = sig - np.diag(np.diag(sig))
    assert np.max(np.abs(off)) <= 1e-12 * scale


@pytest.mark.parametrize("s", STRETCHES)
def test_mooney_rivlin_energy_uniaxial_invariants(s):
    c10, c01, kappa = 1.5e3, 5e2, 5e4
    psi = O.mr_psi(_uniaxial(s), c10, c01, kappa)[0]
    want = c10 * (s * s + 2.0 / s - 3.0) + c01 * (2.0 * s + 1.0 / (s * s) - 3.0)
    assert abs(psi - want) <= 1e-12 * (abs(c10) + abs(c01)) * (s * s + 2.0 * s + 3.0)


@pytest.mark.parametrize("s", STRETCHES)
def test_neo_hookean_incompressible_uniaxial(s):
    mu, lam = 3.4e3, 3.1e4
    F = _uniaxial(s)
    sig = _cauchy(O.nh_pk1(F, mu, lam), F)[0]
    scale = mu * (s * s + 1.0 / s)
    assert abs((sig[0, 0] - sig[1, 1]) - mu * (s * s - 1.0 / s)) <= 1e-12 * scale
    assert abs(sig[1, 1] - sig[2, 2]) <= 1e-12 * scale
    # at J = 1 the lateral true stress of this law is mu (1/s - 1) (no pressure term)
    assert abs(sig[1, 1] - mu * (1.0 / s - 1.0)) <= 1e-12 * scale


def test_mooney_rivlin_pin_catches_swapped_invariant():
    """The uniaxial pin separates the two invariants: the I2 term alone (c10 = 0)
    gives 2 (s^2 - 1/s) c01 / s, which is not the I1 term's 2 (s^2 - 1/s) c10
    at any s != 1 (a law with the invariants swapped would fail the pin)."""
    s = 2.0
    F = _uniaxial(s)
    only_i2 = _cauchy(O.mr_pk1(F, 0.0, 1.0, 0.0), F)[0]
    only_i1 = _cauchy(O.mr_pk1(F, 1.0, 0.0, 0.0), F)[0]
    d2 = only_i2[0, 0] - only_i2[1, 1]
    d1 = only_i1[0, 0] - only_i1[1, 1]
    assert abs(d1 - 2.0 * (s * s - 1.0 / s)) < 1e-12 * d1
    assert abs(d2 - 2.0 * (s * s - 1.0 / s) / s) < 1e-12 * d1
    assert abs(d1 - d2) > 0.1 * d1
