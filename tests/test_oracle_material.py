"""Pins of the oracle's constitutive law (Eq. sig_eq, Eq. const_eq, tensor D) -- CPU."""
import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import material as M

MU, LAM = 1.0, 4.0


@pytest.mark.parametrize("d", [2, 3])
def test_reference_state(d):
    F = np.eye(d)[None]
    assert np.abs(M.cauchy_stress(F, np.ones(1), LAM)).max() == 0
    # at F = I, C is the linear isotropic tensor lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk)
    C = M.spatial_elasticity(F, np.ones(1), LAM)[0]
    for i, j, k, l in np.ndindex(d, d, d, d):
        lin = LAM * (i == j) * (k == l) + MU * ((i == k) * (j == l) + (i == l) * (j == k))
        assert abs(C[i, j, k, l] - lin) < 1e-14


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("s", [0.8, 0.95, 1.1])
def test_uniaxial_strain_closed_form(d, s):
    F = np.eye(d)
    F[0, 0] = s
    sig = M.cauchy_stress(F[None], np.ones(1), LAM)[0]
    assert abs(sig[0, 0] - (MU * (s * s - 1) / s + LAM * np.log(s) / s)) < 1e-14
    for i in range(1, d):
        assert abs(sig[i, i] - LAM * np.log(s) / s) < 1e-14
    assert np.abs(sig - np.diag(np.diag(sig))).max() == 0


@pytest.mark.parametrize("s", [0.85, 1.2])
def test_uniaxial_stress_3d(s):
    # lateral stretch t from mu (t^2 - 1) + lam ln(s t^2) = 0 gives sigma_22 = sigma_33 = 0
    t = brentq(lambda t: MU * (t * t - 1) + LAM * np.log(s * t * t), 0.5, 2.0, xtol=1e-15)
    F = np.diag([s, t, t])
    sig = M.cauchy_stress(F[None], np.ones(1), LAM)[0]
    assert abs(sig[1, 1]) < 1e-12 and abs(sig[2, 2]) < 1e-12
    assert abs(sig[0, 0] - MU * (s * s - t * t) / (s * t * t)) < 1e-12


@pytest.mark.parametrize("d", [2, 3])
def test_D_major_symmetry(d):
    # the tangent is symmetric because D_ijkl = D_jilk (Section 3.1.4)
    rng = np.random.default_rng(0)
    F = np.eye(d) + 0.2 * rng.uniform(-1, 1, (5, d, d))
    D = M.tangent_tensor_D(F, np.full(5, 1.3), LAM)
    assert np.abs(D - np.einsum("nijkl->njilk", D)).max() < 1e-13
