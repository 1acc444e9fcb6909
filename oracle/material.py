"""Compressible neo-Hookean material in the spatial description (oracle, FP64).

sigma  -- Cauchy stress, Eq. (sig_eq):  sigma = mu/J (b - I) + lam ln(J)/J I,  b = F F^T
C      -- spatial elasticity tensor, Eq. (const_eq):
          C_ijkl = lam/J d_ij d_kl + (mu - lam ln J)/J (d_ik d_jl + d_il d_jk)
D      -- Section 3.1.4:  D_ijkl = C_ikjl + d_ij sigma_kl
Arrays carry leading batch axes; mu may be an array broadcastable to those axes.
In 2D (plane strain, F_33 = 1) the d = 2 forms are used as written.
"""
import numpy as np


def cauchy_stress(F, mu, lam):
    d = F.shape[-1]
    J = np.linalg.det(F)
    b = F @ np.swapaxes(F, -1, -2)
    eye = np.eye(d)
    mu = np.asarray(mu)[..., None, None]
    return (mu / J[..., None, None]) * (b - eye) + (lam * np.log(J) / J)[..., None, None] * eye


def spatial_elasticity(F, mu, lam):
    d = F.shape[-1]
    J = np.linalg.det(F)
    dl = np.eye(d)
    t1 = np.einsum("ij,kl->ijkl", dl, dl)
    t2 = np.einsum("ik,jl->ijkl", dl, dl) + np.einsum("il,jk->ijkl", dl, dl)
    a = (lam / J)[..., None, None, None, None]
    c = ((np.asarray(mu) - lam * np.log(J)) / J)[..., None, None, None, None]
    return a * t1 + c * t2


def tangent_tensor_D(F, mu, lam):
    """D_ijkl = C_ikjl + delta_ij sigma_kl (Section 3.1.4)."""
    d = F.shape[-1]
    C = spatial_elasticity(F, mu, lam)
    sig = cauchy_stress(F, mu, lam)
    return np.einsum("...ikjl->...ijkl", C) + np.einsum("ij,...kl->...ijkl", np.eye(d), sig)
