"""Oracle: the mixing matrix A(beta) and its parameter derivatives (Eq. 5, Sec. 2.1).

Columns, for band centre nu:
  CMB:  A_cmb(nu) = 1                                   (thermodynamic units)
  dust: A_d(nu) = nu / (exp(h nu / k T_d) - 1) * (exp(h nu0 / k T_d) - 1) / nu0 * (nu / nu0)^beta_d
  sync: A_s(nu) = (nu / nu0)^beta_s
with nu0 = 353 GHz (dust) and 23 GHz (synchrotron). Eq. 5 is a ratio of Rayleigh-Jeans
brightnesses while the maps are in K_CMB (thermodynamic units), so each foreground column is read as
multiplied by the Rayleigh-Jeans-to-K_CMB factor ratio g(nu) / g(nu0), g(nu) = (e^x - 1)^2 / (x^2 e^x),
x = h nu / (k T_CMB); the beta derivatives are unaffected by it.

Derivatives (closed form):
  dA_d/dbeta_d = A_d ln(nu/nu0),  dA_s/dbeta_s = A_s ln(nu/nu0),
  dA_d/dT_d   = A_d [x e^x/(e^x - 1) - x0 e^x0/(e^x0 - 1)] / T_d,  x = h nu/(k T_d), x0 = h nu0/(k T_d).

Parity pins: hand values from Planck's law (independent physical route), A(nu0) = 1, the
Rayleigh-Jeans limit T_d -> infinity, and central finite differences of the derivatives.
"""
from __future__ import annotations

import numpy as np

H_PLANCK = 6.62607015e-34   # J s
K_BOLTZ = 1.380649e-23      # J / K
H_OVER_K_GHZ = H_PLANCK / K_BOLTZ * 1e9  # K per GHz
NU0_DUST = 353.0
NU0_SYNC = 23.0
T_CMB = 2.7255


def rj_to_cmb(nu_ghz, t_cmb=T_CMB):
    """g(nu) = (e^x - 1)^2 / (x^2 e^x), x = h nu / (k T_CMB): K_RJ -> K_CMB factor."""
    x = H_OVER_K_GHZ * np.asarray(nu_ghz, dtype=np.float64) / t_cmb
    return np.expm1(x) ** 2 / (x * x * np.exp(x))


def dust_column(nu_ghz, beta_d, temp_d, nu0=NU0_DUST, units="K_CMB"):
    nu = np.asarray(nu_ghz, dtype=np.float64)
    bd = np.asarray(beta_d, dtype=np.float64)[..., None]
    td = np.asarray(temp_d, dtype=np.float64)[..., None]
    x = H_OVER_K_GHZ * nu / td
    x0 = H_OVER_K_GHZ * nu0 / td
    col = nu / np.expm1(x) * np.expm1(x0) / nu0 * (nu / nu0) ** bd
    if units == "K_CMB":
        col = col * rj_to_cmb(nu) / rj_to_cmb(nu0)
    return col


def sync_column(nu_ghz, beta_s, nu0=NU0_SYNC, units="K_CMB"):
    nu = np.asarray(nu_ghz, dtype=np.float64)
    bs = np.asarray(beta_s, dtype=np.float64)[..., None]
    col = (nu / nu0) ** bs
    if units == "K_CMB":
        col = col * rj_to_cmb(nu) / rj_to_cmb(nu0)
    return col


def mixing_matrix(nu_ghz, beta_d, temp_d, beta_s, units="K_CMB"):
    """A with shape [..., F, 3]; the leading shape is that of the (broadcast) parameters."""
    ad = dust_column(nu_ghz, beta_d, temp_d, units=units)
    as_ = sync_column(nu_ghz, beta_s, units=units)
    ad, as_ = np.broadcast_arrays(ad, as_)
    return np.stack([np.ones_like(ad), ad, as_], axis=-1)


def mixing_derivatives(nu_ghz, beta_d, temp_d, beta_s, units="K_CMB"):
    """(dA_d/dbeta_d, dA_d/dT_d, dA_s/dbeta_s), each [..., F] (the other entries of dA vanish)."""
    nu = np.asarray(nu_ghz, dtype=np.float64)
    ad = dust_column(nu, beta_d, temp_d, units=units)
    as_ = sync_column(nu, beta_s, units=units)
    td = np.asarray(temp_d, dtype=np.float64)[..., None]
    x = H_OVER_K_GHZ * nu / td
    x0 = H_OVER_K_GHZ * NU0_DUST / td
    dlnb_dt = (x * np.exp(x) / np.expm1(x) - x0 * np.exp(x0) / np.expm1(x0)) / td
    return ad * np.log(nu / NU0_DUST), ad * dlnb_dt, as_ * np.log(nu / NU0_SYNC)
