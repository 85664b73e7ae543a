"""Exchange-correlation potentials of the paper's experiments (Sec. 4), oracle side.

* Slater exchange: V_x = -(3 rho / pi)^(1/3)  (Remark after Eq. (FG)).  Its energy density is
  eps_x = -(3/4)(3/pi)^(1/3) rho^(1/3); the paper prints the exponent as 1/2, a typo: only 1/3 gives
  V_x = d(rho eps_x)/d rho = (4/3) eps_x, the potential it states.
* X-alpha: V_xc = -(3/2) alpha (3 rho / pi)^(1/3) with alpha = 0.77298 for LiH and CH4 (Sec. 4); alpha = 2/3 is Slater.
* LDA: Slater exchange plus the Perdew-Zunger correlation printed in Sec. 4, eps_c(r_s) with the two branches
  split at r_s = 1 (high-density branch for r_s < 1), r_s = (3 / (4 pi rho))^(1/3), and V_xc = eps_xc + rho d eps_xc/d rho.
  Here v_c = eps_c - (r_s/3) d eps_c / d r_s, differentiated per branch.
* rho below 1e-30 gives V_xc = 0 (the limit), avoiding log(0).
"""
from __future__ import annotations

import numpy as np

RHO_MIN = 1e-30
XALPHA_LIH = 0.77298


def eps_x(rho):
    rho = np.asarray(rho, dtype=np.float64)
    return -0.75 * (3.0 / np.pi) ** (1.0 / 3.0) * np.cbrt(rho)


def v_x(rho):
    rho = np.asarray(rho, dtype=np.float64)
    return -np.cbrt(3.0 * rho / np.pi)


def eps_c_pz(rs):
    rs = np.asarray(rs, dtype=np.float64)
    hi = 0.0311 * np.log(rs) - 0.048 + 0.0020 * rs * np.log(rs) - 0.0116 * rs
    lo = -0.1423 / (1.0 + 1.0529 * np.sqrt(rs) + 0.3334 * rs)
    return np.where(rs < 1.0, hi, lo)


def deps_c_pz(rs):
    """d eps_c / d r_s, per branch."""
    rs = np.asarray(rs, dtype=np.float64)
    hi = 0.0311 / rs + 0.0020 * (np.log(rs) + 1.0) - 0.0116
    den = 1.0 + 1.0529 * np.sqrt(rs) + 0.3334 * rs
    lo = 0.1423 * (0.5 * 1.0529 / np.sqrt(rs) + 0.3334) / (den * den)
    return np.where(rs < 1.0, hi, lo)


def v_c_pz(rho):
    rho = np.asarray(rho, dtype=np.float64)
    rs = np.cbrt(3.0 / (4.0 * np.pi * np.maximum(rho, RHO_MIN)))
    return eps_c_pz(rs) - rs / 3.0 * deps_c_pz(rs)


def v_xc(rho, kind: str, alpha: float = XALPHA_LIH):
    """V_xc at densities rho for kind in {'none', 'slater', 'xalpha', 'lda'}."""
    rho = np.asarray(rho, dtype=np.float64)
    if kind == "none":
        return np.zeros_like(rho)
    pos = rho >= RHO_MIN
    r = np.where(pos, rho, 1.0)
    if kind == "slater":
        v = v_x(r)
    elif kind == "xalpha":
        v = 1.5 * alpha * v_x(r)
    elif kind == "lda":
        v = v_x(r) + v_c_pz(r)
    else:
        raise ValueError(kind)
    return np.where(pos, v, 0.0)
