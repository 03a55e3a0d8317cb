"""Wavenumbers and source coefficients (Section 2).

Readings taken where the paper is loose:
- Attenuation (Eq. 2.2, Table 2): alpha(f) [Np/m] = alpha0 [dB/m/MHz^eta] * (f/1 MHz)^eta
  / (20 log10 e).  The paper writes alpha = alpha0 |omega|^eta with the units garbled.
- Harmonic wavenumber (Section 2, after Eq. 2.5): k_n = n omega / c0 + i alpha(n f0).
- Source coefficient: the truncated cascade (Eq. 2.6) has right-hand side
  (beta omega^2 n^2 / (2 rho0 c0^4)) sum_{m=1}^{n-1} p_m p_{n-m} with omega the
  fundamental angular frequency; the volume potential solving the Helmholtz
  equation carries a minus sign (Eq. 3.2).  The oracle folds both into
  C_n = -beta omega^2 n^2 / (2 rho0 c0^4), so p_n = V_{k_n}[C_n sum p_m p_{n-m}]
  with V_k[f] = +int G_k f.
"""
from __future__ import annotations

import math

NP_PER_DB = 1.0 / (20.0 * math.log10(math.e))


def attenuation_np_per_m(f_hz: float, alpha0_db_m_mhz: float, eta: float) -> float:
    """Power-law amplitude attenuation alpha(f) in Np/m (Eq. 2.2, Table 2 units reading)."""
    return alpha0_db_m_mhz * (f_hz / 1.0e6) ** eta * NP_PER_DB


def wavenumber(n: int, f0: float, medium) -> complex:
    """Complex wavenumber of harmonic n: 2 pi n f0 / c0 + i alpha(n f0) (Section 2)."""
    f = n * f0
    return complex(2.0 * math.pi * f / medium.c0,
                   attenuation_np_per_m(f, medium.alpha0, medium.eta))


def source_coefficient(n: int, f0: float, medium) -> float:
    """C_n = -beta omega^2 n^2 / (2 rho0 c0^4), omega = 2 pi f0 (Eq. 2.6 with Eq. 3.2's sign)."""
    omega = 2.0 * math.pi * f0
    return -medium.beta * omega * omega * n * n / (2.0 * medium.rho0 * medium.c0 ** 4)
