"""Reduced units of the oracle (TEST INFRASTRUCTURE ONLY).

Sec 2.3.3 / Table 1: the Bjerrum length is l_B = e^2 / (4 pi eps0 eps k_B T).
With e^2/(4 pi eps0) = 1.43996454784 eV nm and k_B = 8.617333262e-5 eV/K
(CODATA 2018), Table 1's 4.514 nm at 223 K and eps = 16.6 follow.
Potentials are in kT/e and lengths in grid spacings h.
"""
COULOMB_EV_NM = 1.43996454784     # e^2 / (4 pi eps0) in eV nm
KB_EV_PER_K = 8.617333262e-5      # Boltzmann constant in eV / K
E_CHARGE_C = 1.602176634e-19     # elementary charge in C (exact in the SI)


def beta_per_ev(temperature_K: float) -> float:
    """Thermodynamic beta 1/(k_B T) in 1/eV."""
    return 1.0 / (KB_EV_PER_K * temperature_K)


def bjerrum_length_nm(temperature_K: float, eps_r: float) -> float:
    return COULOMB_EV_NM / (eps_r * KB_EV_PER_K * temperature_K)


def bjerrum_length_h(temperature_K: float, eps_r: float, h_nm: float) -> float:
    """l_B in units of the grid spacing h (h_nm = h in nm)."""
    return bjerrum_length_nm(temperature_K, eps_r) / h_nm
