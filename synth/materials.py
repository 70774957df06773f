"""Toy photon attenuation tables (input data, not part of the method).

The paper scales one XCOM value, mu/rho(Al, 1 MeV) = 0.06146 cm^2/g, by the
local density (Sec. 3.4, Eq. 9).  XCOM tables are not available here, so the
energy-dependent tables used by the transport workloads are synthetic:

* Compton: mu_C(E) = rho * (Z/A) * N_A * sigma_KN(E), with sigma_KN the
  closed-form Klein-Nishina total cross-section per electron;
* photoabsorption: mu_pe(E) = rho * k * E^-3 (E in MeV, k in cm^2/g).

Values are tabulated on 32 log-spaced energies from 10 keV to 20 MeV and
converted to 1/mm.  Both the oracle and the CUDA library receive the tables
as plain arrays and interpolate them themselves.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

N_AVOGADRO = 6.02214076e23          # 1/mol
R_ELECTRON_CM = 2.8179403262e-13    # classical electron radius, cm
ME_C2_MEV = 0.51099895              # electron rest energy, MeV
E_GRID_MEV = np.geomspace(0.01, 20.0, 32)


def klein_nishina_sigma_cm2(e_mev: np.ndarray) -> np.ndarray:
    """Total Klein-Nishina cross-section per electron (cm^2)."""
    a = np.asarray(e_mev, dtype=np.float64) / ME_C2_MEV
    l = np.log1p(2.0 * a)
    term = ((1.0 + a) / a**2) * (2.0 * (1.0 + a) / (1.0 + 2.0 * a) - l / a) + l / (2.0 * a) \
        - (1.0 + 3.0 * a) / (1.0 + 2.0 * a) ** 2
    return 2.0 * math.pi * R_ELECTRON_CM**2 * term


@dataclasses.dataclass
class Material:
    name: str
    density: float              # g/cm^3
    energies: np.ndarray        # MeV, increasing
    mu_compton: np.ndarray      # 1/mm
    mu_photo: np.ndarray        # 1/mm

    @property
    def n(self) -> int:
        return int(self.energies.shape[0])


def make_material(name: str, density: float, z_over_a: float, k_photo: float,
                  energies: np.ndarray = E_GRID_MEV) -> Material:
    e = np.asarray(energies, dtype=np.float64)
    mu_c = density * z_over_a * N_AVOGADRO * klein_nishina_sigma_cm2(e) * 0.1
    mu_p = density * k_photo * e**-3.0 * 0.1
    return Material(name, float(density), e.copy(), mu_c, mu_p)


def constant_material(name: str, density: float, mu_per_mm: float, energies=E_GRID_MEV) -> Material:
    """A material whose attenuation does not depend on energy (all Compton-free photoabsorption)."""
    e = np.asarray(energies, dtype=np.float64)
    return Material(name, float(density), e.copy(), np.zeros_like(e), np.full_like(e, mu_per_mm))


def vacuum(energies=E_GRID_MEV) -> Material:
    e = np.asarray(energies, dtype=np.float64)
    return Material("vacuum", 0.0, e.copy(), np.zeros_like(e), np.zeros_like(e))


def toy_materials() -> dict[str, Material]:
    """The five toy materials: water-, lead-, scintillator-, aluminium-like and vacuum."""
    return {
        "water": make_material("water", 1.0, 0.5551, 2e-4),
        "lead": make_material("lead", 11.35, 0.3958, 0.15),
        "scint": make_material("scint", 1.032, 0.5377, 2e-4),
        "al": make_material("al", 2.699, 0.4818, 2e-3),
        "vacuum": vacuum(),
    }
