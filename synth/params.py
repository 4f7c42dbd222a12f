"""Parameter set P0 of the EMT6/Ro spheroid cellular automaton (build reading).

The paper fixes the medium the spheroids sit in (glucose 5.5 mM, oxygen 0.28 mM,
pH 7.4; "The tumour case library" section) and the time step (600 CA steps per
hour; "GA Resolution, constraints" section). Every other constant of the model
lives in the earlier publications the paper defers to ("Underlying model"
section), which are not available here. The values below are therefore THIS
BUILD'S OWN READING, chosen so that an untreated spheroid grows, turns hypoxic
and quiescent in its core and responds to dose fractions. They are not, and do
not claim to be, the published calibration.

This module holds values only: no arithmetic of the method. Both the FP64
oracle and the CUDA library receive these numbers as inputs and derive any
internal quantities (steps per phase, H+ concentrations from pH) themselves.
"""
from __future__ import annotations

import dataclasses

STEPS_PER_HOUR = 600  # paper: each hour is split into 600 steps of model time

# kinds of a lattice site (cell word bits 0..2)
EMPTY, G1, S, G2, M, Q = 0, 1, 2, 3, 4, 5

# model switches (bit flags), used by tests to isolate one mechanism
F_DIVISION = 1 << 0
F_DEATH = 1 << 1
F_QUIESCENCE = 1 << 2
F_REACTION = 1 << 3
F_DIFFUSION = 1 << 4
F_DOOM_IMMEDIATE = 1 << 5   # variant: lethal hits die at once instead of at mitosis
F_DEFAULT = F_DIVISION | F_DEATH | F_QUIESCENCE | F_REACTION | F_DIFFUSION


@dataclasses.dataclass
class Params:
    # cell cycle: phase durations in hours (G1, S, G2, M)
    dur_h: tuple = (9.0, 6.0, 2.0, 1.0)
    # explicit diffusion: substeps per CA step and per-substep diffusion numbers
    # lambda = D*dt_sub/dx^2 for (O2, glucose, H+); 3-D FTCS needs lambda <= 1/6
    n_sub: int = 4
    lam: tuple = (0.15, 0.05, 0.10)
    # medium (paper): oxygen mM, glucose mM, pH
    medium_O: float = 0.28
    medium_G: float = 5.5
    medium_pH: float = 7.4
    # metabolism, per substep per cell (mM per substep)
    q_O: float = 6.0e-4     # maximal O2 uptake
    K_O: float = 5.0e-3     # O2 half-saturation (mM)
    q_G: float = 1.5e-3     # maximal aerobic glucose uptake
    K_G: float = 0.05       # glucose half-saturation (mM)
    k_an: float = 3.0       # glycolytic boost under anoxia
    O_an: float = 0.02      # O2 level at which the anaerobic weight is 1/2 (mM)
    q_H: float = 2.0e-5     # H+ released per unit of anaerobic glucose uptake
    f_Q: float = 0.5        # quiescent uptake relative to proliferating
    # irradiation: linear-quadratic survival with phase and oxygen modifiers
    alpha: float = 0.3      # Gy^-1
    beta: float = 0.03      # Gy^-2
    omf_m: float = 3.0      # maximal oxygen enhancement
    omf_K: float = 4.0e-3   # O2 level of half effect (mM)
    phi: tuple = (1.0, 0.6, 1.4, 1.6, 0.8)  # G1, S, G2, M, Q
    # thresholds: quiescence and death
    O_q: float = 0.01
    G_q: float = 0.1
    pH_q: float = 6.8
    G_d: float = 0.02
    pH_d: float = 6.4
    # sublethal-damage repair half-time (h); 0 = complete repair between fractions
    repair_half_h: float = 0.0
    flags: int = F_DEFAULT

    def replace(self, **kw) -> "Params":
        return dataclasses.replace(self, **kw)


P0 = Params()

# Physical-rate diffusion variant (build reading, not the paper's numbers):
# oxygen spreads D dt / dx^2 ~ 20-50 lattice units per 6 s step at 10-20 um
# sites, far more than P0's coarse-grained 4 x 0.15.  Modelled with many
# explicit substeps at P0's per-substep lambda (O2: 128 x 0.15 = 19.2 per
# step) and the per-substep uptake scaled by 4/128, so that a cell consumes
# per step what it consumes under P0 while the fields relax towards their
# quasi-steady profile within each step.
P_PHYS = P0.replace(n_sub=128, q_O=P0.q_O * 4 / 128, q_G=P0.q_G * 4 / 128)

