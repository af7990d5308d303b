"""Seeded synthetic inputs: rock-salt crystals, oscillator ensembles, parameter sets.

This module only generates inputs (lattices, seeded perturbations, seeded
Maxwell-Boltzmann velocities, potential parameter tables).  It holds none of
the method's arithmetic, and both the CUDA path and the oracle consume what it
produces.

Workloads (synthetic stand-ins for the crystals the paper simulates, Sec. 2.2):

* MgO rock salt, a = 4.21 A, charges +-2 e; Buckingham Mg-O A = 1428.5 eV,
  rho = 0.2945 A; O-O A = 22764 eV, rho = 0.149 A, C = 27.88 eV A^6; DSF
  Coulomb alpha = 0.2 1/A, r_c = 8 A.
* LiH / LiD rock salt, a = 4.08 A, charges +-1 e; Li-H A = 300 eV, rho = 0.30 A;
  H-H A = 150 eV, rho = 0.35 A, C = 5 eV A^6; same alpha and r_c as MgO.
* Quartic double wells V0 (x^2/a^2 - 1)^2, V0 = 0.1 eV, a = 0.5 A, m = 1.008 u,
  one independent well per Cartesian component.
"""
from __future__ import annotations

import numpy as np

KB = 8.617333262e-5            # eV/K
MVV2E = 103.64269652680505     # eV per u A^2/fs^2

MASS = {"Mg": 24.305, "O": 15.999, "Li": 7.016, "H": 1.008, "D": 2.014}


def _pot(names, charges, buck, alpha=0.2, r_cut=8.0):
    nt = len(names)
    A = np.zeros((nt, nt))
    rho = np.ones((nt, nt))
    Cc = np.zeros((nt, nt))
    for (a, b), (AA, rr, CC) in buck.items():
        for i, j in ((a, b), (b, a)):
            A[i, j], rho[i, j], Cc[i, j] = AA, rr, CC
    return {
        "names": list(names),
        "mass": np.array([MASS[n] for n in names]),
        "charge": np.array(charges, dtype=np.float64),
        "buck_A": A, "buck_rho": rho, "buck_C": Cc,
        "dsf_alpha": alpha, "r_cut": r_cut,
    }


def mgo_potential():
    # type 0 = Mg, 1 = O
    return _pot(["Mg", "O"], [2.0, -2.0], {(0, 1): (1428.5, 0.2945, 0.0), (1, 1): (22764.0, 0.149, 27.88)})


def lih_potential(isotope="H"):
    # type 0 = Li, 1 = H (or D: same Born-Oppenheimer surface, heavier mass)
    p = _pot(["Li", isotope], [1.0, -1.0], {(0, 1): (300.0, 0.30, 0.0), (1, 1): (150.0, 0.35, 5.0)})
    return p


def rocksalt(ncell, a, sigma=0.02, seed=777):
    """ncell^3 conventional cells: cation (type 0) on fcc sites, anion (type 1)
    shifted by (a/2, 0, 0); every coordinate perturbed by N(0, sigma^2)."""
    fcc = np.array([[0, 0, 0], [0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]])
    g = np.stack(np.meshgrid(np.arange(ncell), np.arange(ncell), np.arange(ncell), indexing="ij"), -1).reshape(-1, 3)
    cat = (g[:, None, :] + fcc[None, :, :]).reshape(-1, 3)
    ani = cat + np.array([0.5, 0.0, 0.0])
    pos = np.concatenate([cat, ani]) * a
    types = np.concatenate([np.zeros(len(cat), np.int32), np.ones(len(ani), np.int32)])
    box = np.array([ncell * a] * 3, dtype=np.float64)
    rng = np.random.default_rng(seed)
    pos = pos + rng.normal(0.0, sigma, pos.shape)
    pos = np.mod(pos, box)
    return pos, types, box


def maxwell_boltzmann(masses, T, seed, n_beads=1):
    """Velocities [P, N, 3] (A/fs) drawn at temperature T, zero total momentum per bead."""
    rng = np.random.default_rng(seed)
    m = np.asarray(masses, dtype=np.float64)
    sd = np.sqrt(KB * T / (m * MVV2E))
    v = rng.normal(0.0, 1.0, (n_beads, len(m), 3)) * sd[None, :, None]
    if len(m) > 1:
        ptot = (v * m[None, :, None]).sum(1, keepdims=True)
        v = v - ptot / m.sum()
    return v


def beads_from(pos, n_beads):
    """All P beads start on the classical position."""
    return np.repeat(np.asarray(pos, np.float64)[None], n_beads, axis=0)


def system(pos, types, box, pot, T, gamma, n_beads=1, vel_seed=4242, vel=None):
    """A system description consumed by both the library binding and the oracle."""
    masses = pot["mass"][types]
    beads = beads_from(pos, n_beads)
    if vel is None:
        vel = maxwell_boltzmann(masses, T, vel_seed, n_beads)
    return {"pos": beads, "vel": np.asarray(vel, np.float64), "types": np.asarray(types, np.int32),
            "box": np.asarray(box, np.float64), "T": float(T), "gamma": float(gamma)}


def mgo_system(ncell, T, gamma=1e-3, n_beads=1, sigma=0.02, seed=777, vel_seed=4242):
    pot = mgo_potential()
    pos, types, box = rocksalt(ncell, 4.21, sigma, seed)
    return system(pos, types, box, pot, T, gamma, n_beads, vel_seed), pot


def lih_system(ncell, T, gamma=1e-3, n_beads=1, isotope="H", sigma=0.02, seed=777, vel_seed=4242):
    pot = lih_potential(isotope)
    pos, types, box = rocksalt(ncell, 4.08, sigma, seed)
    return system(pos, types, box, pot, T, gamma, n_beads, vel_seed), pot


def well_potential(mass=1.008):
    return {"names": ["H"], "mass": np.array([mass]), "charge": np.zeros(1), "buck_A": np.zeros((1, 1)),
            "buck_rho": np.ones((1, 1)), "buck_C": np.zeros((1, 1)), "dsf_alpha": 0.0, "r_cut": 0.0}


def oscillators(n_atoms, T, gamma, n_beads=1, x0=0.0, spread=0.0, seed=99, mass=1.008, vel_seed=4243):
    """n_atoms particles in a separable external potential: 3 n_atoms 1-D oscillators."""
    pot = well_potential(mass)
    rng = np.random.default_rng(seed)
    pos = x0 + spread * rng.normal(size=(n_atoms, 3))
    types = np.zeros(n_atoms, np.int32)
    return system(pos, types, np.zeros(3), pot, T, gamma, n_beads, vel_seed), pot


# The benchmark configurations (synthetic stand-ins, sizes as stated).
CONFIGS = {
    "mgo_2x2x2_qtb_fp64": dict(kind="mgo", ncell=2, T=300.0, gamma=1e-3, dt=1.0, steps=2000, n_taps=513,
                               omega_max=0.3, n_beads=1),
    "mgo_10x10x10_qtb_mixed": dict(kind="mgo", ncell=10, T=100.0, gamma=1e-3, dt=1.0, steps=100000, n_taps=2049,
                                   omega_max=0.3, n_beads=1),
    "lih_6x6x6_qtbpimd_p8": dict(kind="lih", ncell=6, T=50.0, gamma=1e-3, dt=0.25, steps=40000, n_taps=2049,
                                 omega_max=0.6, n_beads=8),
    "lih_6x6x6_pimd_p32": dict(kind="lih", ncell=6, T=50.0, gamma=1e-3, dt=0.25, steps=40000, n_taps=0,
                               omega_max=0.6, n_beads=32),
}


def sweep_systems(n_systems=64, gamma=1e-3, sigma=0.02):
    """Heat-capacity sweep: MgO of 3..8 cells per side at T_i = 10 * 150^(i/63) K."""
    out = []
    for i in range(n_systems):
        ncell = 3 + (i % 6)
        T = 10.0 * 150.0 ** (i / max(n_systems - 1, 1))
        s, pot = mgo_system(ncell, T, gamma, 1, sigma, seed=777 + i, vel_seed=4242 + i)
        out.append(s)
    return out, mgo_potential()
