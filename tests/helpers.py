"""Shared test plumbing: build GPU contexts and oracle simulations from the same
seeded workload dictionaries (paper_1905_02521_gb300.workloads)."""
import numpy as np


def gpu_params(pot, dt, precision=0, filter_prec=1, seed=12345, potential=0, ext=None, obs_stride=1,
               max_records=4096, skin=0.0, nm_layout=0, list_lanes=0, rebuild_scope=0, npt=None):
    p = {k: pot[k] for k in ("mass", "charge", "buck_A", "buck_rho", "buck_C")}
    p.update(dsf_alpha=pot["dsf_alpha"], r_cut=pot["r_cut"], dt=dt, precision=precision, filter_prec=filter_prec,
             seed=seed, potential=potential, obs_stride=obs_stride, max_records=max_records, skin=skin,
             nm_layout=nm_layout, list_lanes=list_lanes, rebuild_scope=rebuild_scope)
    if npt is not None:   # isothermal-isobaric cell: dict(pressure, mass, gamma), as the oracle's
        p.update(npt=1, pressure=npt["pressure"], cell_mass=npt["mass"], cell_gamma=npt["gamma"])
    ext = ext or {}
    p["ext_omega"] = ext.get("omega", 0.0)
    p["ext_V0"] = ext.get("V0", 0.0)
    p["ext_a"] = ext.get("a", 1.0)
    return p


def gpu_ctx(qtb, systems, pot, dt, **kw):
    return qtb.qtb_init(systems, gpu_params(pot, dt, **kw))


def oracle_sim(oracle, s, pot, dt, seed=12345, sys=0, taps=None, potential=0, ext=None, npt=None):
    return oracle.Sim(s["pos"], s["vel"], s["types"], pot, s["box"] if potential == 0 else None, s["T"], s["gamma"],
                      dt, seed=seed, sys=sys, taps=taps, potential=potential, ext=ext, npt=npt)


def minimg(d, box):
    box = np.asarray(box, np.float64)
    return d - box * np.round(d / box)


def rel_l2(a, b):
    """||a - b||_2 / ||b||_2  (relative error of a vector)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())


def rel_inf(a, b):
    """max |a - b| / RMS(b)  (norm-wise relative error)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b).max() / np.sqrt((b ** 2).mean())
