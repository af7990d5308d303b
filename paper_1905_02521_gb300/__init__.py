"""GB300 (sm_103a) implementation of the quantum-thermal-bath MD hot path.

Method: Dammak, Hayoun, Brieuc, Geneste, "Nuclear quantum effects in molecular
dynamics simulations": QTB-MD (Eqs. 6-9) and QTB-PIMD (Eqs. 10-12).

* ``csrc/``     CUDA kernels and the C ABI (``include/qtb.h``), built by ``build.py``
* ``qtb``       thin ctypes binding with the C names (imports the built library)
* ``workloads`` seeded synthetic inputs (rock-salt crystals, oscillators)
"""
