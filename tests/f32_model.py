"""Rounding model of the FP32 pair force, for the tolerance of the mixed form.

The mixed form evaluates every pair term in FP32 from exact fixed-point
displacements and sums the terms without further error (float-float).  This
module evaluates the same terms with IEEE float32 numpy arithmetic (each
operation correctly rounded; exp and erfc correctly rounded from FP64), i.e.
the smallest error any FP32 evaluation of the pair terms can have, and sums
them in FP64.  Compared with the FP64 oracle it gives the FP32 floor of the
force error on a configuration, against which the parity tolerance of the
GPU's FP32 forces is set.  Test-side analysis only.
"""
import numpy as np
from scipy.special import erfc

KE = 14.3996454784   # e^2 / (4 pi eps0), eV A


def quantize(x, box):
    """Positions as the mixed form holds them: 30-bit fixed point per box edge."""
    box = np.asarray(box, np.float64)
    fix = np.round((np.asarray(x, np.float64) / box) % 1.0 * 2.0 ** 30).astype(np.int64) % (1 << 30)
    return fix, fix * (box / 2.0 ** 30)


def forces_model(x, types, box, pot, dtype=np.float32):
    """[N][3] forces (eV/A) of one periodic configuration from the fixed-point
    positions, every operation of the pair terms rounded to `dtype`
    (Buckingham, DSF Coulomb), the terms summed in FP64."""
    def fl(v):
        return np.asarray(v, dtype=dtype)
    f32 = dtype
    x = np.asarray(x, np.float64).reshape(-1, 3)
    types = np.asarray(types)
    box = np.asarray(box, np.float64)
    N = len(x)
    nt = len(pot["mass"])
    A = np.asarray(pot["buck_A"], np.float64).reshape(nt, nt)
    rho = np.asarray(pot["buck_rho"], np.float64).reshape(nt, nt)
    C = np.asarray(pot["buck_C"], np.float64).reshape(nt, nt)
    q = np.asarray(pot["charge"], np.float64)
    al, rc = float(pot["dsf_alpha"]), float(pot["r_cut"])
    fshift = erfc(al * rc) / rc ** 2 + 2 * al / np.sqrt(np.pi) * np.exp(-al * al * rc * rc) / rc
    fix, _ = quantize(x, box)   # exact integer displacements
    sc = fl(box / 2.0 ** 30)
    nmax = [int(np.ceil(rc / b)) for b in box]
    F = np.zeros((N, 3))
    for sx in range(-nmax[0], nmax[0] + 1):
        for sy in range(-nmax[1], nmax[1] + 1):
            for sz in range(-nmax[2], nmax[2] + 1):
                d = fix[None, :, :] - fix[:, None, :] + np.array([sx, sy, sz]) * (1 << 30)
                r2x = ((d * (box / 2.0 ** 30)) ** 2).sum(-1)
                m = (r2x < rc * rc) & (r2x > 0)
                if not m.any():
                    continue
                ii, jj = np.nonzero(m)
                dd = d[ii, jj]
                a, b = types[ii], types[jj]
                dx = fl(fl(dd.astype(f32)) * sc)
                r2 = fl(fl(dx[:, 0] * dx[:, 0]) + fl(fl(dx[:, 1] * dx[:, 1]) + fl(dx[:, 2] * dx[:, 2])))
                r = fl(np.sqrt(r2.astype(np.float64)))
                rinv = fl(1.0 / r.astype(np.float64))
                r2i = fl(rinv * rinv)
                r6i = fl(fl(r2i * r2i) * r2i)
                inv_rho = fl(np.where(A[a, b] != 0.0, 1.0 / rho[a, b], 0.0))
                ex = fl(np.exp(fl(-r * inv_rho).astype(np.float64)))
                gg = fl(np.exp(-(fl(fl(al * al) * r2)).astype(np.float64)))
                er = fl(erfc(fl(fl(al) * r).astype(np.float64)))
                qq = fl(KE * q[a] * q[b])
                fb = fl(fl(fl(A[a, b] * inv_rho.astype(np.float64)) * ex) - fl(fl(fl(6.0 * C[a, b]) * r6i) * rinv))
                fc = fl(fl(er * r2i) + fl(fl(fl(fl(2 * al / np.sqrt(np.pi)) * gg) * rinv) - fl(fshift)))
                fo = fl(fl(fl(qq * fc) + fb) * rinv)
                contrib = -(fo.astype(np.float64)[:, None] * dx.astype(np.float64))
                np.add.at(F, ii, contrib)
    return F
