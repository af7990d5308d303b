"""Edge cases of the GPU path (through the C ABI), against the oracle or exact laws.

* ragged systems: 61 ions (units of 8 and warps of 32 left partly empty, a net
  charge) with P = 1, 3 and 5 beads; FP64 trajectories against the oracle, and
  the record of the initial state (spring energy included);
* the smallest crystals: one ion (no pair within r_cut: zero force, constant
  potential), two ions (every interaction through periodic images);
* thermostat off (gamma = 0): the step conserves the total energy (one bead) or
  the ring-polymer Hamiltonian, and the total momentum, in both forms;
* qtb_step_n with zero steps changes nothing; a run split at every step equals
  one call bit for bit (one-bead and ring-polymer paths);
* the bounded device wait of the grid barriers gives up after about a second on
  a flag that nothing sets, reports it, and leaves the context usable.
"""
import numpy as np
import pytest

from helpers import gpu_ctx, minimg, oracle_sim, rel_inf
from paper_1905_02521_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qtb():
    import torch
    assert torch.cuda.is_available()
    from paper_1905_02521_gb300 import build
    build.build()
    from paper_1905_02521_gb300 import qtb as q
    return q


def _ragged(P, drop=(5, 17, 40)):
    s, pot = W.mgo_system(2, 300.0, n_beads=P)
    keep = np.setdiff1d(np.arange(s["pos"].shape[1]), drop)
    rng = np.random.default_rng(9)
    s = dict(s, pos=s["pos"][:, keep] + rng.normal(0, 0.01, (P, len(keep), 3)), vel=s["vel"][:, keep],
             types=s["types"][keep])
    return s, pot


@pytest.mark.parametrize("P", [1, 3, 5])
def test_ragged_system_fp64_trajectory(qtb, oracle, P):
    s, pot = _ragged(P)
    N = len(s["types"])
    assert N == 61
    ctx = gpu_ctx(qtb, [s], pot, 0.5, precision=0, seed=21)
    try:
        sim = oracle_sim(oracle, s, pot, 0.5, seed=21)
        # the record of the initial state (no integrator has run): springs included
        obs, oo = qtb.qtb_observables(ctx, 0), sim.observe()
        for k in (1, 2, 3, 4, 18, 19):
            assert obs[k] == pytest.approx(oo[k], rel=1e-10, abs=1e-10), k
        qtb.qtb_step_n(ctx, 40)
        sim.step(40, record=False)
        xg, vg = qtb.qtb_get_state(ctx, 0, P, N)
        fg = qtb.qtb_get_forces(ctx, 0, P, N)
        xo, vo, fo, _ = sim.state()
        assert np.abs(minimg(xg - xo, s["box"])).max() < 1e-10
        assert rel_inf(vg, vo) < 1e-11 and rel_inf(fg, fo) < 1e-11
        obs, oo = qtb.qtb_observables(ctx, 0), sim.observe()
        for k in (1, 2, 3, 4, 18, 19):
            assert obs[k] == pytest.approx(oo[k], rel=1e-10, abs=1e-10)
    finally:
        qtb.qtb_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1])
def test_one_and_two_ion_crystals(qtb, oracle, precision):
    pot = W.mgo_potential()
    box = np.array([8.42, 8.42, 8.42])
    for pos, types in ((np.array([[1.0, 2.0, 3.0]]), np.array([0], np.int32)),
                       (np.array([[1.0, 2.0, 3.0], [3.3, 2.1, 2.9]]), np.array([0, 1], np.int32))):
        s = W.system(pos, types, box, pot, 300.0, 1e-3)
        N = len(types)
        ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=precision, seed=3)
        try:
            f0 = qtb.qtb_get_forces(ctx, 0, 1, N)[0]
            x0, _ = qtb.qtb_get_state(ctx, 0, 1, N)
            fo, eo, _ = oracle.pair_forces(x0[0], types, box, pot)
            if N == 1:
                assert np.all(f0 == 0.0)                       # no other ion within r_cut
            tol = 1e-12 if precision == 0 else 1e-5
            assert np.abs(f0 - fo).max() <= tol * max(np.abs(fo).max(), 1.0)
            assert qtb.qtb_observables(ctx, 0)[2] == pytest.approx(eo, rel=10 * tol, abs=10 * tol)
            qtb.qtb_step_n(ctx, 100)
            obs = qtb.qtb_observables(ctx, 0)
            assert np.all(np.isfinite(obs)) and obs[0] == 100
        finally:
            qtb.qtb_destroy(ctx)


@pytest.mark.parametrize("precision,P", [(0, 1), (1, 1), (0, 4), (1, 4)])
def test_thermostat_off_conserves_energy_and_momentum(qtb, precision, P):
    s, pot = W.mgo_system(3, 300.0, gamma=0.0, n_beads=P)
    rng = np.random.default_rng(4)
    s["pos"] = s["pos"] + (rng.normal(0, 0.01, s["pos"].shape) if P > 1 else 0.0)
    dt = 1.0 if P == 1 else 0.25
    ctx = gpu_ctx(qtb, [s], pot, dt, precision=precision, seed=2, max_records=4096)
    try:
        r0 = qtb.qtb_observables(ctx, 0)
        qtb.qtb_step_n(ctx, 2000)
        ser = qtb.qtb_get_series(ctx, 0, 4096)
    finally:
        qtb.qtb_destroy(ctx)
    H = ser[:, 1] + ser[:, 2] + (ser[:, 3] if P > 1 else 0.0)     # ring polymer: springs too
    H0 = r0[1] + r0[2] + (r0[3] if P > 1 else 0.0)
    assert np.abs(H - H0).max() < 2e-3 * r0[1]
    mom_tol = 1e-9 if precision == 0 else 1e-4 * np.sqrt(r0[1])
    assert np.abs(ser[:, 14:17] - r0[14:17]).max() < mom_tol


@pytest.mark.parametrize("P", [1, 4])
def test_zero_steps_and_step_by_step_splitting(qtb, P):
    s, pot = W.mgo_system(2, 300.0, n_beads=P)
    N = len(s["types"])
    out = []
    for split in ([0, 70], [1] * 70):
        ctx = gpu_ctx(qtb, [s], pot, 0.5, precision=1, seed=6)
        try:
            if P == 1:
                qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, 257, 0.3)
            else:
                qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB_PIMD, 257, 0.6)
            before = qtb.qtb_get_state(ctx, 0, P, N)
            qtb.qtb_step_n(ctx, 0)
            assert qtb.qtb_get_step(ctx) == 0
            after = qtb.qtb_get_state(ctx, 0, P, N)
            assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
            for n in split:
                qtb.qtb_step_n(ctx, n)
            out.append(qtb.qtb_get_state(ctx, 0, P, N))
        finally:
            qtb.qtb_destroy(ctx)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_bounded_wait_gives_up_and_the_context_stays_usable(qtb):
    s, pot = W.mgo_system(2, 300.0)
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=1, seed=7)
    try:
        gave_up, ms = qtb.qtb_wait_selftest(ctx)
        assert gave_up and 500.0 < ms < 5000.0, (gave_up, ms)
        qtb.qtb_step_n(ctx, 20)
        qtb.qtb_sync(ctx)                              # no error recorded in the context
        obs = qtb.qtb_observables(ctx, 0)
        assert obs[0] == 20 and np.all(np.isfinite(obs))
    finally:
        qtb.qtb_destroy(ctx)


def test_fp32_peak_is_measured_and_plausible(qtb):
    # the step kernel's roofline denominator: FMA chains filling every SM; between
    # half and 1.05 of the nominal 152 SMs x 128 lanes x 2 flops at the highest SM
    # clock this GPU reports
    import torch
    t, ms = qtb.qtb_fp32_peak()
    mhz = torch.cuda.get_device_properties(0).clock_rate / 1e3 if hasattr(
        torch.cuda.get_device_properties(0), "clock_rate") else 2070.0
    nominal = 152 * 128 * 2 * max(mhz, 2070.0) * 1e6 / 1e12
    print(f"FP32 FMA peak {t:.1f} TFLOP/s in {ms:.2f} ms (nominal {nominal:.1f})")
    assert 0.5 * nominal < t < 1.05 * nominal
    assert ms > 0.5
