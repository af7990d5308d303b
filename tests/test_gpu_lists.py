"""Verlet neighbour lists on the GPU.

* rebuilds decided and carried out on the device (inside the cooperative step
  launch, when the producer of the positions requested one) keep the forces
  equal to the oracle's brute force on the GPU's own configuration, in small
  boxes (several periodic images per pair) and larger ones, FP64 and mixed;
* the skin changes nothing but the summation order (FP64 trajectories with
  and without a skin agree to rounding);
* a cold crystal with the default skin rebuilds (almost) never;
* uploaded states: the state qtb_get_state reports (wrapped into the box) goes
  back without a rebuild, a moved ion forces one, and qtb_rebuild_lists
  rebuilds on demand without touching the state.
Bit-identical fused (graph) and unfused (single-step) stepping is checked by
test_gpu_parity.py::test_stepping_is_deterministic_and_split_invariant.
"""
import numpy as np
import pytest

from helpers import gpu_ctx, minimg, rel_inf, rel_l2
from paper_1905_02521_gb300 import workloads as W

pytestmark = pytest.mark.gpu

from tolerances import F32_INF, F32_L2  # noqa: E402


@pytest.fixture(scope="module")
def qtb():
    import torch
    assert torch.cuda.is_available()
    from paper_1905_02521_gb300 import build
    build.build()
    from paper_1905_02521_gb300 import qtb as q
    return q


@pytest.mark.parametrize("ncell", [2, 5])
@pytest.mark.parametrize("precision", [0, 1])
def test_rebuilds_keep_forces_exact(qtb, oracle, ncell, precision):
    # hot crystal (2000 K, white Langevin) with a small skin: ions cross skin/2
    # every few tens of steps; 300 direct steps, one captured block, 50 direct
    s, pot = W.mgo_system(ncell, 2000.0, sigma=0.05, seed=7)
    N = len(s["types"])
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=precision, seed=3, skin=0.3)
    try:
        r0 = qtb.qtb_list_rebuilds(ctx)
        assert r0 == 1
        for n in (300, 256, 50):
            qtb.qtb_step_n(ctx, n)
            x, _ = qtb.qtb_get_state(ctx, 0, 1, N)
            f = qtb.qtb_get_forces(ctx, 0, 1, N)[0]
            fo, eo, _ = oracle.pair_forces(x[0], s["types"], s["box"], pot)
            if precision == 0:
                assert rel_inf(f, fo) < 1e-12
            else:
                assert rel_l2(f, fo) < F32_L2 and rel_inf(f, fo) < F32_INF, (rel_l2(f, fo), rel_inf(f, fo))
        nreb = qtb.qtb_list_rebuilds(ctx) - r0
        print("ncell %d precision %d: %d rebuilds in 606 steps" % (ncell, precision, nreb))
        assert nreb >= 5
    finally:
        qtb.qtb_destroy(ctx)


def test_skin_only_changes_summation_order(qtb):
    s, pot = W.mgo_system(3, 300.0, seed=11)
    N = len(s["types"])
    out = []
    for skin in (-1.0, 0.8):      # no skin (rebuild whenever anything moved) / default
        ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=0, seed=21, skin=skin)
        try:
            qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, 513, 0.3)
            qtb.qtb_step_n(ctx, 512 + 40)
            out.append((qtb.qtb_get_state(ctx, 0, 1, N), qtb.qtb_list_rebuilds(ctx)))
        finally:
            qtb.qtb_destroy(ctx)
    (x0, v0), n0 = out[0]
    (x1, v1), n1 = out[1]
    assert n0 == 553 and n1 < n0
    assert np.abs(minimg(x1 - x0, s["box"])).max() < 1e-9
    assert rel_inf(v1, v0) < 1e-9


def test_cold_crystal_rarely_rebuilds(qtb):
    s, pot = W.mgo_system(4, 100.0)
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=1, filter_prec=1, seed=2)
    try:
        qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, 1025, 0.3)
        qtb.qtb_step_n(ctx, 1024)
        assert qtb.qtb_list_rebuilds(ctx) <= 3
    finally:
        qtb.qtb_destroy(ctx)


def test_pimd_beads_keep_their_images(qtb, oracle):
    # Mg ions sit on the box boundary: after a rebuild the beads of one ion can
    # be wrapped into different periodic images; the integrator must move each
    # bead within its own image (else every later step sees a box-length jump
    # and rebuilds).  Per-bead forces stay exact (1/P of the replica's forces).
    P = 4
    s, pot = W.mgo_system(3, 300.0, n_beads=P, seed=5)
    N = len(s["types"])
    ctx = gpu_ctx(qtb, [s], pot, 0.5, precision=0, seed=9, skin=0.4)
    try:
        qtb.qtb_step_n(ctx, 600)
        nreb = qtb.qtb_list_rebuilds(ctx)
        x, _ = qtb.qtb_get_state(ctx, 0, P, N)
        f = qtb.qtb_get_forces(ctx, 0, P, N)
        for b in range(P):
            fo, _, _ = oracle.pair_forces(x[b], s["types"], s["box"], pot)
            assert rel_inf(f[b], fo / P) < 1e-12
    finally:
        qtb.qtb_destroy(ctx)
    print("P = 4 MgO, skin 0.4: %d list rebuilds in 600 steps" % nreb)
    assert 2 <= nreb < 150


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("P", [8, 32])
def test_integrator_layouts_are_bit_identical(qtb, precision, P):
    # the compact and the wide layout of the ring-polymer integrator do the same
    # arithmetic per value: identical trajectories, through graph blocks and
    # direct launches (P = 32: four rows per thread task in both layouts)
    s, pot = W.mgo_system(3, 300.0, n_beads=P, seed=6)
    N = len(s["types"])
    out = []
    for layout in (1, 2):
        ctx = gpu_ctx(qtb, [s], pot, 0.5, precision=precision, filter_prec=1, seed=4, nm_layout=layout)
        try:
            qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB_PIMD, 513, 0.6)
            qtb.qtb_step_n(ctx, 256 + 37)
            out.append(qtb.qtb_get_state(ctx, 0, P, N))
        finally:
            qtb.qtb_destroy(ctx)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("precision", [0, 1])
def test_lane_counts_give_the_same_forces(qtb, oracle, precision):
    # 8, 16 or 32 lanes per bead-atom: the same terms summed in another order
    s, pot = W.mgo_system(3, 300.0, sigma=0.05, seed=12)
    N = len(s["types"])
    for lanes in (8, 16, 32):
        ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=precision, seed=3, list_lanes=lanes)
        try:
            qtb.qtb_step_n(ctx, 40)
            x, _ = qtb.qtb_get_state(ctx, 0, 1, N)
            f = qtb.qtb_get_forces(ctx, 0, 1, N)[0]
            fo, _, _ = oracle.pair_forces(x[0], s["types"], s["box"], pot)
            if precision == 0:
                assert rel_inf(f, fo) < 1e-12
            else:
                assert rel_l2(f, fo) < F32_L2 and rel_inf(f, fo) < F32_INF
        finally:
            qtb.qtb_destroy(ctx)


def test_autotune_picks_a_valid_configuration(qtb, oracle):
    from helpers import gpu_params
    s, pot = W.mgo_system(4, 300.0)
    params = gpu_params(pot, 1.0, precision=1, filter_prec=1, seed=5)
    # candidates timed from the state reached after two blocks (lists built on it)
    tuned, info = qtb.qtb_autotune([s], params, qtb.NOISE_QTB, 513, 0.3, n_blocks=1, equil_blocks=2)
    print("autotune:", info)
    assert info["n_tried"] == 1 + 4 * 3
    assert 0 < info["ms_per_step"] <= info["default_ms_per_step"]
    assert tuned["list_lanes"] in (0, 8, 16, 32) and tuned["skin"] in (0.0, 0.5, 0.8, 1.2, 1.6)
    assert tuned["rebuild_scope"] == 0          # one system: the scope is not a candidate
    N = len(s["types"])
    ctx = qtb.qtb_init([s], tuned)
    try:
        qtb.qtb_step_n(ctx, 300)
        x, _ = qtb.qtb_get_state(ctx, 0, 1, N)
        f = qtb.qtb_get_forces(ctx, 0, 1, N)[0]
        fo, _, _ = oracle.pair_forces(x[0], s["types"], s["box"], pot)
        assert rel_l2(f, fo) < F32_L2 and rel_inf(f, fo) < F32_INF
    finally:
        qtb.qtb_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1])
def test_state_round_trip_keeps_lists(qtb, oracle, precision):
    # between rebuilds positions move on without wrapping (the lists' periodic images
    # stay valid), while qtb_get_state reports them wrapped into the box: uploading
    # that state again must reproduce the stored one and keep the lists (ions on the
    # box-edge planes cross the edge within a few steps of every rebuild)
    s, pot = W.mgo_system(3, 300.0, seed=23)
    N = len(s["types"])
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=precision, seed=5)     # default skin 0.8 A
    try:
        for _ in range(3):
            qtb.qtb_step_n(ctx, 300)
            x0, v0 = qtb.qtb_get_state(ctx, 0, 1, N)
            f0 = qtb.qtb_get_forces(ctx, 0, 1, N)[0]
            r0 = qtb.qtb_list_rebuilds(ctx)
            qtb.qtb_set_state(ctx, 0, x0, v0)
            f1 = qtb.qtb_get_forces(ctx, 0, 1, N)[0]
            assert qtb.qtb_list_rebuilds(ctx) == r0
            x1, v1 = qtb.qtb_get_state(ctx, 0, 1, N)
            assert np.array_equal(v1, v0)
            if precision == 0:   # an ion across the box edge: one rounding of x -/+ L
                assert np.abs(minimg(x1 - x0, s["box"])).max() < 1e-12
            else:                # fixed point: exact
                assert np.array_equal(x1, x0)
            fo, _, _ = oracle.pair_forces(x1[0], s["types"], s["box"], pot)
            if precision == 0:
                assert rel_inf(f1, f0) < 1e-12 and rel_inf(f1, fo) < 1e-12
            else:
                assert rel_inf(f1, f0) < F32_INF
                assert rel_l2(f1, fo) < F32_L2 and rel_inf(f1, fo) < F32_INF
    finally:
        qtb.qtb_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1])
def test_forced_rebuild_keeps_the_state(qtb, oracle, precision):
    # qtb_rebuild_lists: one rebuild of every list on the current positions at the next
    # force evaluation; the state is unchanged, the forces and the steps that follow
    # match the oracle
    s, pot = W.mgo_system(3, 300.0, seed=29)
    N = len(s["types"])
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=precision, seed=6)
    try:
        qtb.qtb_step_n(ctx, 300)
        x0, v0 = qtb.qtb_get_state(ctx, 0, 1, N)
        r0 = qtb.qtb_list_rebuilds(ctx)
        qtb.qtb_rebuild_lists(ctx)
        f = qtb.qtb_get_forces(ctx, 0, 1, N)[0]
        assert qtb.qtb_list_rebuilds(ctx) == r0 + 1
        x1, v1 = qtb.qtb_get_state(ctx, 0, 1, N)
        assert np.array_equal(v1, v0)
        assert np.abs(minimg(x1 - x0, s["box"])).max() < 1e-12
        for step in (0, 256):
            qtb.qtb_step_n(ctx, step)
            x, _ = qtb.qtb_get_state(ctx, 0, 1, N)
            f = qtb.qtb_get_forces(ctx, 0, 1, N)[0]
            fo, _, _ = oracle.pair_forces(x[0], s["types"], s["box"], pot)
            if precision == 0:
                assert rel_inf(f, fo) < 1e-12
            else:
                assert rel_l2(f, fo) < F32_L2 and rel_inf(f, fo) < F32_INF
    finally:
        qtb.qtb_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1])
def test_uploaded_states_rebuild_only_when_needed(qtb, oracle, precision):
    # qtb_set_state keeps a system's lists while every uploaded bead-atom lies within
    # skin/2 of its position at the last rebuild (the stepping criterion), rebuilds
    # otherwise; the forces match the oracle either way
    s, pot = W.mgo_system(3, 300.0, seed=21)
    N = len(s["types"])
    ctx = gpu_ctx(qtb, [s], pot, 1.0, precision=precision, seed=9)     # default skin 0.8 A
    try:
        x0, v0 = qtb.qtb_get_state(ctx, 0, 1, N)
        r0 = qtb.qtb_list_rebuilds(ctx)
        tol = 1e-12 if precision == 0 else None
        for shift, rebuilt in ((0.0, 0), (0.1, 0), (0.5, 1)):
            x = x0.copy()
            x[0, 7, 0] += shift                        # one ion, inside or outside skin/2 = 0.4 A
            qtb.qtb_set_state(ctx, 0, x, v0)
            f = qtb.qtb_get_forces(ctx, 0, 1, N)[0]
            assert qtb.qtb_list_rebuilds(ctx) - r0 == rebuilt, shift
            r0 += rebuilt
            xg, _ = qtb.qtb_get_state(ctx, 0, 1, N)
            fo, _, _ = oracle.pair_forces(xg[0], s["types"], s["box"], pot)
            if tol:
                assert rel_inf(f, fo) < tol
            else:
                assert rel_l2(f, fo) < F32_L2 and rel_inf(f, fo) < F32_INF
    finally:
        qtb.qtb_destroy(ctx)


def test_minimum_image_variant_is_bit_identical(qtb):
    # a crystal whose cell exceeds twice (r_cut + 2 skin) runs alone on the step-kernel
    # variant that takes list displacements by minimum image; batched with a small cell
    # (which needs the image bits) the context uses the image-bit variant.  Each system
    # rebuilds on its own schedule, so the big crystal's trajectory must agree bit for bit
    s_big, pot = W.mgo_system(5, 300.0, seed=41)          # 21.05 A > 2 (8 + 1.6) A
    s_small, _ = W.mgo_system(2, 300.0, seed=42)          # 8.42 A
    N = len(s_big["types"])
    out = []
    for systems in ([s_big], [s_big, s_small]):
        ctx = gpu_ctx(qtb, systems, pot, 1.0, precision=1, filter_prec=1, seed=7)
        try:
            qtb.qtb_set_filter(ctx, 0, qtb.NOISE_QTB, 513, 0.3)
            qtb.qtb_step_n(ctx, 300)
            out.append(qtb.qtb_get_state(ctx, 0, 1, N) + (qtb.qtb_list_rebuilds(ctx),))
        finally:
            qtb.qtb_destroy(ctx)
    (xa, va, _), (xb, vb, _) = out
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
