"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bar (FP64 path): relative L2 temperature error <= 1e-9 on both levels, and
element states bit-exact except where an element mean lies within 1e-6 K of
T_melt in either run (ties are counted and must be zero on these inputs).
"""
import numpy as np
import pytest

from oracle import twolevel as TL
from paper_2110_12932_gb300 import build as tlbuild
from paper_2110_12932_gb300 import tl, workloads

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def lib():
    tlbuild.build()
    return tl.load()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def compare(prob, ref, what=""):
    Tf, org = prob.temperature(tl.TL_FINE)
    Tc, _ = prob.temperature(tl.TL_COARSE)
    assert tuple(org) == tuple(ref.origin), (what, org, ref.origin)
    ef, ec = rel(Tf, ref.Tf), rel(Tc, ref.Tc)
    assert ef <= TOL and ec <= TOL, (what, ef, ec)
    sf = prob.state(tl.TL_FINE)
    sc = prob.state(tl.TL_COARSE)
    ref_sf = ref.fine_state().reshape(-1)
    mesh = ref.fine_mesh()
    tie_f = np.abs(mesh.element_mean(ref.Tf) - ref.cfg["T_melt"]) < 1e-6
    tie_c = np.abs(ref.coarse.element_mean(ref.Tc) - ref.cfg["T_melt"]) < 1e-6
    assert tie_f.sum() == 0 and tie_c.sum() == 0, (what, "threshold ties")
    assert np.array_equal(sf, ref_sf), (what, np.count_nonzero(sf != ref_sf))
    assert np.array_equal(sc, ref.state_c), (what, np.count_nonzero(sc != ref.state_c))
    return ef, ec


def run_both(cfg, nmacro, check_every=1):
    prob = tl.Problem(cfg)
    ref = TL.TwoLevel(cfg)
    errs = []
    done = 0
    while done < nmacro:
        k = min(check_every, nmacro - done)
        prob.macro_steps(k)
        ref.run(k)
        done += k
        errs.append(compare(prob, ref, f"macro {done}"))
    return prob, ref, errs


def test_single_track_tiny_full_run():
    cfg = workloads.workload("single_track_tiny")
    prob, ref, errs = run_both(cfg, cfg["macro_steps"], check_every=5)
    st = prob.stats()
    assert st["macro_steps"] == 50 and st["substeps"] == 200
    assert st["patch_moves"] > 0
    melted = np.count_nonzero(ref.state_map == TL.MELTED)
    assert melted > 0
    prob.close()


def test_energy_account_matches_oracle_and_identity():
    cfg = workloads.workload("single_track_tiny")
    prob, ref, _ = run_both(cfg, 12, check_every=12)
    st = prob.stats()
    for lvl in ("fine", "coarse"):
        s, l, f = (st[f"energy_{lvl}_{k}"] for k in ("stored", "laser", "flux"))
        assert abs(s - l - f) <= 1e-9 * max(abs(s), abs(l)), lvl
        for k in ("stored", "laser", "flux"):
            o = ref.energy[f"{lvl}_{k}"]
            assert abs(st[f"energy_{lvl}_{k}"] - o) <= 1e-8 * max(abs(o), abs(l)), (lvl, k)
    prob.close()


def test_ragged_tiles_and_odd_ratios():
    # 15 x 9 x 9 fine elements: ragged y tiles; r = 3, m = 3
    cfg = workloads.workload("single_track_tiny", NXc=13, NYc=7, NZc=5, Lx=13 * 125e-6,
                             Ly=7 * 125e-6, Lz=5 * 125e-6, pNXc=5, pNYc=3, pNZc=3, r=3, m=3,
                             tracks=[(0.0, 0.45e-3, 13 * 125e-6, 0.45e-3, 0.8)], macro_steps=10)
    run_both(cfg, 10, check_every=5)


def test_several_x_tiles():
    # 36 x 12 x 8 fine elements: two x tiles (32 + 4) and two y tiles (8 + 4)
    cfg = workloads.workload("single_track_tiny", pNXc=9, pNYc=3, pNZc=2, r=4, m=2)
    run_both(cfg, 8, check_every=4)


def test_patch_covering_plate_is_single_level():
    cfg = workloads.workload("single_track_tiny", NXc=8, NYc=4, NZc=2, pNXc=8, pNYc=4, pNZc=2,
                             r=2, m=2)
    prob, ref, _ = run_both(cfg, 6, check_every=3)
    sl = TL.SingleLevel(cfg, 16, 8, 4, cfg["dt_coarse"] / 2)
    for _ in range(12):
        sl.step()
    Tf, _ = prob.temperature(tl.TL_FINE)
    assert rel(Tf, sl.T) <= TOL


def test_unit_ratios_gaussian_coarse_source():
    cfg = workloads.workload("single_track_tiny", r=1, m=1, coarse_source=1, pNXc=6, pNYc=4, pNZc=2)
    run_both(cfg, 20, check_every=10)


def test_literal_bc_weight_and_laser_off_tail():
    # printed weight i/m; the scan ends before the run does (laser off, patch parked)
    cfg = workloads.workload("single_track_tiny", bc_weight_literal=1,
                             tracks=[(0.2e-3, 0.5e-3, 1.0e-3, 0.5e-3, 0.8)])
    run_both(cfg, 24, check_every=8)


def test_alternating_tracks_whole_scan():
    """Three alternating 1.03 mm tracks (hatch 100 um < the 500 um patch) on
    the 2 x 1 x 0.5 mm plate with the box source on the coarse level, run to
    past the end of the scan and compared after every macro step: the coarse
    source split between two tracks in the macro steps that hold a turn
    (the 26th and the 52nd; the scan ends in the 78th), the patch turning
    round, and the patch returning over material the previous track
    consolidated (the plate-wide fine state map)."""
    cfg = workloads.workload("single_track_tiny", coarse_source=0,
                             tracks=workloads.raster_tracks(0.5e-3, 1.53e-3, 0.5e-3, 3, 100e-6, 0.8))
    prob = tl.Problem(cfg)
    ref = TL.TwoLevel(cfg)
    revisited = 0
    first_track = None
    for n in range(82):
        prob.macro_steps(1)
        ref.run(1)
        compare(prob, ref, f"macro {n + 1}")
        if n + 1 == 25:  # the first track ends during the 26th step
            first_track = ref.state_map == TL.MELTED
        if n + 1 >= 32:  # back over the first track's melt, 100 um aside
            o, r = ref.origin, ref.r
            win = ref.fine_state()
            revisited += int(np.count_nonzero(first_track[:, o[1] * r:o[1] * r + win.shape[1],
                                                          o[0] * r:o[0] * r + win.shape[2]]))
    assert revisited > 0
    st = prob.stats()
    assert st["patch_moves"] >= 10
    s, l, f = (st[f"energy_coarse_{k}"] for k in ("stored", "laser", "flux"))
    assert abs(s - l - f) <= 1e-9 * max(abs(s), abs(l))
    assert abs(l - ref.energy["coarse_laser"]) <= 1e-9 * abs(l)
    prob.close()


def test_no_tracks_stays_at_initial_temperature():
    cfg = workloads.workload("single_track_tiny", tracks=[])
    prob = tl.Problem(cfg)
    prob.macro_steps(3)
    Tf, org = prob.temperature(tl.TL_FINE)
    assert np.all(Tf == cfg["T0"])
    assert tuple(org) == (6, 2, 2)
    prob.close()


def test_multitrack_10mm_first_macro_step():
    """Full-size fine patch (65 x 65 x 33 nodes) and coarse plate
    (81 x 41 x 17), same launch configuration as the benchmark."""
    cfg = workloads.workload("multitrack_10mm")
    prob = tl.Problem(cfg)
    ref = TL.TwoLevel(cfg, energy=False)
    prob.macro_steps(1)
    ref.run(1)
    compare(prob, ref, "macro 1")
    prob.close()


def test_call_order_is_enforced():
    cfg = workloads.workload("single_track_tiny")
    prob = tl.Problem(cfg)
    h = prob.h
    assert tl.tl_fine_substeps(h, 1) == tl.TL_ESTATE
    assert tl.tl_restrict(h) == tl.TL_ESTATE
    assert tl.tl_coarse_step(h, tl.TL_CORRECT) == tl.TL_ESTATE
    assert tl.tl_coarse_step(h, tl.TL_PREDICT) == tl.TL_OK
    assert tl.tl_coarse_step(h, tl.TL_PREDICT) == tl.TL_ESTATE
    assert tl.tl_fine_substeps(h, cfg["m"] + 1) == tl.TL_ESTATE
    assert tl.tl_fine_substeps(h, 2) == tl.TL_OK
    assert tl.tl_restrict(h) == tl.TL_ESTATE
    assert tl.tl_fine_substeps(h, 2) == tl.TL_OK
    assert tl.tl_restrict(h) == tl.TL_OK
    assert tl.tl_coarse_step(h, tl.TL_CORRECT) == tl.TL_OK
    assert tl.tl_sync(h) == tl.TL_OK
    prob.close()


def test_iteration_cap_reports_noconv_and_leaves_state():
    cfg = workloads.workload("single_track_tiny", max_iter=1)
    prob = tl.Problem(cfg)
    T0f, _ = prob.temperature(tl.TL_FINE)
    assert tl.tl_macro_steps(prob.h, 1) == tl.TL_ENOCONV
    Tf, _ = prob.temperature(tl.TL_FINE)
    Tc, _ = prob.temperature(tl.TL_COARSE)
    assert np.array_equal(Tf, T0f)
    assert np.all(Tc == cfg["T0"])
    prob.close()


def test_deterministic_reruns():
    cfg = workloads.workload("single_track_tiny")
    out = []
    for _ in range(2):
        prob = tl.Problem(cfg)
        prob.macro_steps(10)
        out.append(prob.temperature(tl.TL_FINE)[0])
        prob.close()
    assert np.array_equal(out[0], out[1])


# ---- precision form: FP32 inner CG with FP64 defect correction -------------
# Bar: relative L2 <= 1e-6 against the FP64 oracle (the form's stated
# accuracy); the outer residual tolerance 1e-10 typically gives ~1e-10.

REFINED_TOL = 1e-6


@pytest.mark.parametrize("inner_tiles", [1, 2])
def test_refined_single_track_tiny_against_oracle(inner_tiles):
    cfg = workloads.workload("single_track_tiny", precision=tl.TL_FP32_REFINED, tol=1e-10, tol_inner=1e-5,
                             inner_tiles=inner_tiles)
    prob = tl.Problem(cfg)
    ref = TL.TwoLevel(cfg, energy=False)
    for _ in range(5):
        prob.macro_steps(10)
        ref.run(10)
        Tf, org = prob.temperature(tl.TL_FINE)
        Tc, _ = prob.temperature(tl.TL_COARSE)
        assert tuple(org) == tuple(ref.origin)
        assert rel(Tf, ref.Tf) <= REFINED_TOL and rel(Tc, ref.Tc) <= REFINED_TOL
        assert np.array_equal(prob.state(tl.TL_FINE), ref.fine_state().reshape(-1))
    st = prob.stats()
    assert st["outer_iters_fine"] >= st["solves_fine"]
    prob.close()


def test_refined_matches_fp64_gpu_path_multitrack():
    base = workloads.workload("multitrack_10mm")
    p64 = tl.Problem(dict(base, precision=tl.TL_FP64, tol=1e-12))
    p32 = tl.Problem(dict(base, precision=tl.TL_FP32_REFINED, tol=1e-10, tol_inner=1e-5))
    p64.macro_steps(6)
    p32.macro_steps(6)
    a, _ = p64.temperature(tl.TL_FINE)
    b, _ = p32.temperature(tl.TL_FINE)
    assert rel(b, a) <= REFINED_TOL
    assert np.array_equal(p64.state(tl.TL_FINE), p32.state(tl.TL_FINE))
    p64.close()
    p32.close()


@pytest.mark.parametrize("inner_tiles", [1, 2])
def test_refined_energy_identity(inner_tiles):
    cfg = workloads.workload("single_track_tiny", precision=tl.TL_FP32_REFINED, tol=1e-10, tol_inner=1e-5,
                             inner_tiles=inner_tiles)
    prob = tl.Problem(cfg)
    prob.macro_steps(10)
    st = prob.stats()
    for lvl in ("fine", "coarse"):
        s, l, f = (st[f"energy_{lvl}_{k}"] for k in ("stored", "laser", "flux"))
        assert abs(s - l - f) <= 1e-7 * max(abs(s), abs(l)), lvl
    prob.close()


def test_refined_wide_tiles_ragged_against_oracle():
    """Wide inner tiles (64 x 4 elements) on a 72 x 18 x 12 fine patch: a
    ragged second tile in x (8 elements), a ragged last row of tiles in y (2),
    several tiles in z."""
    cfg = workloads.workload("single_track_tiny", precision=tl.TL_FP32_REFINED, tol=1e-10, tol_inner=1e-5,
                             inner_tiles=2, pNXc=12, pNYc=3, pNZc=2, r=6, m=2, macro_steps=3)
    prob = tl.Problem(cfg)
    ref = TL.TwoLevel(cfg, energy=False)
    prob.macro_steps(3)
    ref.run(3)
    Tf, org = prob.temperature(tl.TL_FINE)
    Tc, _ = prob.temperature(tl.TL_COARSE)
    assert tuple(org) == tuple(ref.origin)
    assert rel(Tf, ref.Tf) <= REFINED_TOL and rel(Tc, ref.Tc) <= REFINED_TOL
    assert np.array_equal(prob.state(tl.TL_FINE), ref.fine_state().reshape(-1))
    prob.close()


def test_refined_wide_equals_element_tiles_multitrack():
    """Both inner tilings converge to the same solution (outer tolerance 1e-10)."""
    base = workloads.workload("multitrack_10mm", precision=tl.TL_FP32_REFINED, tol=1e-10, tol_inner=1e-5)
    out = []
    for tiles in (1, 2):
        p = tl.Problem(dict(base, inner_tiles=tiles))
        p.macro_steps(4)
        out.append((p.temperature(tl.TL_FINE)[0], p.state(tl.TL_FINE)))
        p.close()
    assert rel(out[1][0], out[0][0]) <= 1e-8
    assert np.array_equal(out[0][1], out[1][1])


def test_refined_20mm_full_size_against_fp64_gpu_path():
    """The 20 x 10 x 4 mm plate at full size (129 x 129 x 65 fine nodes, wide
    inner tiles): the precision form against the FP64 path after 3 macro steps
    (the oracle would need tens of minutes per step at this size), plus the
    energy identity of the refined solves."""
    base = workloads.workload("multitrack_20mm")
    out = []
    for prec, tol in ((tl.TL_FP64, 1e-12), (tl.TL_FP32_REFINED, 1e-10)):
        p = tl.Problem(dict(base, precision=prec, tol=tol))
        p.macro_steps(3)  # raises on a failed solve
        assert p.sync() == tl.TL_OK
        out.append((p.temperature(tl.TL_FINE)[0], p.temperature(tl.TL_COARSE)[0], p.state(tl.TL_FINE), p.stats()))
        p.close()
    (a, ac, sa, _), (b, bc, sb, st) = out
    assert rel(b, a) <= REFINED_TOL and rel(bc, ac) <= REFINED_TOL
    assert np.array_equal(sa == tl.MELTED, sb == tl.MELTED)
    for lvl in ("fine", "coarse"):
        s_, l_, f_ = (st[f"energy_{lvl}_{k}"] for k in ("stored", "laser", "flux"))
        assert abs(s_ - l_ - f_) <= 1e-7 * max(abs(s_), abs(l_)), lvl


# ---- iterated two-level coupling at the correction step ---------------------

@pytest.mark.parametrize("precision", [tl.TL_FP64, tl.TL_FP32_REFINED])
def test_coupled_correction_against_oracle(precision):
    cfg = workloads.workload("single_track_tiny", coupling_sweeps=6, coupling_tol=1e-10, precision=precision,
                             tol=1e-12 if precision == tl.TL_FP64 else 1e-10)
    bar = TOL if precision == tl.TL_FP64 else REFINED_TOL
    prob = tl.Problem(cfg)
    ref = TL.TwoLevel(cfg)
    for _ in range(4):
        prob.macro_steps(5)
        ref.run(5)
        Tf, org = prob.temperature(tl.TL_FINE)
        Tc, _ = prob.temperature(tl.TL_COARSE)
        assert tuple(org) == tuple(ref.origin)
        assert rel(Tf, ref.Tf) <= bar and rel(Tc, ref.Tc) <= bar
        assert np.array_equal(prob.state(tl.TL_FINE), ref.fine_state().reshape(-1))
        assert np.array_equal(prob.state(tl.TL_COARSE), ref.state_c)
    st = prob.stats()
    assert st["coupling_resolves"] >= 20  # at least one re-solve per macro step
    for lvl in ("fine", "coarse"):
        for k in ("stored", "laser", "flux"):
            o = ref.energy[f"{lvl}_{k}"]
            assert abs(st[f"energy_{lvl}_{k}"] - o) <= 1e-7 * max(abs(o), abs(ref.energy[f"{lvl}_laser"]))
    prob.close()


def test_coupled_correction_multitrack_first_macro_step():
    cfg = workloads.workload("multitrack_10mm", coupling_sweeps=2, coupling_tol=1e-10)
    prob = tl.Problem(cfg)
    ref = TL.TwoLevel(cfg, energy=False)
    prob.macro_steps(1)
    ref.run(1)
    compare(prob, ref, "coupled macro 1")
    assert prob.stats()["coupling_resolves"] >= 1
    prob.close()


@pytest.mark.parametrize("over", [dict(coupling_sweeps=3), dict(picard_iters=3, latent=2.86e5),
                                  dict(interface_coupling=1)])
def test_coupled_and_picard_problems_stay_out_of_batches(over):
    cfg = workloads.workload("single_track_tiny", **over)
    p = tl.Problem(cfg)
    b = tl.Batch(launches_per_round=2, max_jobs=2)
    with pytest.raises(tl.TLError):
        b.add(p, 2)
    b.close()
    p.close()


# ---- preconditioners: Jacobi and the tensor-product mass preconditioner -----

def test_jacobi_preconditioner_against_oracle():
    cfg = workloads.workload("single_track_tiny", precond=1)
    prob, ref, errs = run_both(cfg, 20, check_every=5)
    prob.close()


@pytest.mark.parametrize("precond", [1, 2])
@pytest.mark.parametrize("inner_tiles", [1, 2])
def test_refined_preconditioners_against_oracle(inner_tiles, precond):
    cfg = workloads.workload("single_track_tiny", precision=tl.TL_FP32_REFINED, tol=1e-10, tol_inner=1e-5,
                             precond=precond, inner_tiles=inner_tiles)
    prob = tl.Problem(cfg)
    ref = TL.TwoLevel(cfg, energy=False)
    prob.macro_steps(20)
    ref.run(20)
    Tf, _ = prob.temperature(tl.TL_FINE)
    Tc, _ = prob.temperature(tl.TL_COARSE)
    assert rel(Tf, ref.Tf) <= REFINED_TOL and rel(Tc, ref.Tc) <= REFINED_TOL
    assert np.array_equal(prob.state(tl.TL_FINE), ref.fine_state().reshape(-1))
    prob.close()


def test_preconditioners_agree_and_tensor_needs_fewer_iterations():
    base = workloads.workload("multitrack_10mm")
    out = []
    for pc in (1, 0):  # 0: the default, the tensor-product preconditioner
        p = tl.Problem(dict(base, precond=pc))
        p.macro_steps(2)
        out.append((p.temperature(tl.TL_FINE)[0], p.state(tl.TL_FINE), p.stats()))
        p.close()
    (a, sa, st1), (b, sb, st2) = out
    assert rel(b, a) <= 1e-10 and np.array_equal(sa, sb)
    assert st2["cg_iters_fine"] * 2 < st1["cg_iters_fine"]


# ---- latent heat and Picard iterations of the nonlinear step ------------------

@pytest.mark.parametrize("picard", [1, 4])
def test_latent_heat_picard_against_oracle(picard):
    cfg = workloads.workload("single_track_tiny", latent=2.86e5, picard_iters=picard)
    prob, ref, errs = run_both(cfg, 16, check_every=4)
    st = prob.stats()
    assert st["solves_fine"] == 16 * cfg["m"] * picard and st["solves_coarse"] == 16 * 2 * picard
    for lvl in ("fine", "coarse"):  # the energy account of the last solve of every step
        for k in ("stored", "laser", "flux"):
            o = ref.energy[f"{lvl}_{k}"]
            assert abs(st[f"energy_{lvl}_{k}"] - o) <= 1e-8 * max(abs(o), abs(ref.energy[f"{lvl}_laser"])), (lvl, k)
    prob.close()


def test_latent_heat_picard_refined_against_oracle():
    cfg = workloads.workload("single_track_tiny", latent=2.86e5, picard_iters=4, precision=tl.TL_FP32_REFINED,
                             tol=1e-10, tol_inner=1e-5)
    prob = tl.Problem(cfg)
    ref = TL.TwoLevel(cfg, energy=False)
    prob.macro_steps(12)
    ref.run(12)
    Tf, _ = prob.temperature(tl.TL_FINE)
    Tc, _ = prob.temperature(tl.TL_COARSE)
    assert rel(Tf, ref.Tf) <= REFINED_TOL and rel(Tc, ref.Tc) <= REFINED_TOL
    assert np.array_equal(prob.state(tl.TL_FINE), ref.fine_state().reshape(-1))
    prob.close()


def test_zero_latent_and_one_picard_iteration_is_the_plain_step():
    base = tl.Problem(workloads.workload("single_track_tiny"))
    same = tl.Problem(workloads.workload("single_track_tiny", latent=0.0, picard_iters=0))
    base.macro_steps(4)
    same.macro_steps(4)
    assert np.array_equal(base.temperature(tl.TL_FINE)[0], same.temperature(tl.TL_FINE)[0])
    assert np.array_equal(base.temperature(tl.TL_COARSE)[0], same.temperature(tl.TL_COARSE)[0])
    base.close()
    same.close()


# ---- top-surface convection and radiation (Section 3.1) ---------------------
# Coefficients far above the physical ones (h ~ 10 W/(m^2 K)) so that the term
# moves the solution well beyond the parity tolerance.

SURFACE_CASES = [
    dict(h_conv=2e5),
    dict(h_conv=1e4, emissivity=0.8),
    dict(h_conv=1e5, T_amb=600.0),                       # heat enters through the top
    dict(h_conv=1e4, emissivity=0.8, picard_iters=3),    # h_rad at the Picard iterate
]


def _energy_identity_with_loss(st, ref, tol):
    for lvl in ("fine", "coarse"):
        s_, l_, f_, x_ = (st[f"energy_{lvl}_{k}"] for k in ("stored", "laser", "flux", "loss"))
        scale = max(abs(s_), abs(l_), abs(x_))
        assert abs(s_ - l_ - f_ + x_) <= tol * scale, (lvl, s_, l_, f_, x_)
        o = ref.energy[f"{lvl}_loss"]
        assert o != 0.0 and abs(x_ - o) <= 10 * tol * scale, (lvl, x_, o)


@pytest.mark.parametrize("over", SURFACE_CASES)
def test_top_surface_losses_against_oracle(over):
    cfg = workloads.workload("single_track_tiny", **over)
    prob, ref, _ = run_both(cfg, 16, check_every=4)
    plain = tl.Problem(workloads.workload("single_track_tiny"))
    plain.macro_steps(16)
    assert rel(prob.temperature(tl.TL_FINE)[0], plain.temperature(tl.TL_FINE)[0]) > 1e-6  # the term matters
    plain.close()
    _energy_identity_with_loss(prob.stats(), ref, 1e-9)
    prob.close()


@pytest.mark.parametrize("inner_tiles", [1, 2])
def test_top_surface_losses_refined_against_oracle(inner_tiles):
    """The precision form with both inner tilings on the ragged 72 x 18 x 12
    patch (wide tiles: a ragged x tile and y row), radiation included."""
    cfg = workloads.workload("single_track_tiny", precision=tl.TL_FP32_REFINED, tol=1e-10, tol_inner=1e-5,
                             inner_tiles=inner_tiles, pNXc=12, pNYc=3, pNZc=2, r=6, m=2, h_conv=1e4,
                             emissivity=0.8)
    prob = tl.Problem(cfg)
    ref = TL.TwoLevel(cfg)
    for _ in range(3):
        prob.macro_steps(2)
        ref.run(2)
        Tf, org = prob.temperature(tl.TL_FINE)
        Tc, _ = prob.temperature(tl.TL_COARSE)
        assert tuple(org) == tuple(ref.origin)
        assert rel(Tf, ref.Tf) <= REFINED_TOL and rel(Tc, ref.Tc) <= REFINED_TOL
        assert np.array_equal(prob.state(tl.TL_FINE), ref.fine_state().reshape(-1))
    _energy_identity_with_loss(prob.stats(), ref, 1e-7)
    prob.close()


def test_top_surface_losses_in_a_batch_equal_alone():
    base = workloads.workload("single_track_tiny", h_conv=1e4, emissivity=0.8)
    jobs = [dict(base, macro_steps=6), dict(base, macro_steps=4, P=150.0, precision=tl.TL_FP32_REFINED,
                                             tol=1e-10, tol_inner=1e-5)]
    alone = []
    for cfg in jobs:
        p = tl.Problem(cfg)
        p.macro_steps(cfg["macro_steps"])
        alone.append(p.temperature(tl.TL_FINE)[0])
        p.close()
    probs = [tl.Problem(c) for c in jobs]
    b = tl.Batch(launches_per_round=3, max_jobs=4)
    for p, c in zip(probs, jobs):
        b.add(p, c["macro_steps"])
    b.run()
    b.close()
    for p, c, a in zip(probs, jobs, alone):
        assert p.sync() == tl.TL_OK
        tol = 1e-6 if c.get("precision", 0) == tl.TL_FP32_REFINED else 1e-9
        assert rel(p.temperature(tl.TL_FINE)[0], a) <= tol
        p.close()


def test_autotuned_tilings_keep_the_results():
    """The autotuner only changes how blocks walk the mesh: an autotuned
    problem matches the cost-model one (the FP32 summation order may differ:
    precision form within 1e-8 of each other, FP64 within 1e-10), reports its
    picks as tuned, and a second problem of the same shape reuses them."""
    for prec, tol in ((tl.TL_FP32_REFINED, 1e-8), (tl.TL_FP64, 1e-10)):
        base = workloads.workload("multitrack_10mm", precision=prec, tol=1e-10 if prec else 1e-12)
        out, picks = [], []
        for at in (0, 1, 1):
            p = tl.Problem(dict(base, autotune=at))
            picks.append(p.tiling(tl.TL_FINE))
            p.macro_steps(3)
            out.append((p.temperature(tl.TL_FINE)[0], p.state(tl.TL_FINE)))
            p.close()
        assert not picks[0]["tuned"] and picks[1]["tuned"] and picks[1] == picks[2]
        assert rel(out[1][0], out[0][0]) <= tol and np.array_equal(out[1][1], out[0][1])
        assert np.array_equal(out[1][0], out[2][0])


# ---- flux-jump coupling (Section 3, Eq. globalPbmAlternate) -------------------

@pytest.mark.parametrize("over", [dict(), dict(h_conv=1e4, emissivity=0.8), dict(coarse_source=1, r=2, m=3)])
def test_flux_jump_coupling_against_oracle(over):
    """The correction solves the global problem with the interface load
    (kappa_+ - kappa_-) dT-/dn on the immersed patch faces instead of the
    injected values: fields and states against the oracle every 4 macro
    steps (the patch starts at the plate's edge, where its x- face is not
    immersed), and the coarse energy account with the interface heat in the
    flux term."""
    cfg = workloads.workload("single_track_tiny", interface_coupling=1, **over)
    prob, ref, _ = run_both(cfg, 16, check_every=4)
    st = prob.stats()
    s_, l_, f_, x_ = (st[f"energy_coarse_{k}"] for k in ("stored", "laser", "flux", "loss"))
    assert abs(s_ - l_ - f_ + x_) <= 1e-9 * max(abs(s_), abs(l_))
    assert abs(f_ - ref.energy["coarse_flux"]) <= 1e-8 * max(abs(f_), abs(l_))
    iface = sum(e.get("interface", 0.0) for lvl, e in ref.step_energy if lvl == "coarse")
    assert abs(iface) > 1e-3 * abs(l_)  # the interface term matters
    prob.close()


def test_flux_jump_refined_against_oracle():
    cfg = workloads.workload("single_track_tiny", interface_coupling=1, precision=tl.TL_FP32_REFINED, tol=1e-10,
                             tol_inner=1e-5)
    prob = tl.Problem(cfg)
    ref = TL.TwoLevel(cfg, energy=False)
    for _ in range(3):
        prob.macro_steps(5)
        ref.run(5)
        assert rel(prob.temperature(tl.TL_FINE)[0], ref.Tf) <= REFINED_TOL
        assert rel(prob.temperature(tl.TL_COARSE)[0], ref.Tc) <= REFINED_TOL
        assert np.array_equal(prob.state(tl.TL_FINE), ref.fine_state().reshape(-1))
    prob.close()


def test_flux_jump_with_agreeing_conductivities_is_the_single_level_coarse_solve():
    """One conductivity law and no powder: the interface load vanishes and the
    coarse field is the single-level coarse solve (Gaussian source)."""
    cfg = workloads.workload("single_track_tiny", interface_coupling=1, coarse_source=1, k1=0.0, powder_depth=0.0)
    prob = tl.Problem(cfg)
    sl = TL.SingleLevel(cfg, cfg["NXc"], cfg["NYc"], cfg["NZc"], cfg["dt_coarse"])
    for n in range(10):
        prob.macro_steps(1)
        sl.step()
        assert rel(prob.temperature(tl.TL_COARSE)[0], sl.T) <= 1e-9, n
    prob.close()


@pytest.mark.parametrize("dims", [(11, 3, 3, 5), (7, 5, 2, 4)])
def test_refined_wide_tiles_ragged_everywhere_against_oracle(dims):
    """Wide inner tiles with the preconditioner fused into the apply on
    patches ragged in x (55 or 28 elements of a 64-wide tile), in y (15 or 20
    rows in 4-row tiles) and in z (15 or 8 layers in tiles of about nz / 8),
    the patch touching the plate's sides in some macro steps."""
    pnx, pny, pnz, r = dims
    cfg = workloads.workload("single_track_tiny", precision=tl.TL_FP32_REFINED, tol=1e-10, tol_inner=1e-5,
                             inner_tiles=2, pNXc=pnx, pNYc=pny, pNZc=pnz, r=r, m=2)
    prob = tl.Problem(cfg)
    ref = TL.TwoLevel(cfg, energy=False)
    for _ in range(3):
        prob.macro_steps(2)
        ref.run(2)
        Tf, org = prob.temperature(tl.TL_FINE)
        assert tuple(org) == tuple(ref.origin)
        assert rel(Tf, ref.Tf) <= REFINED_TOL
        assert rel(prob.temperature(tl.TL_COARSE)[0], ref.Tc) <= REFINED_TOL
        assert np.array_equal(prob.state(tl.TL_FINE), ref.fine_state().reshape(-1))
    assert prob.tiling(tl.TL_FINE)["wide"][0] == 64
    prob.close()
