"""The interaction kernel that sph_step times -- the neighbour-list walk --
against the FP64 oracle, one evaluation at a time (Sect. 2, Eq 15-18, 21-22,
35-36; Sect. 5.1).

sph_eval_step runs the step's own launches without advancing the engine:
stage 0 is the first evaluation of the next step (state n), stage 1 the second
(the half-step state of Eq 33-34).  With the list kept across steps (the
default) both states are those kept in the order and cells of the list's
build, with cell offsets up to half the skin outside [0, cs), and both walks
go over the chunk records with the two-candidate carry-over; the library is
built with FP32 flush-to-zero.  The oracle evaluates Eq 15-18, 21-22 and 36 in
FP64 on the evaluated state (positions from the GPU's cell + offset, velocity
and density as stored), so the comparison isolates the evaluation itself.

Tolerances: dv/dt, drho/dt and mu_max within 1e-4 of max|.| (FP32 against
FP64); dt of Eq 35 within 1e-4 relative; the pair count equal up to the pairs
within 1e-6 (relative) of (2h)^2, on which FP32 and FP64 may disagree (their
kernel weight is ~1e-18).
"""
import numpy as np
import pytest

import oracle
from paper_2104_00537_gb300 import cases, sph
from tests.test_gpu_parity import n_ambiguous, rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-4


def n_band(case, pos):
    """Ordered pairs (all types) with |r^2 - (2h)^2| < 1e-6 (2h)^2: an upper
    bound of the pairs on which FP32 and FP64 may disagree, counted without
    listing pairs (for the full-size cases)."""
    from scipy.spatial import cKDTree
    R2 = 4.0 * case.params["h"] ** 2
    tree = cKDTree(pos)
    lo, hi = tree.count_neighbors(tree, np.sqrt(R2 * np.array([1 - 1e-6, 1 + 1e-6])))
    return int(hi - lo)


def check_step_eval(case, eng, stage, icase=0, exact_pairs=True):
    """One evaluation of the next step (stage 0 or 1) against the oracle on
    the evaluated state; returns the GPU results."""
    g = eng.eval_step(stage, icase)
    vel = g["vel"].astype(np.float64)
    rho = g["rho"].astype(np.float64)
    acc, drho, mu, npairs = oracle.interact(case.params, g["pos"], vel, rho, case.ptype)
    f = case.ptype == 0
    b = ~f
    amb = n_ambiguous(case, g["pos"]) if exact_pairs else n_band(case, g["pos"])
    assert abs(g["pairs"] - npairs) <= amb, (g["pairs"], npairs, amb)
    assert rel_err(g["acc"][f], acc[f]) < TOL
    assert np.all(g["acc"][b] == 0)
    if case.params.get("boundary_mode", 0) == 1:  # Eq 38 sets boundary densities
        assert rel_err(g["drho"][f], drho[f]) < TOL
        assert np.all(g["drho"][b] == 0)
    else:
        assert rel_err(g["drho"], drho) < TOL
    assert rel_err(g["mumax"][f], mu[f]) < TOL
    assert np.all(g["mumax"][b] == 0)
    if stage == 0:
        dt = oracle.time_step(case.params, acc, mu, case.ptype)
        assert abs(g["dt"] - dt) < TOL * dt
    return g


def mid_list_eval(case, eng, stage):
    """check_step_eval on a state kept since an earlier list build: asserts
    that the evaluation did not rebuild the list (so the state is in the
    build's cells), returning False where it had to (a pending rebuild)."""
    b0 = eng.list_info()["builds"]
    check_step_eval(case, eng, stage)
    return eng.list_info()["builds"] == b0


@pytest.mark.parametrize("variant", [3, 4, 5])
@pytest.mark.parametrize("cell_mode", [0, 1, 2])
def test_list_evaluation_at_rest(cell_mode, variant):
    """t = 0: both evaluations of the first step (the list built on state n)."""
    case = cases.dam_break(0.02, cell_mode=cell_mode)
    eng = sph.Engine.create(case)
    eng.set_options(pi_variant=variant)
    for stage in (0, 1):
        check_step_eval(case, eng, stage)
    eng.destroy()


@pytest.mark.parametrize("variant", [3, 4, 5])
def test_list_evaluation_in_motion(variant):
    """After 60 steps the column moves: the viscosity and diffusion terms and
    mu_max are active, and the kept list has been walked for several steps."""
    case = cases.dam_break(0.02)
    eng = sph.Engine.create(case)
    eng.set_options(pi_variant=variant, use_graph=1)
    eng.step(60)
    for stage in (0, 1):
        g = check_step_eval(case, eng, stage)
        assert np.abs(g["mumax"]).max() > 0
    if variant == 5:
        assert eng.list_info()["builds"] < 60
    eng.destroy()


@pytest.mark.parametrize("lanes", [1, 2, 4, 8])
def test_list_evaluation_lanes_per_target(lanes):
    """pi_lanes threads per target: thread k takes the candidates at bit
    positions k, k + lanes, ... of each record (a record may hold none of a
    thread's) and the partial sums are added at the end.  On the same state
    the pair set is that of one thread per target (first evaluation from
    rest); both evaluations after 60 steps against the oracle; the run stays
    within rounding of the run with one thread per target (its sums are added
    in another order)."""
    case = cases.dam_break(0.02)
    eng = sph.Engine.create(case)
    one = sph.Engine.create(case)
    eng.set_options(pi_variant=5, use_graph=1, pi_lanes=lanes)
    one.set_options(pi_variant=5, use_graph=1, pi_lanes=1)
    ga, gb = eng.eval_step(0), one.eval_step(0)
    assert ga["pairs"] == gb["pairs"]
    assert rel_err(ga["acc"], gb["acc"]) < 1e-5
    eng.step(60)
    one.step(60)
    for stage in (0, 1):
        check_step_eval(case, eng, stage)
    sa, sb = eng.get_state(), one.get_state()
    assert np.abs(sa["pos"] - sb["pos"]).max() < 1e-3 * case.params["dp"]
    pa, pb = eng.stats()["interactions"], one.stats()["interactions"]
    assert abs(pa - pb) <= 1e-6 * pb, (pa, pb)
    eng.destroy()
    one.destroy()


@pytest.mark.parametrize("variant", [4, 5])
def test_pair_once_evaluation(variant):
    """pair_once: each pair evaluated once by the target of lower index over
    a half list, the partner's share added atomically.  Both evaluations at
    rest and after 60 steps against the oracle (dv/dt, drho/dt, mu_max per
    particle, dt, the directed pair count), and the half lists checked by
    brute force at every evaluation of the 60 steps."""
    case = cases.dam_break(0.02)
    eng = sph.Engine.create(case)
    eng.set_options(pi_variant=variant, use_graph=1, pair_once=1)
    for stage in (0, 1):
        check_step_eval(case, eng, stage)
    # the half lists (candidates of larger index only) hold every such pair
    eng.set_options(pi_variant=variant, use_graph=1, pair_once=1, check_list=1)
    eng.step(60)
    li = eng.list_info()
    assert li["check_bad"] == 0 and li["check_pairs"] > 0
    for stage in (0, 1):
        g = check_step_eval(case, eng, stage)
        assert np.abs(g["mumax"]).max() > 0
    eng.destroy()


def test_pair_once_through_the_splash_and_in_a_batch():
    """pair_once over the collapse (600 steps, kept list with rebuilds) and
    in a batch of three uneven cases (each case's evaluations against the
    oracle; a case's partner shares never cross into another case)."""
    case = cases.dam_break(0.02)
    eng = sph.Engine.create(case)
    eng.set_options(pi_variant=5, use_graph=1, pair_once=1)
    eng.step(600)
    for stage in (0, 1):
        check_step_eval(case, eng, stage)
    eng.destroy()
    cs = [cases.dam_break(0.04, seed=1), cases.sloshing_tank(2000, 0.25, 0.02, 1.0, seed=2),
          cases.dam_break(0.03, seed=3, column=(0.3, 0.2, 0.3))]
    bat = sph.Engine.batch(cs)
    bat.set_options(use_graph=1, pair_once=1, check_list=1)
    bat.step(40)
    assert bat.list_info()["check_bad"] == 0
    for i, c in enumerate(cs):
        for stage in (0, 1):
            check_step_eval(c, bat, stage, icase=i)
    bat.destroy()


@pytest.mark.parametrize("variant,pair_once", [(5, 0), (4, 0), (5, 1)])
def test_wide_records_equal_narrow(variant, pair_once):
    """Wide list records (a 32-bit first index, the row taken from the first
    candidate's cell: what an engine beyond 2^25 particles uses), asked for on
    a small case: both evaluations against the oracle at rest and after 60
    steps, every pair listed, and (with each target's own sums) the same steps
    bit for bit as the narrow records."""
    case = cases.dam_break(0.02)
    wide = sph.Engine.create(case)
    wide.set_options(pi_variant=variant, use_graph=1, wide_records=1, pair_once=pair_once)
    for stage in (0, 1):
        check_step_eval(case, wide, stage)
    wide.set_options(pi_variant=variant, use_graph=1, wide_records=1, pair_once=pair_once,
                     check_list=1)
    wide.step(60)
    li = wide.list_info()
    assert li["check_bad"] == 0 and li["builds"] > 0
    for stage in (0, 1):
        check_step_eval(case, wide, stage)
    if not pair_once:
        narrow = sph.Engine.create(case)
        narrow.set_options(pi_variant=variant, use_graph=1, check_list=1)
        narrow.step(60)
        a, b = wide.get_state(), narrow.get_state()
        for k in ("pos", "vel", "rho"):
            assert np.array_equal(a[k], b[k]), k
        narrow.destroy()
    wide.destroy()


def test_wide_records_beyond_two_to_the_25():
    """An engine beyond 2^25 particles (the wave flume at dp = 0.0077 m,
    35.6M particles) walks wide records instead of falling back to the cell
    walk: its list is built and both evaluations of a step match the oracle."""
    case = cases.wave_flume(0.0077)
    assert case.n >= 1 << 25
    eng = sph.Engine.create(case)
    eng.set_options(use_graph=1)
    eng.step(3)
    assert eng.list_info()["builds"] >= 1
    f = case.ptype == 0
    for stage in (0, 1):
        g = eng.eval_step(stage)
        acc, drho, mu, npairs = oracle.interact(case.params, g["pos"],
                                                g["vel"].astype(np.float64),
                                                g["rho"].astype(np.float64), case.ptype)
        # pairs within FP32 rounding of the cut-off may differ (weight ~1e-18):
        # at most the evaluated pairs with |r^2 - (2h)^2| < 1e-6 (2h)^2, counted
        # by the oracle with the cut-off moved to either edge of that band
        band = 0
        for sgn in (1, -1):
            p = dict(case.params, h=case.params["h"] * np.sqrt(1 + sgn * 1e-6))
            band += sgn * oracle.interact(p, g["pos"], g["vel"].astype(np.float64),
                                          g["rho"].astype(np.float64), case.ptype)[3]
        assert abs(g["pairs"] - npairs) <= band, (g["pairs"], npairs, band)
        assert rel_err(g["acc"][f], acc[f]) < TOL
        assert rel_err(g["drho"], drho) < TOL
        assert rel_err(g["mumax"][f], mu[f]) < TOL
    eng.destroy()


def test_kept_list_evaluation_through_the_splash():
    """The dam break through its collapse and splash (~1,050 steps, t ~ 0.3 s),
    with the list kept across steps and rebuilt as the flow needs: both
    evaluations at seven points of the run.  Where a point falls on a step
    that starts with a rebuild, the run goes on a step at a time until an
    evaluation is in the middle of a kept list (state in the build's cells),
    so that all seven points test that state."""
    case = cases.dam_break(0.02)
    eng = sph.Engine.create(case)
    eng.set_options(pi_variant=5, use_graph=1)
    done = 0
    for chunk in (150,) * 7:
        eng.step(chunk)
        done += chunk
        for _ in range(8):
            kept = mid_list_eval(case, eng, 0)
            check_step_eval(case, eng, 1)
            if kept:
                break
            eng.step(1)
            done += 1
        assert kept, done
    builds = eng.list_info()["builds"]
    assert 5 < builds < done // 2, builds
    assert eng.stats()["t"] > 0.25
    eng.destroy()


def test_evaluation_does_not_perturb_the_run():
    """sph_eval_step leaves the engine as it found it: a run with evaluations
    of both stages in its middle (one of them at a pending rebuild) takes the
    same steps, bit for bit, as a run without."""
    case = cases.dam_break(0.02)
    a = sph.Engine.create(case)
    b = sph.Engine.create(case)
    for e in (a, b):
        e.set_options(pi_variant=5, use_graph=1)
    a.step(250)
    a.eval_step(0)
    a.eval_step(1)
    a.step(1)
    a.eval_step(1)
    a.step(49)
    b.step(300)
    sa, sb = a.get_state(), b.get_state()
    for k in ("pos", "vel", "rho"):
        assert np.array_equal(sa[k], sb[k]), k
    assert sa["t"] == sb["t"] and sa["step"] == sb["step"] == 300
    assert a.list_info()["builds"] == b.list_info()["builds"]
    a.destroy()
    b.destroy()


@pytest.mark.parametrize("lanes,pair_once", [(0, 0), (4, 0), (0, 1)])
@pytest.mark.parametrize("physics", ["fourtakas", "sps", "mdbc"])
def test_list_evaluation_extended_physics(physics, lanes, pair_once):
    """The list kernels of the Eq 19-20 diffusion (EXT 1), of laminar + SPS
    viscosity (EXT 2, with its strain pass over the list) and the list walk of
    an mDBC case (boundary values of Eq 38-39 in the build's cells), with the
    default threads per target, with four, and with pair_once asked for (which
    these physics ignore: their lists stay whole)."""
    kw = dict(fourtakas=dict(ddt_mode=2), sps=dict(visc_mode=1, nu0=1e-3),
              mdbc=dict(boundary_mode=1))[physics]
    case = cases.dam_break(0.02, **kw)
    eng = sph.Engine.create(case)
    eng.set_options(pi_variant=5, use_graph=1, pi_lanes=lanes, pair_once=pair_once)
    eng.step(60)
    for stage in (0, 1):
        check_step_eval(case, eng, stage)
    eng.destroy()


@pytest.mark.parametrize("pair_once", [0, 1])
def test_verlet_list_evaluation(pair_once):
    """The Verlet scheme's one evaluation per step (Eq 30-31) over the kept
    list, with each target's own pairs and with each pair once."""
    case = cases.dam_break(0.02, integrator=1)
    eng = sph.Engine.create(case)
    eng.set_options(pi_variant=5, use_graph=1, pair_once=pair_once)
    eng.step(60)
    check_step_eval(case, eng, 0)
    with pytest.raises(sph.SphError):
        eng.eval_step(1)
    eng.destroy()


def test_list_evaluation_wave_flume_fiftieth_scale():
    """The piston-wavemaker flume on its 1/50-particle-count copy (768k
    particles): the piston's imposed velocity (Eq 37) enters the viscosity of
    its fluid neighbours; both evaluations after 20 steps."""
    case = cases.wave_flume(0.008 * 50 ** (1 / 3))
    eng = sph.Engine.create(case)
    eng.set_options(pi_variant=5, use_graph=1)
    eng.step(20)
    for stage in (0, 1):
        g = check_step_eval(case, eng, stage, exact_pairs=False)
    piston = case.group >= 0
    assert np.abs(g["vel"][piston, 0]).max() > 0
    eng.destroy()


@pytest.mark.parametrize("pair_once", [0, 1])
def test_full_size_dam_break_order_and_evaluation(pair_once):
    """The 1.48M-particle dam break (dp = 0.004 m) in the bench's launch
    configuration (kept list, CUDA-graph replay; each target's own sums, and
    each pair once as the bench times it): the cell order after the 3-pass
    radix sort of 23-bit keys bit-exact at t = 0, then both evaluations of
    step 21 against the oracle."""
    case = cases.dam_break(0.004, cell_mode=1)
    eng = sph.Engine.create(case)
    ids, cells, ninside = eng.order()
    order, inside = oracle.sort_order(case.params, case.pos, case.ptype)
    assert ninside == inside == case.n
    assert np.array_equal(ids, order)
    assert np.array_equal(cells, oracle.cells(case.params, case.pos)[order])
    eng.set_options(pi_variant=5, use_graph=1, pair_once=pair_once)
    eng.step(20)
    for stage in (0, 1):
        check_step_eval(case, eng, stage, exact_pairs=False)
    eng.destroy()


def test_eval_step_rejects_what_it_cannot_evaluate():
    case = cases.dam_break(0.02)
    eng = sph.Engine.create(case)
    with pytest.raises(sph.SphError):
        eng.eval_step(2)
    eng.set_options(pi_variant=0)
    check_step_eval(case, eng, 0)  # the cell walk's first evaluation
    with pytest.raises(sph.SphError) as ex:
        eng.eval_step(1)
    assert ex.value.code == -1
    eng.destroy()
