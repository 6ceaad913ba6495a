"""Verlet scheme (Eq 30-31) on the GPU path against the FP64 oracle.

Same tolerances as the Symplectic tests: free fall to FP32 offset rounding,
100 steps of the dam break with the front within 0.5 dp and the kinetic
energy within 1 %, moving boundaries by their law, bit-exact checkpoint
resume and batch-versus-alone.
"""
import numpy as np
import pytest

import oracle
from paper_2104_00537_gb300 import cases, sph

pytestmark = pytest.mark.gpu


def verlet(case_fn, *a, ns=40, **kw):
    return case_fn(*a, integrator=1, verlet_steps=ns, **kw)


@pytest.mark.parametrize("ns", [1, 3, 40])
def test_verlet_free_fall_gpu(ns):
    """Constant acceleration is integrated exactly by Eq 30 and Eq 31."""
    c = verlet(cases.free_particle, ns=ns)
    eng = sph.Engine.create(c)
    eng.step(40)
    st = eng.get_state()
    t = st["t"]
    g = np.array(c.params["gravity"])
    assert np.abs(st["pos"][0] - (c.pos[0] + c.vel[0] * t + 0.5 * g * t * t)).max() < 1e-7
    assert np.abs(st["vel"][0] - (c.vel[0] + g * t)).max() < 1e-5
    assert st["step"] == 40
    eng.destroy()


@pytest.mark.parametrize("variant", [5, 0])
@pytest.mark.parametrize("use_graph", [0, 1])
def test_verlet_dam_break_100_steps(use_graph, variant):
    c = verlet(cases.dam_break, 0.02, ns=40)
    eng = sph.Engine.create(c)
    eng.set_options(use_graph=use_graph, pi_variant=variant)
    m0 = eng.stats()["mass"]
    eng.step(100)
    s = eng.stats()
    st = eng.get_state()
    o = oracle.OracleState(c)
    o.step(100)
    od = o.diag()
    dp = c.params["dp"]
    assert s["step"] == 100
    assert abs(s["t"] - o.t.value) < 1e-3 * o.t.value
    assert abs(s["front"] - od["front"]) < 0.5 * dp
    assert abs(s["ke"] - od["ke"]) < 0.01 * od["ke"]
    assert s["mass"] == m0 == od["mass"]
    assert np.abs(st["pos"] - o.pos).max() < 0.5 * dp
    assert np.abs(st["rho"] - o.rho).max() < 1.0
    assert s["n_out"] == 0 and s["flags"] == 0
    # one interaction evaluation per step
    assert s["interactions"] == pytest.approx(100 * eng.eval_forces()["pairs"], rel=0.05)
    eng.destroy()


def test_verlet_eq31_schedule_matches_oracle():
    """A short N_S (every 4th step is Eq 31) and a moving tank: positions and
    densities follow the oracle step by step."""
    c = verlet(cases.sloshing_tank, 3000, 0.3, 0.03, 1.2, ns=4)
    eng = sph.Engine.create(c)
    o = oracle.OracleState(c)
    for _ in range(3):
        eng.step(7)
        o.step(7)
        st = eng.get_state()
        assert abs(st["t"] - o.t.value) < 1e-4 * st["t"]
        assert np.abs(st["pos"] - o.pos).max() < 0.01 * c.params["dp"]
        assert np.abs(st["rho"] - o.rho).max() < 0.05
    b = c.ptype == 1
    m = c.motions[0]
    np.testing.assert_allclose(st["pos"][b, 0] - c.pos[b, 0], m["amp"] * np.sin(m["omega"] * st["t"]),
                               atol=1e-6)
    eng.destroy()


def test_verlet_raw_resume_is_bit_exact():
    """The snapshot carries v^{n-1}, rho^{n-1}: resuming mid-cycle (step 10,
    N_S = 4) continues bit for bit."""
    c = verlet(cases.dam_break, 0.04, ns=4)
    a = sph.Engine.create(c)
    a.step(10)
    b = sph.Engine.from_raw(c, a.get_raw())
    a.step(9)
    b.step(9)
    sa, sb = a.get_state(), b.get_state()
    for k in ("pos", "vel", "rho"):
        assert np.array_equal(sa[k], sb[k]), k
    assert sa["t"] == sb["t"] and sa["step"] == sb["step"] == 19
    with pytest.raises(sph.SphError):  # a Symplectic engine cannot take it
        sph.Engine.from_raw(cases.dam_break(0.04), a.get_raw())
    a.destroy()
    b.destroy()


def test_verlet_batch_on_kept_list_equals_alone():
    """The Verlet scheme on the list kept across steps, in a batch: each case
    takes bit for bit the steps it takes alone (rebuilds per case)."""
    cs = [verlet(cases.dam_break, 0.04, seed=1, ns=5),
          verlet(cases.sloshing_tank, 2000, 0.25, 0.02, 1.0, seed=2, ns=7)]
    bat = sph.Engine.batch(cs)
    bat.set_options(pi_variant=5, check_list=1)
    bat.step(30)
    assert bat.list_info()["check_bad"] == 0
    for i, c in enumerate(cs):
        e = sph.Engine.create(c)
        e.step(30)
        sa, sb = e.get_state(), bat.get_state(i)
        for k in ("pos", "vel", "rho"):
            assert np.array_equal(sa[k], sb[k]), (i, k)
        e.destroy()
    bat.destroy()


def test_verlet_batch_equals_alone():
    cs = [verlet(cases.dam_break, 0.04, seed=1, ns=5),
          verlet(cases.sloshing_tank, 2000, 0.25, 0.02, 1.0, seed=2, ns=7)]
    bat = sph.Engine.batch(cs)
    bat.set_options(pi_variant=0)         # the compacted loop: bit for bit
    bat.step(12)
    for i, c in enumerate(cs):
        e = sph.Engine.create(c)
        e.set_options(pi_variant=0)
        e.step(12)
        sa, sb = e.get_state(), bat.get_state(i)
        for k in ("pos", "vel", "rho"):
            assert np.array_equal(sa[k], sb[k]), (i, k)
        e.destroy()
    bat.destroy()


def test_verlet_rejected_where_unsupported():
    with pytest.raises(sph.SphError):  # mixed schemes in one engine
        sph.Engine.batch([cases.dam_break(0.04), verlet(cases.dam_break, 0.04)])
    pool = sph.Engine.pool(100000, 1000000, 4)
    with pytest.raises(sph.SphError):  # pools run the Symplectic scheme
        pool.admit(verlet(cases.dam_break, 0.04), t_end=1.0)
    pool.destroy()


@pytest.mark.parametrize("use_graph", [0, 1])
def test_verlet_kept_list_finds_every_pair(use_graph):
    """The Verlet scheme on the list kept across steps (one PI per step):
    brute-force check of every evaluation, dam break and moving tank."""
    for c in (verlet(cases.dam_break, 0.03, seed=4),
              verlet(cases.sloshing_tank, 3000, 0.3, 0.04, 1.2, seed=5, ns=4)):
        eng = sph.Engine.create(c)
        eng.set_options(pi_variant=5, use_graph=use_graph, check_list=1)
        eng.step(150)
        li, st = eng.list_info(), eng.stats()
        assert li["check_bad"] == 0
        assert li["check_pairs"] == st["interactions"]
        assert 2 <= li["builds"] < 75, li
        eng.destroy()


def test_verlet_batch_variants_fall_back():
    """Per-step lists (3, 4) do not apply to the one-PI Verlet step: the
    engine runs the compacted loop and gives the same state as variant 0."""
    c = verlet(cases.dam_break, 0.04, seed=2)
    a, b = sph.Engine.create(c), sph.Engine.create(c)
    a.set_options(pi_variant=4)
    b.set_options(pi_variant=0)
    a.step(10)
    b.step(10)
    for k in ("pos", "vel", "rho"):
        assert np.array_equal(a.get_state()[k], b.get_state()[k]), k
    a.destroy()
    b.destroy()
