"""Laminar viscosity + SPS stress (Eq 23-27, visc_mode 1) and the Fourtakas
density diffusion (Eq 19-20) on the GPU path against the FP64 oracle.

Tolerances as for the default model: one interaction evaluation within 1e-4
of max|.| per result (FP32 against FP64), 100 steps of the dam break with
the front within 0.5 dp and the kinetic energy within 1 %.
"""
import numpy as np
import pytest

import oracle
from paper_2104_00537_gb300 import cases, sph
from tests.test_gpu_parity import check_eval

pytestmark = pytest.mark.gpu


def sps_case(dp=0.02, **kw):
    # nu0 of water is 1e-6 m^2/s; 1e-3 makes the laminar term visible in the
    # comparison without changing the flow's character over 100 steps
    return cases.dam_break(dp, visc_mode=1, nu0=kw.pop("nu0", 1e-3), **kw)


def test_sps_strain_pass_matches_oracle():
    """tau/rho of Eq 25 after 60 steps of motion, particle by particle, on
    the GPU's own state: within 1e-4 of max|tau| per component (FP32 vs FP64;
    tau is quadratic in the velocity gradient)."""
    c = sps_case()
    eng = sph.Engine.create(c)
    eng.step(60)
    st = eng.get_state()
    tau = eng.eval_sps()
    ref = oracle.sps_tau(c.params, st["pos"], st["vel"].astype(np.float64),
                         st["rho"].astype(np.float64), c.ptype)
    assert np.abs(ref).max() > 0
    for k in range(6):
        scale = np.abs(ref[:, k]).max()
        assert np.abs(tau[:, k] - ref[:, k]).max() < 1e-4 * scale + 1e-12, k
    assert np.all(tau[c.ptype == 1] == 0)
    eng.destroy()


@pytest.mark.parametrize("steps", [0, 60])
def test_sps_one_evaluation(steps):
    c = sps_case()
    eng = sph.Engine.create(c)
    eng.step(steps)
    g, (acc, drho, mu) = check_eval(c, eng)
    eng.destroy()


@pytest.mark.parametrize("variant", [5, 4, 3, 0])
def test_sps_dam_break_100_steps(variant):
    """Per-step list (3: strain pass and interaction over the list at the half
    step) and two neighbour lists per step (0)."""
    c = sps_case()
    eng = sph.Engine.create(c)
    eng.set_options(use_graph=1, pi_variant=variant)
    eng.step(100)
    s = eng.stats()
    st = eng.get_state()
    o = oracle.OracleState(c)
    o.step(100)
    od = o.diag()
    dp = c.params["dp"]
    assert abs(s["t"] - o.t.value) < 1e-3 * o.t.value
    assert abs(s["front"] - od["front"]) < 0.5 * dp
    assert abs(s["ke"] - od["ke"]) < 0.01 * od["ke"]
    assert np.abs(st["pos"] - o.pos).max() < 0.5 * dp
    assert s["flags"] == 0
    eng.destroy()


def test_mixed_physics_batch_matches_oracle():
    """One batch with the default model, Eq 19-20 diffusion and laminar + SPS
    viscosity: every case follows its own oracle."""
    cs = [cases.dam_break(0.04, seed=1),
          cases.dam_break(0.04, seed=2, ddt_mode=2),
          cases.dam_break(0.03, seed=3, column=(0.3, 0.2, 0.3), visc_mode=1, nu0=1e-3)]
    bat = sph.Engine.batch(cs)
    bat.step(30)
    for i, c in enumerate(cs):
        check_eval(c, bat, icase=i)
    bat.destroy()


@pytest.mark.parametrize("variant", [5, 4])
def test_pool_sps_case_equals_alone(variant):
    c = sps_case(0.04, seed=4)
    other = cases.dam_break(0.04, seed=5)
    pool = sph.Engine.pool(200000, 2000000, 4)
    pool.set_options(pi_variant=variant)
    pool.admit(other, t_end=1.0)
    s = pool.admit(c, t_end=1.0)
    pool.pool_step(8)
    e = sph.Engine.create(c)
    e.set_options(pi_variant=variant)
    e.step(8)
    a, b = pool.get_state(s), e.get_state()
    for k in ("pos", "vel", "rho"):
        assert np.array_equal(a[k], b[k]), k
    e.destroy()
    pool.destroy()


@pytest.mark.parametrize("variant", [5, 4, 3, 0])
def test_fourtakas_dam_break_steps(variant):
    """Eq 19-20 over whole steps, with the per-step list (3) and with two
    neighbour lists per step (0), against the oracle."""
    c = cases.dam_break(0.02, ddt_mode=2)
    eng = sph.Engine.create(c)
    eng.set_options(pi_variant=variant)
    eng.step(60)
    s, st = eng.stats(), eng.get_state()
    o = oracle.OracleState(c)
    o.step(60)
    od = o.diag()
    dp = c.params["dp"]
    assert abs(s["t"] - o.t.value) < 1e-3 * o.t.value
    assert abs(s["ke"] - od["ke"]) < 0.01 * od["ke"]
    assert np.abs(st["pos"] - o.pos).max() < 0.5 * dp
    assert np.abs(st["rho"] - o.rho).max() < 1.0
    assert s["flags"] == 0
    eng.destroy()
