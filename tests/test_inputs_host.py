"""The seeded input generators (paper_2104_00537_gb300/cases.py) against the
workloads they stand in for: the 3-D dam break of SPHERIC test 2 at the two
resolutions, the uneven batch, the wave flume with its piston wavemaker, and
the sloshing-tank serving trace.  Host only (no GPU).

Checked here: particle counts, the constants every case carries (h = sqrt(3)
dp, cs0 = 10 sqrt(g H), the Tait exponent), the hydrostatic start (Eq 28
solved for the density at rho0 g d), the jitter bound, the parameter ranges
of the batch and the trace, and that a seed fixes every array.
"""
import math

import numpy as np
import pytest

from paper_2104_00537_gb300 import cases

G = 9.81


def lattice_offsets(c):
    """Distance of each fluid coordinate from the nearest lattice point (dp units)."""
    f = c.ptype == 0
    x = c.pos[f] / c.params["dp"]
    return np.abs(x - np.round(x))


@pytest.mark.parametrize("dp,nf,nb", [(0.02, 8000, 20062), (0.004, 1000000, 479826)])
def test_dam_break_counts_and_constants(dp, nf, nb):
    c = cases.dam_break(dp)
    assert c.n_fluid == nf and c.n - c.n_fluid == nb
    p = c.params
    assert p["h"] == pytest.approx(math.sqrt(3.0) * dp)
    assert p["cs0"] == pytest.approx(10.0 * math.sqrt(G * 0.4))
    assert (p["rho0"], p["gamma"], p["alpha"], p["delta"], p["cfl"]) == (1000.0, 7.0, 0.01,
                                                                         0.1, 0.2)
    # the fluid sits on the lattice to within the seeded jitter of 1e-4 dp
    off = lattice_offsets(c)
    assert off.max() <= 1e-4 * (1 + 1e-9) and off.max() > 0.5e-4
    # two wall layers: boundary particles exactly on the lattice
    b = c.ptype == 1
    assert np.all(np.abs(c.pos[b] / dp - np.round(c.pos[b] / dp)) < 1e-9)


def test_dam_break_hydrostatic_start():
    """Fluid densities make the Tait pressure (Eq 28) equal rho0 g d, d the
    depth below the surface half a spacing above the top layer."""
    c = cases.dam_break(0.02)
    p = c.params
    f = c.ptype == 0
    d = (20 + 0.5) * 0.02 - c.pos[f, 2]
    B = p["cs0"] ** 2 * p["rho0"] / p["gamma"]
    P = B * ((c.rho[f] / p["rho0"]) ** p["gamma"] - 1.0)
    # densities are stored in FP32: relative 6e-8 of rho moves P by 7 x that of B
    assert np.abs(P - p["rho0"] * G * d).max() < 7 * 6e-8 * B * 1.5
    assert np.all(c.vel == 0.0)


def test_a_seed_fixes_every_array():
    a, b = cases.dam_break(0.04, seed=3), cases.dam_break(0.04, seed=3)
    for k in ("pos", "vel", "rho", "ptype", "group"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
    c = cases.dam_break(0.04, seed=4)
    assert not np.array_equal(a.pos, c.pos)
    assert np.array_equal(a.ptype, c.ptype)


def test_uneven_batch_follows_its_recipe():
    """256 dam breaks: fluid counts log-uniform over 5k-200k, column width /
    height ratio in [0.5, 2], tank length 3-5 x the column width (within the
    rounding of lengths to whole spacings), one seed per case."""
    cs = cases.batch_dam_breaks(256, seed=0)
    assert len(cs) == 256
    nf = np.array([c.n_fluid for c in cs], np.float64)
    assert nf.min() >= 0.8 * 5000 and nf.max() <= 1.2 * 200000
    # log-uniform: the logs spread evenly (quartiles near 1/4 and 3/4 of the span)
    u = (np.log(nf) - math.log(5000)) / (math.log(200000) - math.log(5000))
    q1, q3 = np.quantile(u, [0.25, 0.75])
    assert 0.15 < q1 < 0.35 and 0.65 < q3 < 0.85
    dp = cs[0].params["dp"]
    for c in cs:
        w, _, H = c.meta["column"]
        L = c.meta["tank"][0]
        assert 0.5 * (1 - 2 * dp / H) <= w / H <= 2.0 * (1 + 2 * dp / H)
        assert 3.0 * w - 2 * dp <= L <= 5.0 * w + 2 * dp
        assert c.params["cs0"] == pytest.approx(10.0 * math.sqrt(G * H))
    seeds = [c.meta["seed"] for c in cs]
    assert len(set(seeds)) == 256
    assert sum(c.n for c in cs) == pytest.approx(26.56e6, rel=0.01)


def test_wave_flume_counts_and_piston():
    """The 25 x 1 x 1.2 m flume filled to 0.6 m: (L/dp - 1)(W/dp - 1)(D/dp)
    fluid particles (29.05M at dp = 0.008 m, 120.4M at the config's 0.005 m,
    counted from the same lattice here at a coarse dp); the piston is one
    group of boundary particles moving as (stroke/2) sin(2 pi t / period)."""
    for dp, expect in ((0.008, 3124 * 124 * 75), (0.005, 4999 * 199 * 120)):
        nx, ny, nz = round(25.0 / dp), round(1.0 / dp), round(0.6 / dp)
        assert (nx - 1) * (ny - 1) * nz == expect
    assert 3124 * 124 * 75 == pytest.approx(29.05e6, rel=1e-3)
    c = cases.wave_flume(0.04)
    assert c.n_fluid == (625 - 1) * (25 - 1) * 15
    m = c.motions[0]
    assert m["amp"] == pytest.approx(0.05) and m["omega"] == pytest.approx(2 * math.pi / 1.5)
    piston = c.group == 0
    assert piston.sum() > 0 and np.all(c.ptype[piston] == 1)
    assert np.all(c.pos[piston, 0] <= 1e-12)
    # at t = 0 the piston moves at amp * omega along x
    assert np.allclose(c.vel[piston], [m["amp"] * m["omega"], 0.0, 0.0], rtol=1e-6)


def test_sloshing_trace_follows_its_recipe():
    """Poisson arrivals at 20 requests per second, fluid counts log-uniform
    over the range, fill depth 0.2-0.4 m, amplitude 0.01-0.05 m, frequency
    0.5-1.5 Hz; the same seed gives the same trace."""
    tr = cases.sloshing_trace(200, rate=20.0, seed=0, n_min=10000, n_max=20000, t_end=1.0)
    t = np.array([a for a, _, _ in tr])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert gaps.mean() == pytest.approx(1.0 / 20.0, rel=0.2)
    # exponential gaps: coefficient of variation near 1
    assert 0.75 < gaps.std() / gaps.mean() < 1.25
    for _, c, te in tr:
        assert te == 1.0
        assert 0.75 * 10000 <= c.n_fluid <= 1.25 * 20000
        assert 0.2 <= c.meta["depth"] <= 0.4
        assert 0.01 <= c.meta["amp"] <= 0.05
        assert 0.5 <= c.meta["freq"] <= 1.5
        assert c.motions[0]["amp"] == c.meta["amp"]
    again = cases.sloshing_trace(200, rate=20.0, seed=0, n_min=10000, n_max=20000, t_end=1.0)
    assert all(a == b and np.array_equal(ca.pos, cb.pos)
               for (a, ca, _), (b, cb, _) in zip(tr, again))
