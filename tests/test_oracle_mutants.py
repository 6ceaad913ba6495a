"""Each pin of the FP64 oracle fails on a plausible mistake in the equation it
guards.

For every mistake below, a copy of oracle/sph_oracle.c with that one mistake
planted is compiled with gcc (on the CPU), every call of the oracle module is
routed to that build (oracle.library), and the pin is run: it must fail.  A
control build of the unpatched copy, made the same way, must pass every pin
used here, so a failure comes from the planted mistake and from nothing else.
The oracle itself is never modified.
"""
import os

import pytest

import oracle
from oracle import build as obuild
from tests import test_oracle_pins as pins

SRC = obuild.SRC

# context that is unique to orc_step (the Symplectic step)
_DT_LINE = ("    double dt = orc_dt(p, n, acc, mu, type, out);\n    double t0 = *t;\n"
            "    memcpy(pos0, pos, sizeof(double) * 3 * (size_t)n);\n")

MUTANTS = {
    # Eq 33: the velocity corrector with the force of state n instead of n+1/2
    "eq33_corrector_uses_F_n": (
        [(_DT_LINE, _DT_LINE.replace(
            "    double t0", "    double *acc_n = (double *)malloc(sizeof(double) * 3 * N);\n"
            "    memcpy(acc_n, acc, sizeof(double) * 3 * (size_t)n);\n    double t0")),
         ("double vn = vel0[3 * a + k] + dt * acc[3 * a + k];",
          "double vn = vel0[3 * a + k] + dt * acc_n[3 * a + k];")],
        [pins.test_symplectic_scheme_is_second_order]),
    # Eq 33: the position corrector with v^n alone (forward Euler)
    "eq33_position_with_v_n": (
        [("pos[3 * a + k] = pos0[3 * a + k] + dt * 0.5 * (vn + vel0[3 * a + k]);",
          "pos[3 * a + k] = pos0[3 * a + k] + dt * vel0[3 * a + k];")],
        [pins.test_symplectic_scheme_is_second_order]),
    # Eq 34: the first-order factor 1 - eps instead of (2 - eps)/(2 + eps)
    "eq34_one_minus_eps": (
        [("double rhonew = rho0[a] * (2.0 - eps) / (2.0 + eps);",
          "double rhonew = rho0[a] * (1.0 - eps);")],
        [pins.test_symplectic_density_update_against_the_closed_form]),
    # Eq 34: the half-step density as the base of the update
    "eq34_half_step_base": (
        [("double rhonew = rho0[a] * (2.0 - eps) / (2.0 + eps);",
          "double rhonew = rho[a] * (2.0 - eps) / (2.0 + eps);")],
        [pins.test_symplectic_density_update_against_the_closed_form]),
    # Eq 34: eps from the density rate of state n instead of n+1/2
    "eq34_eps_from_R_n": (
        [(_DT_LINE, _DT_LINE.replace(
            "    double t0", "    double *drho_n = (double *)malloc(sizeof(double) * N);\n"
            "    memcpy(drho_n, drho, sizeof(double) * (size_t)n);\n    double t0")),
         ("double eps = -(drho[a] / rho[a]) * dt;", "double eps = -(drho_n[a] / rho[a]) * dt;")],
        [pins.test_symplectic_density_update_against_the_closed_form]),
    # Eq 21: mu_ab without the factor h
    "eq21_mu_without_h": (
        [("double muab = p->h * vr / (r2 + p->eta2);", "double muab = vr / (r2 + p->eta2);")],
        [pins.test_artificial_viscosity_two_particle_value]),
    # Eq 21: rho_a in place of the mean density
    "eq21_rho_a_for_the_mean": (
        [("double rhobar = 0.5 * (rhoa + rhob);", "double rhobar = rhoa;")],
        [pins.test_artificial_viscosity_two_particle_value]),
    # Eq 21: eta (0.001 h^2 read as eta, not eta^2)
    "eq21_eta_not_squared": (
        [("double muab = p->h * vr / (r2 + p->eta2);",
          "double muab = p->h * vr / (r2 + p->eta2 * p->eta2);")],
        [pins.test_artificial_viscosity_two_particle_value]),
    # Eq 18 as printed (anti-diffusive orientation)
    "eq18_printed_sign": (
        [("double psi_dot_gradW = -2.0 * drho_ba * F;", "double psi_dot_gradW = 2.0 * drho_ba * F;")],
        [pins.test_density_diffusion_bump_sign_and_conservation]),
    # Eq 11: a_D of the 2-D kernel (7 / (4 pi h^2)) in 3-D
    "eq11_2d_normalisation": (
        [("  double aD = 21.0 / (16.0 * M_PI * h * h * h);\n  double t = 1.0 - 0.5 * q;\n"
          "  return aD * t * t * t * t",
          "  double aD = 7.0 / (4.0 * M_PI * h * h);\n  double t = 1.0 - 0.5 * q;\n"
          "  return aD * t * t * t * t")],
        [lambda: pins.test_wendland_normalises_to_one(0.0346)]),
    # Eq 28 without the -1 (no zero pressure at rho0)
    "eq28_without_minus_one": (
        [("return B * (pow(rho / p->rho0, p->gamma) - 1.0);",
          "return B * pow(rho / p->rho0, p->gamma);")],
        [pins.test_tait_reference_state_and_sound_speed]),
    # Eq 35: dt_f without the square root
    "eq35_dt_f_without_sqrt": (
        [("double d = sqrt(p->h / f);", "double d = p->h / f;")],
        [lambda: pins.test_time_step_isolated_particle_closed_form(2.0e4)]),
    # Eq 38: a non-positive extrapolated boundary density used as it is
    "eq38_no_fallback": (
        [("    if (!(rB > 0.0 && rB < 1e30)) rB = rhs[0] / sw; /* not a usable density: Shepard */\n",
          "")],
        [pins.test_mdbc_non_positive_extrapolation_takes_the_shepard_value]),
}


def build_variant(tmp_path, name, patches):
    """Compile a copy of sph_oracle.c with `patches` applied (each old text
    must occur exactly once) into a uniquely named library."""
    src = open(SRC).read()
    for old, new in patches:
        assert src.count(old) == 1, (name, old)
        src = src.replace(old, new)
    c = os.path.join(str(tmp_path), "orc_%s.c" % name)
    with open(c, "w") as f:
        f.write(src)
    return obuild.compile_source(c, os.path.join(str(tmp_path), "liborc_%s.so" % name))


def test_control_build_passes_the_pins(tmp_path):
    lib = build_variant(tmp_path, "control", [])
    with oracle.library(lib):
        seen = set()
        for _, checks in MUTANTS.values():
            for check in checks:
                if id(check) not in seen:
                    seen.add(id(check))
                    check()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pin_fails_on_planted_mistake(tmp_path, name):
    patches, checks = MUTANTS[name]
    lib = build_variant(tmp_path, name, patches)
    with oracle.library(lib):
        for check in checks:
            with pytest.raises(AssertionError):
                check()
