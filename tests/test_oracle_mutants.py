"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins catch
each one: a pin suite that passes a mutated oracle would not be pinning anything.

Each mutant is a one-token change of oracle/bm_oracle.c compiled into a private
library; the pin tests run against it in a subprocess and must fail.  The
discharge-inflow boundary (its conveyance split, momentum flux, critical depth and
wave speed) is caught by tests/test_oracle_inflow.py, the outflow laws (Poleni's weir,
the h-Q split and rating curve, the characteristic boundary state) by
tests/test_oracle_outflow.py, the speeds of Eq. 16 by the coupled-system bracket in
tests/test_oracle_morpho.py.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "bm_oracle.c")

# (name, original text, mutated text); every original occurs exactly once
MUTANTS = [
    ("pressure_correction_sign", "double GL = F[1] - pL, GR = F[1] - pR;",
     "double GL = F[1] + pL, GR = F[1] - pR;"),
    ("modified_state_min_bed", "double zs = fmax(m->z[L], m->z[R]);", "double zs = fmin(m->z[L], m->z[R]);"),
    ("contact_picks_wrong_side", "F[2] = H0 * (Ss >= 0 ? vL : vR);", "F[2] = H0 * (Ss >= 0 ? vR : vL);"),
    ("wave_speed_sign", "double us = 0.5 * (uL + uR) + cL - cR;", "double us = 0.5 * (uL + uR) - cL + cR;"),
    ("dry_front_speed", "*SL = uL - cL; *SR = uL + 2 * cL;", "*SL = uL - cL; *SR = uL + cL;"),
    ("wall_not_mirrored", "orc_hllc(hs, unL, utL, hs, -unL, utL, g, F);",
     "orc_hllc(hs, unL, utL, hs, unL, utL, g, F);"),
    ("rho_factor", "double rho = 4.0 * m->area[i] / (3.0 * m->len[e]);\n        if (m->p.cfl_mode == 0 && rho",
     "double rho = 2.0 * m->area[i] / (3.0 * m->len[e]);\n        if (m->p.cfl_mode == 0 && rho"),
    ("friction_stage_state", "double k1 = c * sqrt(q1x * q1x + q1y * q1y);",
     "double k1 = c * sqrt(q0x * q0x + q0y * q0y);"),
    ("friction_exponent", "double c = g * n * n / pow(h, 7.0 / 3.0);", "double c = g * n * n / pow(h, 4.0 / 3.0);"),
    ("normal_transposed", "m->nx[e] = dy / l;\n    m->ny[e] = -dx / l;", "m->nx[e] = -dy / l;\n    m->ny[e] = dx / l;"),
    ("tangent_rotation", "double unL = uL * nx + vL * ny, utL = -uL * ny + vL * nx;",
     "double unL = uL * nx + vL * ny, utL = uL * ny + vL * nx;"),
    ("update_sign", "double Hn = H[i] - r * s0;", "double Hn = H[i] + r * s0;"),
    ("hll_state_jump", "double H0 = FL0 - SL * ((FR0 - FL0) - SR * (hR - hL)) / d;",
     "double H0 = FL0 - SL * ((FR0 - FL0) - SR * (hL - hR)) / d;"),
]
# flood tracking, caught by tests/test_oracle_tracking.py
TRACK_MUTANTS = [
    ("track_shear_exponent", "u * u / cbrt(h);", "u * u / sqrt(h);"),
    ("track_arrival_threshold", "if (isnan(arr[i]) && h > h_arr) arr[i] = t;",
     "if (isnan(arr[i]) && h > hmin) arr[i] = t;"),
    ("track_max_of_surface", "if (h > hmax[i]) hmax[i] = h;", "if (H[i] > hmax[i]) hmax[i] = H[i];"),
    ("track_discharge_as_velocity", "u = q / h;", "u = q;"),
]
# passive scalars, caught by tests/test_oracle_scalars.py
SCALAR_MUTANTS = [
    ("scalar_contact_side", "orc_hllc(hLs, unL, pL, hRs, unR, phi[c * n + R], g, F);",
     "orc_hllc(hLs, unL, phi[c * n + R], hRs, unR, pL, g, F);"),
    ("scalar_update_sign", "double v = hc[c * n + i] - r * sum;", "double v = hc[c * n + i] + r * sum;"),
    ("scalar_inflow_sign", "f = q > 0 ? -q * c_in[c] : 0.0;", "f = q > 0 ? q * c_in[c] : 0.0;"),
    ("scalar_concentration_of_surface", "double h = H[i] - m->z[i];\n      for (int c = 0; c < K; ++c) phi",
     "double h = H[i];\n      for (int c = 0; c < K; ++c) phi"),
]

SOURCE_MUTANTS = [
    ("source_mm_per_hour", "v / 3.6e6;", "v / 3.6e3;"),
    ("source_region_area", "m->src_area[reg[i]] += m->area[i];", "m->src_area[reg[i]] = m->area[i];"),
    ("source_sign", "Hn = Hn + add;", "Hn = Hn - add;"),
    ("sink_available_test", "(Hn - m->z[i]) + add < 0", "(Hn - m->z[i]) - add < 0"),
]

MORPHO_MUTANTS = [
    ("bed_update_sign", "const double dz = -(dt / m->area[i] * sum)", "const double dz = +(dt / m->area[i] * sum)"),
    ("bed_porosity", "* sum) / (1.0 - m->mp_p);", "* sum) / (1.0 + m->mp_p);"),
    ("bed_keeps_surface", "      H[i] += dz;", "      H[i] += 0.0 * dz;"),
    ("shields_depth_power", "(sd * d * cbrt(h))", "(sd * d * h)"),
    ("eq16_root_sign", "const double r = sqrt(a * a + 4.0 * dqb * c * c);",
     "const double r = sqrt(a * a - 4.0 * dqb * c * c);"),
    ("eq16_root_factor", "const double r = sqrt(a * a + 4.0 * dqb * c * c);",
     "const double r = sqrt(a * a + 2.0 * dqb * c * c);"),
    ("eq16_celerity_sign", "const double a = un - c;", "const double a = un + c;"),
    ("eq16_bedload_derivative", "(2.0 * theta / sp) / h;", "(theta / sp) / h;"),
]

# discharge inflow, caught by tests/test_oracle_inflow.py
INFLOW_MUTANTS = [
    ("inflow_weight_by_depth", "return h > h_min ? l * pow(h, 5.0 / 3.0) : 0.0;", "return h > h_min ? l * h : 0.0;"),
    ("inflow_momentum_factor", "Gn = q * q / hb + 0.5 * g * hb * hb - p;", "Gn = q * q / hb + g * hb * hb - p;"),
    ("inflow_wave_speed", "double lb = m->qin[e] / hb + sqrt(g * hb);", "double lb = sqrt(g * hb);"),
    ("inflow_critical_depth", "double hcr = cbrt(q * q / g);", "double hcr = sqrt(q * q / g);"),
    ("inflow_dry_split_per_edge", "m->qin[e] = m->inflow_len > 0 ? Q / m->inflow_len : 0.0;",
     "m->qin[e] = m->inflow_len > 0 ? Q * m->len[e] / m->inflow_len : 0.0;"),
]

# outflow boundaries (h-Q relation, weir), caught by tests/test_oracle_outflow.py
OUTFLOW_MUTANTS = [
    ("weir_poleni_factor", "return (2.0 / 3.0) * mu * sqrt(2.0 * g) * eta * sqrt(eta);",
     "return (1.0 / 3.0) * mu * sqrt(2.0 * g) * eta * sqrt(eta);"),
    ("weir_gravity", "return (2.0 / 3.0) * mu * sqrt(2.0 * g) * eta * sqrt(eta);",
     "return (2.0 / 3.0) * mu * sqrt(g) * eta * sqrt(eta);"),
    ("weir_head_exponent", "return (2.0 / 3.0) * mu * sqrt(2.0 * g) * eta * sqrt(eta);",
     "return (2.0 / 3.0) * mu * sqrt(2.0 * g) * eta * cbrt(eta);"),
    ("weir_crest_below_bed", "double crest = m->weir_crest > m->z[i] ? m->weir_crest : m->z[i];",
     "double crest = m->weir_crest;"),
    ("outflow_invariant_factor", "const double w = un + 2.0 * sqrt(g * h), sg = sqrt(g);",
     "const double w = un + sqrt(g * h), sg = sqrt(g);"),
    ("outflow_critical_cap", "const double qmax = w * w * w / (27.0 * g);", "const double qmax = w * w * w / (8.0 * g);"),
    ("outflow_wave_speed", "double lb = hb > 0 ? q / hb + sqrt(g * hb) : 0.0;", "double lb = hb > 0 ? sqrt(g * hb) : 0.0;"),
    ("outflow_momentum_cell_depth", "Gn = qo * (qo / hbo) + 0.5 * g * hbo * hbo - p;", "Gn = qo * (qo / hs);"),
    ("hq_uniform_split", "m->qout[e] = Q * inflow_weight(m->len[e], h, hmin) / (m->len[e] * W);",
     "m->qout[e] = Q / sl;"),
    ("rating_segment", "double w = (S - m->hq_s[k - 1]) / (m->hq_s[k] - m->hq_s[k - 1]);",
     "double w = (S - m->hq_s[k - 1]) / (m->hq_s[k] - m->hq_s[0]);"),
]

# water-level boundary, caught by tests/test_oracle_level.py
LEVEL_MUTANTS = [
    ("level_invariant_factor", "un + 2.0 * sqrt(g * h) - 2.0 * sqrt(g * *hb)", "un + sqrt(g * h) - sqrt(g * *hb)"),
    ("level_invariant_sign", "un + 2.0 * sqrt(g * h) - 2.0 * sqrt(g * *hb)", "un - 2.0 * sqrt(g * h) + 2.0 * sqrt(g * *hb)"),
    ("level_not_over_bed", "*hb = fmax(0.0, m->zh_now - m->z[i]);", "*hb = fmax(0.0, m->zh_now);"),
    ("level_flux_of_cell_state", "orc_hllc(hs, unL, utL, hb, ub, utL, g, F);", "orc_hllc(hs, unL, utL, hs, unL, utL, g, F);"),
    ("level_frozen_in_time", "m->zh_now = level_at(m, t);", "m->zh_now = level_at(m, 0.0);"),
]

FRICTION_MUTANTS = [
    ("chezy_constant", "return h > r ? 6.25 + log(h / r) : 6.25;", "return h > r ? 6.5 + log(h / r) : 6.25;"),
    ("bezzola_branch", "if (x > 2.0) return", "if (x > 1.0) return"),
    ("closure_cf_squared", "double c = 1.0 / (h * h * cf * cf);", "double c = 1.0 / (h * h * cf);"),
]


@pytest.mark.slow
@pytest.mark.parametrize("name,orig,mut,pins",
                         [m + ("test_oracle_pins.py",) for m in MUTANTS]
                         + [m + ("test_oracle_tracking.py",) for m in TRACK_MUTANTS]
                         + [m + ("test_oracle_scalars.py",) for m in SCALAR_MUTANTS]
                         + [m + ("test_oracle_sources.py",) for m in SOURCE_MUTANTS]
                         + [m + ("test_oracle_morpho.py",) for m in MORPHO_MUTANTS]
                         + [m + ("test_oracle_friction.py",) for m in FRICTION_MUTANTS]
                         + [m + ("test_oracle_inflow.py",) for m in INFLOW_MUTANTS]
                         + [m + ("test_oracle_outflow.py",) for m in OUTFLOW_MUTANTS]
                         + [m + ("test_oracle_level.py",) for m in LEVEL_MUTANTS],
                         ids=[m[0] for m in MUTANTS + TRACK_MUTANTS + SCALAR_MUTANTS + SOURCE_MUTANTS
                              + MORPHO_MUTANTS + FRICTION_MUTANTS + INFLOW_MUTANTS + OUTFLOW_MUTANTS
                              + LEVEL_MUTANTS])
def test_pins_catch_mutant(name, orig, mut, pins, tmp_path):
    src = open(SRC).read()
    assert src.count(orig) == 1, f"mutation site for {name} not unique"
    msrc = tmp_path / "bm_oracle_mutant.c"
    msrc.write_text(src.replace(orig, mut))
    env = dict(os.environ, ORACLE_MUTANT_SRC=str(msrc), ORACLE_MUTANT_LIB=str(tmp_path / "libmut.so"),
               PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
