"""The pins catch plausible mistakes: each case plants one slip in a copy of
the oracle's C source (on the CPU), builds it, and runs the pins against it
in a subprocess; the pins must fail.  The oracle itself is never modified."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "soc_oracle.c")

MUTANTS = {
    "uniform_not_cosine_entry": ("float mu = sqrtf(u);                 /* cosine-weighted inward angle */",
                                 "float mu = u;"),
    "exp_drops_ln2_lo": ("    r = fmaf(-t, LN2_LO, r);\n", ""),
    "log_drops_ln2_lo": ("return (t * LN2_LO + lm) + t * LN2_HI;", "return lm + t * LN2_HI;"),
    "series_one_term_short": ("    p = fmaf(p, r, 0x1.555556p-3f);             /* 1/3! */\n", ""),
    "hg_sign": ("mu = ((1.0f + g2) - tmp * tmp) / (g + g);", "mu = ((1.0f + g2) - tmp) / (g + g);"),
    "rotation_sign": ("ny = (sint * ((dy * dz) * c + dx * s)) / t + dy * mu;",
                      "ny = (sint * ((dy * dz) * c - dx * s)) / t + dy * mu;"),
    "sibling_entry_side": ("if (up && b == 0) { p->cell += 1 << a; p->x[a] = 0.0f;",
                           "if (up && b == 0) { p->cell += 1 << a; p->x[a] = 1.0f;"),
    "climb_drops_octant": ("p->x[i] = (p->x[i] + (float)((oct >> i) & 1)) * 0.5f;", "p->x[i] = p->x[i] * 0.5f;"),
    "level_scale_kept": ("        p->h = p->h * 0.5f;\n        p->cell = G->child", "        p->cell = G->child"),
    "face_area_swap": ("cum[1] = cum[0] + ax; cum[2] = cum[1] + ay;", "cum[1] = cum[0] + ay; cum[2] = cum[1] + ax;"),
    "free_path_halved": ("tauf = -oracle_log(rng_u(r));\n            continue;",
                         "tauf = -0.5f * oracle_log(rng_u(r));\n            continue;"),
    "point_source_hemisphere": ("float mu = 2.0f * rng_u(r) - 1.0f;\n    float c, s;\n    disk_azimuth(r, &c, &s);\n    float sint",
                                "float mu = rng_u(r);\n    float c, s;\n    disk_azimuth(r, &c, &s);\n    float sint"),
    "escape_not_counted": ("            st->escaped += (int64_t)p.W;\n", ""),
    "philox_key_bump": ("k0 += PHILOX_W0; k1 += PHILOX_W1;", "k0 += PHILOX_W1; k1 += PHILOX_W0;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new, 1))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    "-o", str(so), str(mut), "-lm"], check=True)
    env = dict(os.environ, SOC_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"


# The FP64 tracer: its own pins plus its agreement with the FP32 contract
# (test_oracle_fp64.py) must catch a slip planted in it.
SRC64 = os.path.join(ROOT, "oracle", "soc_oracle64.c")
MUTANTS64 = {
    "fp64_uniform_not_cosine_entry": ("p->d[a] = low ? sqrt(u) : -sqrt(u);", "p->d[a] = low ? u : -u;"),
    "fp64_hg_sign": ("(1.0 + g * g - q * q) / (2.0 * g)", "(1.0 + g * g - q) / (2.0 * g)"),
    "fp64_level_scale_dropped": ("-expm1(-rho * it->kabs * p->h * seg)", "-expm1(-rho * it->kabs * seg)"),
    "fp64_free_path_halved": ("double tauf = -log(draw(s));", "double tauf = -0.5 * log(draw(s));"),
    "fp64_climb_drops_octant": ("p->x[i] = 0.5 * (p->x[i] + ((oct >> i) & 1));", "p->x[i] = 0.5 * p->x[i];"),
    "fp64_escape_not_counted": ("if (!next_cell(G, p, axis)) { st->escaped += p->W; break; }",
                                "if (!next_cell(G, p, axis)) { break; }"),
    "fp64_stream_key_without_freq": ("^ ((uint32_t)it->iteration << 16) ^ (uint32_t)it->freq;",
                                     "^ ((uint32_t)it->iteration << 16);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS64))
def test_fp64_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS64[name]
    src = open(SRC64).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mut = tmp_path / "mut64.c"
    mut.write_text(src.replace(old, new, 1))
    so = tmp_path / "libmut64.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    "-o", str(so), str(mut), SRC, "-lm"], check=True)
    env = dict(os.environ, SOC_ORACLE64_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_fp64.py")],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
