"""Plant plausible mistakes in copies of the oracle (a dropped term, a wrong sign, a wrong
index, a transposed operand) and check that the pin suite fails on every one of them."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mkoracle.c")
PINS = ["tests/test_oracle_propagation.py", "tests/test_oracle_kalman.py", "tests/test_oracle_search.py",
        "tests/test_oracle_modules.py", "tests/test_oracle_highland.py"]

MUTANTS = {
    "jacobian_sign": ("A[0 * 6 + 4] = -dy;", "A[0 * 6 + 4] = dy;"),
    "jacobian_dk": ("A[4 * 6 + 3] = -cB * s;", "A[4 * 6 + 3] = cB * s;"),
    "transport_transposed": ("acc += T[i][l] * J[j * 6 + l];", "acc += T[i][l] * J[l * 6 + j];"),
    "ms_dropped_kk": ("C[ix(3, 3)] += k * k * cot * cot * th02;", ";"),
    "ms_ktheta_sign": ("C[ix(5, 3)] += -k * cot * th02;", "C[ix(5, 3)] += k * cot * th02;"),
    "ms_phi_sin": ("C[ix(4, 4)] += th02 / (st * st);", "C[ix(4, 4)] += th02;"),
    "highland_log": ("log(t / (beta * beta))", "log(t * beta * beta)"),
    "highland_scale": ("*theta0 = 0.0136 /", "*theta0 = 0.0141 /"),
    "highland_log_coefficient": ("(1.0 + 0.038 * log", "(1.0 + 0.040 * log"),
    "eloss_sign": ("double e2 = e - direction * orc_eloss(pm, t);", "double e2 = e + direction * orc_eloss(pm, t);"),
    "update_sign": ("pout[i] = p[i] + K[i][0] * r[0]", "pout[i] = p[i] - K[i][0] * r[0]"),
    "chi2_index": ("double y2 = (r[2] - Lc[3] * y0 - Lc[4] * y1) / Lc[5];",
                   "double y2 = (r[2] - Lc[4] * y0 - Lc[3] * y1) / Lc[5];"),
    "helix_cot": ("out[2] = p[2] + s * cos(p[5]) / sin(p[5]);", "out[2] = p[2] + s * sin(p[5]) / cos(p[5]);"),
    "seed_charge": ("k = -om / cB;", "k = om / cB;"),
    "seed_straight_threshold": ("if (fabs(cross) < 1e-12 * chord2) {", "if (fabs(cross) < 1e-7 * chord2) {"),
    "seed_module_plane_ignored": ("if (ids) {\n            if (!at_hit_surface(g, ids[j]",
                                  "if (0) {\n            if (!at_hit_surface(g, ids[j]"),
    "window_index": ("ve += ge[i] * M[i][j] * ge[j];", "ve += ge[i] * M[i][i] * ge[j];"),
    "miss_penalty_sign": ("ch.score = cd->score - P->score_hole;", "ch.score = cd->score + P->score_hole;"),
    "child_order": ("if (x->score != y->score) return x->score > y->score ? -1 : 1;",
                    "if (x->score != y->score) return x->score < y->score ? -1 : 1;"),
    "bin_guard": ("int e0 = eta_bin(L, w[0] - w[2] - eps), e1 = eta_bin(L, w[0] + w[2] + eps);",
                  "int e0 = eta_bin(L, w[0]), e1 = eta_bin(L, w[0]);"),
    "plane_jacobian_dropped_z": ("double gp = n[0] * A[0 * 6 + j] + n[1] * A[1 * 6 + j] + n[2] * A[2 * 6 + j];",
                                 "double gp = n[0] * A[0 * 6 + j] + n[1] * A[1 * 6 + j];"),
    "module_ignored": ("int m = hit_module(g, id);\n    if (margin)", "int m = -1;\n    if (margin)"),
    "overlap_same_module": ("if (hit_module(g, mh->v[q].gid) != hit_module(g, b1)) b2 = mh->v[q].gid;",
                            "if (hit_module(g, mh->v[q].gid) == hit_module(g, b1)) b2 = mh->v[q].gid;"),
    "bkfit_module_ignored": ("if (!at_hit_surface(g, h, q, Cq, pp, Cp, NULL)) { st = 1; break; }",
                             "memcpy(pp, q, sizeof(q)); memcpy(Cp, Cq, sizeof(Cq));"),
    "overlap_swapped": ("k->ovl = hit_module(g, k->gid) != hit_module(g, b1) ? b1 : b2;",
                        "k->ovl = hit_module(g, k->gid) != hit_module(g, b1) ? b2 : b1;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-I", os.path.join(ROOT, "oracle"), "-o", str(so), str(mut), "-lm"])
    env = dict(os.environ, MKORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode != 0, f"pins did not catch mutant {name}:\n{r.stdout[-2000:]}"


def _compile(src_text, tmp_path):
    mut = tmp_path / "mut.c"
    mut.write_text(src_text)
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-I", os.path.join(ROOT, "oracle"), "-o", str(so), str(mut), "-lm"])
    return so


def test_highland_scale_shared_with_the_generator_is_caught(tmp_path):
    """The same wrong Highland scale typed into the oracle and into the event generator: the
    oracle still models the simulated detector (their agreement test passes), and only the PDG
    pin fails."""
    src = open(SRC).read()
    old, new = MUTANTS["highland_scale"]
    so = _compile(src.replace(old, new), tmp_path)
    driver = (
        "import sys; sys.path.insert(0, %r)\n"
        "import numpy as np\n"
        "from paper_2312_11728_gb300 import synth as S\n"
        "def _hl(p, t):\n"
        "    beta = p / np.sqrt(p * p + 0.13957039 ** 2)\n"
        "    return 0.0141 / (beta * p) * np.sqrt(t) * (1.0 + 0.038 * np.log(t / (beta * beta)))\n"
        "S._highland = _hl\n"
        "import pytest\n"
        "sys.exit(pytest.main(['-q', '-p', 'no:cacheprovider', sys.argv[1]]))\n" % ROOT)
    env = dict(os.environ, MKORACLE_LIB=str(so))
    agree = subprocess.run([sys.executable, "-c", driver,
                            "tests/test_oracle_propagation.py::test_material_model_equals_the_simulated_detector"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert agree.returncode == 0, agree.stdout[-2000:]
    pin = subprocess.run([sys.executable, "-c", driver, "tests/test_oracle_highland.py"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert pin.returncode != 0, pin.stdout[-2000:]
