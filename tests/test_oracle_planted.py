"""Planted mistakes: each plausible error in the oracle (a dropped term, a
reversed tie-break, a wrong index or transition) is written into a copy of
its source, compiled on the CPU, and run against the oracle's pins (the
hand-worked examples, the set-based restatements, the invariants); every
mutant must fail at least one. This shows the pins constrain every step,
not only that the oracle passes them."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "snnmap_oracle.c")

MUTANTS = [
    ("shared inbound count dropped",
     "if (nd && is_dest(L, a, m)) s->ov[m] += L->k[a];", "if (0) s->ov[m] += L->k[a];"),
    ("candidate ties to the higher id",
     "(s->score[m] == bs && m < best)", "(s->score[m] == bs && m > best)"),
    ("best child ties to the higher id",
     "(cscore[c] == cscore[best] && c < best)", "(cscore[c] == cscore[best] && c > best)"),
    ("self-destination not recorded",
     "if (tmp[i] == s2) { sd = 1; continue; }", "if (tmp[i] == s2) { continue; }"),
    ("internal axons lost", "if (sd) internal[s2] += L->k[a];", "if (0) internal[s2] += L->k[a];"),
    ("Conn counts lambda, not lambda - 1",
     "cost += L->w[a] * (lam - 1);", "cost += L->w[a] * lam;"),
    ("save counted where two pins share the partition",
     "if (pc.cnt[j] == 1) save += L->w[a];", "if (pc.cnt[j] == 2) save += L->w[a];"),
    ("Delta test ignores already-inbound axons",
     "ps[p].pin_cnt + L->in_count[n] - ovp[p] <= prm->delta;",
     "ps[p].pin_cnt + L->in_count[n] <= prm->delta;"),
    ("move ties to the higher partition",
     "(gain == bg && p < best)", "(gain == bg && p > best)"),
    ("zero-gain moves proposed",
     "(bg > 0 || prm->refine_nonpositive)", "(bg >= 0 || prm->refine_nonpositive)"),
    ("variant flag ignored",
     "(bg > 0 || prm->refine_nonpositive)", "(bg > 0)"),
    ("inbound transition off by one",
     "if (dcf == 1) ps2[f].pin_cnt -= L->k[a];", "if (dcf == 0) ps2[f].pin_cnt -= L->k[a];"),
    ("replayed gain charges a non-empty target",
     "g += L->w[a] * ((cf == 1 ? 1 : 0) - (ct == 0 ? 1 : 0));",
     "g += L->w[a] * ((cf == 1 ? 1 : 0) - (ct == 1 ? 1 : 0));"),
    ("prefix ties to the longest",
     "nviol == 0 && G > 0 && G > bestG)", "nviol == 0 && G > 0 && G >= bestG)"),
    ("G_P keeps self-cycles",
     "if (tmp[i] == s2) continue;            /* self-cycle broken */", ""),
    ("G_P loses internal weight", "inw += L->w[a];", "inw += 0;"),
    ("force without the max(., 1) term",
     "s += mdist(width, h, g[q]) - (dk > 1 ? dk : 1);", "s += mdist(width, h, g[q]) - dk;"),
    ("swap proposals tie to the higher core",
     "if (best < 0 || t > bt) { best = k; bt = t; }", "if (best < 0 || t >= bt) { best = k; bt = t; }"),
    ("swap prefix ties to the longest",
     "if (G > 0 && G > bestG) { bestG = G; istar = i + 1; }\n        }\n        for (int32_t i = 0; i < istar; i++) {",
     "if (G > 0 && G >= bestG) { bestG = G; istar = i + 1; }\n        }\n        for (int32_t i = 0; i < istar; i++) {"),
    ("matching ignores roots without a candidate",
     "reached[n] = 1;            /* a free root */", "continue;"),
    ("folding faces the weaker child to the sibling",
     "int flip = right ? (ca > cb) : (cb > ca);", "int flip = right ? (cb > ca) : (ca > cb);"),
    ("bisection halves at the floor",
     "int32_t mid = lo[s] + (n + 1) / 2;", "int32_t mid = lo[s] + n / 2;"),
    ("bisection swaps tie to the higher node",
     "(d == bd && d > 0 && (x < ba || (x == ba && y < bb)))",
     "(d == bd && d > 0 && (x > ba || (x == ba && y > bb)))"),
    ("Hilbert quadrant not mirrored",
     "if (rx == 1) { x = s - 1 - x; y = s - 1 - y; }", "if (0) { x = s - 1 - x; y = s - 1 - y; }"),
]

BATTERY = ["tests/test_golden.py", "tests/test_gp.py", "tests/test_oracle_bruteforce.py",
           "tests/test_oracle_invariants.py", "tests/test_placement.py",
           "tests/test_initial_placement.py"]


# the pin file closest to each mutant runs first (-x stops at the first
# failure; the mutant must fail the battery either way)
FIRST = {"force without the max(., 1) term": "tests/test_placement.py",
         "swap proposals tie to the higher core": "tests/test_placement.py",
         "swap prefix ties to the longest": "tests/test_placement.py",
         "matching ignores roots without a candidate": "tests/test_placement.py",
         "folding faces the weaker child to the sibling": "tests/test_initial_placement.py",
         "bisection halves at the floor": "tests/test_initial_placement.py",
         "bisection swaps tie to the higher node": "tests/test_initial_placement.py",
         "Hilbert quadrant not mirrored": "tests/test_initial_placement.py",
         "G_P keeps self-cycles": "tests/test_gp.py",
         "G_P loses internal weight": "tests/test_gp.py"}


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(name, old, new, tmp_path):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique: {name}"
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-w", "-o", str(lib),
                           str(mut)])
    env = dict(os.environ, SNNMAP_ORACLE_LIB=str(lib))
    first = FIRST.get(name)
    battery = ([first] if first else []) + [f for f in BATTERY if f != first]
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-k", "not cfg2s", *battery], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant survived the pins: {name}"
