"""The oracle's pins catch plausible mistakes (no GPU).

Each case copies ``oracle/hist_oracle.c``, plants one mistake (a dropped term,
a wrong comparison, a swapped operand, a wrong order), builds it on the CPU and
runs the pin suite ``tests/test_oracle.py`` against the mutant.  The suite must
fail for every mutant; a mutant that passes would mean a part of the oracle is
not pinned.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hist_oracle.c")

MUTANTS = [
    ("hist skips the first pixel", "for (size_t i = 0; i < n; ++i) h[x[i]] += 1;",
     "for (size_t i = 1; i < n; ++i) h[x[i]] += 1;"),
    ("hist skips the last pixel", "for (size_t i = 0; i < n; ++i) h[x[i]] += 1;",
     "for (size_t i = 0; i + 1 < n; ++i) h[x[i]] += 1;"),
    ("hist off-by-one bin", "h[x[i]] += 1;", "h[(uint8_t)(x[i] + (x[i] == 255))] += 1;"),
    ("u32 bound off by one", "if ((uint64_t)n >= ((uint64_t)1 << 32)) return -1;",
     "if ((uint64_t)n > ((uint64_t)1 << 32)) return -1;"),
    ("argmax keeps the last tie", "if (h[b] > m) {", "if (h[b] >= m) {"),
    ("total counts bins", "t += h[b];", "t += (h[b] != 0);"),
    ("switch strict", "return lhs >= rhs ?", "return lhs > rhs ?"),
    ("switch on empty", "if (t == 0) return ORACLE_FLAG_PLAIN;", "if (t == 0) return ORACLE_FLAG_ADAPTIVE;"),
    ("switch operands swapped", "unsigned __int128 lhs = (unsigned __int128)m * 1000u;",
     "unsigned __int128 lhs = (unsigned __int128)t * 1000u;"),
    ("switch in 64 bits", "unsigned __int128 lhs = (unsigned __int128)m * 1000u;",
     "unsigned __int128 lhs = (uint64_t)(m * 1000u);"),
    ("want drops the +1", "uint64_t want = 1 + (spare * (uint64_t)h[b]) / total;",
     "uint64_t want = (spare * (uint64_t)h[b]) / total; if (want == 0) want = 1;"),
    ("spare is the whole budget", "uint64_t spare = budget - ORACLE_BINS;", "uint64_t spare = budget;"),
    ("cap at 16", "k[b] = kk > ORACLE_KMAX ? ORACLE_KMAX : kk;", "k[b] = kk > 16 ? 16 : kk;"),
    ("floor strict", "if (sum <= budget) floor_k = f;", "if (sum < budget) floor_k = f;"),
    ("no floor", "if (sum <= budget) floor_k = f;", "if (sum <= budget) floor_k = 1;"),
    ("floor ignores proportional k", "sum += k[b] > f ? k[b] : f;", "sum += f;"),
    ("layout smallest first", "for (int lk = 5; lk >= 0; --lk) {", "for (int lk = 0; lk <= 5; ++lk) {"),
    ("layout ties by descending bin", "for (int b = 0; b < ORACLE_BINS; ++b) {\n      if (log2k[b] == lk) {",
     "for (int b = ORACLE_BINS - 1; b >= 0; --b) {\n      if (log2k[b] == lk) {"),
    ("default regions mirrored wrong", "{1, 2, 4, 8, 8, 4, 2, 1}", "{1, 2, 4, 8, 4, 8, 2, 1}"),
    ("default threshold strict", "if (budget >= 960) scale = 1u << log2_floor_u64(budget / 960);",
     "if (budget > 960) scale = 1u << log2_floor_u64(budget / 960);"),
    ("default scale from the wrong base", "if (budget >= 960) scale = 1u << log2_floor_u64(budget / 960);",
     "if (budget >= 960) scale = 1u << log2_floor_u64(budget / 480);"),
    ("empty history not default", "if (total == 0) return oracle_default_pattern(budget, p);",
     "if (total == 0) total = 1;"),
    ("budget range", "if (budget < ORACLE_BUDGET_MIN || budget > ORACLE_BUDGET_MAX) return -1;\n  uint64_t total",
     "if (budget < ORACLE_BUDGET_MIN) return -1;\n  uint64_t total"),
    ("regime run start rounds up", "uint64_t start = (t * (uint64_t)n) / 256;",
     "uint64_t start = (t * (uint64_t)n + 255) / 256;"),
    ("regime runs of 8", "for (uint64_t u = 0; u < 16; ++u) h[x[start + u]] += 1;",
     "for (uint64_t u = 0; u < 8; ++u) h[x[start + u]] += 2;"),
    ("regime runs spaced by 4096 / n", "uint64_t start = (t * (uint64_t)n) / 256;",
     "uint64_t start = t * 16;"),
    ("regime whole image up to 4097", "if (n <= ORACLE_REGIME_SAMPLE) {", "if (n <= ORACLE_REGIME_SAMPLE + 1) {"),
    ("regime sample of 2048", "uint64_t m = n < ORACLE_REGIME_SAMPLE ? (uint64_t)n : ORACLE_REGIME_SAMPLE;",
     "uint64_t m = n < 2048 ? (uint64_t)n : 2048;"),
    ("regime degeneracy strict", "if (mx * 1000u >= (uint64_t)theta_milli * m)", "if (mx * 1000u > (uint64_t)theta_milli * m)"),
    ("regime peaked strict", "if (64u * sq >= m * m)", "if (64u * sq > m * m)"),
    ("regime 32 effective bins", "if (64u * sq >= m * m)", "if (32u * sq >= m * m)"),
    ("regime squares dropped", "sq += h[b] * h[b];", "sq += h[b];"),
    ("regime empty is degenerate", "if (n == 0) return ORACLE_REGIME_WIDE;", "if (n == 0) return ORACLE_REGIME_DEGENERATE;"),
]


@pytest.mark.slow
@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation anchor not found: %r" % old
    shutil.copy(os.path.join(ROOT, "oracle", "oracle.h"), tmp_path / "oracle.h")
    (tmp_path / "hist_oracle.c").write_text(src.replace(old, new, 1))
    so = str(tmp_path / "liboracle_mutant.so")
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-shared", "-fPIC", str(tmp_path / "hist_oracle.c"), "-o", so])
    env = dict(os.environ, HIST_ORACLE_SO=so)
    r = subprocess.run(
        [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", os.path.join(ROOT, "tests", "test_oracle.py")],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=600,
    )
    assert r.returncode != 0, "pins did not catch mutant %r:\n%s" % (name, r.stdout[-2000:])
