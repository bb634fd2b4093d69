"""Plants plausible mistakes in a copy of the oracle's bands-method,
preprocessing and whitening code and checks that the pin tests catch each
one (run by hand: python tests/oracle_mutations.py; a few minutes on CPU).
Every mistake must make at least one pin fail."""
import os
import shutil
import subprocess
import sys
import tempfile

SRC = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DST = os.path.join(tempfile.gettempdir(), "oracle_mutations_repo")
muts = [
 ("bands: band boundary off by one", "while (k < 9 && rank >= ((int64_t)(k + 1) * n) / 10)", "while (k < 9 && rank > ((int64_t)(k + 1) * n) / 10)"),
 ("bands: derivative to the right sample", "D[band[i]] += fabs(d);", "D[band[i + 1]] += fabs(d);"),
 ("bands: bands in ascending D", "while (b > 0 && D[order[b - 1]] < D[v]) {", "while (b > 0 && D[order[b - 1]] > D[v]) {"),
 ("bands: window from cosines only", "S[k] = re * re + im * im;", "S[k] = re * re;"),
 ("bands: non-strict left neighbour", "int left_ok = (k == 0) || (S[k] > S[k - 1]);\n        int right_ok = (k == nk - 1) || (S[k] >= S[k + 1]);\n        if (!(left_ok && right_ok) || orc_is_one_day", "int left_ok = (k == 0) || (S[k] >= S[k - 1]);\n        int right_ok = (k == nk - 1) || (S[k] >= S[k + 1]);\n        if (!(left_ok && right_ok) || orc_is_one_day"),
 ("bands: one-day periods kept", "return f > 0.0 && fabs(1.0 / f - 1.0) < 1e-4;", "return 0;"),
 ("prep: sample standard deviation", "r.e_std = sqrt(v / (double)n);", "r.e_std = sqrt(v / (double)(n - 1));"),
 ("prep: weights 1/e", "double w = 1.0 / (e[i] * e[i]);", "double w = 1.0 / e[i];"),
 ("prep: correlation with t", "fit[i] = r.a0 + r.a1 * out_t[i];\n    r.r = orc_pearson(out_x, fit, k);", "fit[i] = r.a0 + r.a1 * out_t[i];\n    r.r = orc_pearson(out_x, out_t, k);"),
 ("prep: limit exclusive", "r.kept = k >= min_n;", "r.kept = k > min_n;"),
 ("prep: intercept kept", "out_x[i] -= fit[i];", "out_x[i] -= r.a1 * out_t[i];"),
 ("whiten: window shifted by one", "int64_t q = k - w / 2 + j;", "int64_t q = k - w / 2 + j + 1;"),
 ("whiten: window not circular", "q = ((q % n) + n) % n;", "q = q < 0 ? 0 : (q >= n ? n - 1 : q);"),
 ("whiten: phase of t times P0", "double q = t[i] / p0;", "double q = t[i] * p0;"),
]
tests = ["tests/test_oracle_bands.py", "tests/test_oracle_prep.py", "tests/test_oracle_whiten.py"]
results = []
for name, old, new in muts:
    if os.path.exists(DST):
        shutil.rmtree(DST)
    # the oracle, the input generators and the tests: all a pin needs
    for d in ('oracle', 'synth', 'tests'):
        shutil.copytree(os.path.join(SRC, d), os.path.join(DST, d),
                        ignore=shutil.ignore_patterns('*.so', '__pycache__'))
    p = os.path.join(DST, 'oracle', 'ckp_oracle.c')
    s = open(p).read()
    assert s.count(old) == 1, name
    open(p, 'w').write(s.replace(old, new))
    r = subprocess.run([sys.executable, '-m', 'pytest', '-x', '-q', '-p', 'no:cacheprovider'] + tests, cwd=DST,
                       capture_output=True, text=True, timeout=600)
    caught = r.returncode != 0
    failed = [l for l in r.stdout.splitlines() if l.startswith('FAILED')]
    results.append((name, caught, failed[:1]))
    print("%-40s %s %s" % (name, "caught" if caught else "MISSED", failed[:1]), flush=True)
print("caught %d of %d" % (sum(c for _, c, _ in results), len(results)))
sys.exit(0 if all(c for _, c, _ in results) else 1)
