"""Plants plausible mistakes in a copy of the oracle -- the statistic and its
kernels, the order statistics, the sigma_t rule, the thresholds, the searches,
the bands method, preprocessing and whitening -- and checks that the pin tests
catch each one (run by hand: python tests/oracle_mutations.py; some minutes on
CPU).  Every mistake must make at least one pin fail."""
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
 ("whiten batch: output of later curves shifted", "orc_whiten(times + a, x, n, p0[c], w, out + a);",
  "orc_whiten(times + a, x, n, p0[c], w, out + (c > 0 ? a - 1 : a));"),
 ("whiten batch: period guard inverted", "if (p0[c] > 0.0 && isfinite(p0[c]))", "if (!(p0[c] > 0.0 && isfinite(p0[c])))"),
 ("whiten batch: zero period whitened", "if (p0[c] > 0.0 && isfinite(p0[c]))", "if (p0[c] >= 0.0 && isfinite(p0[c]))"),
 ("whiten batch: infinite period whitened", "if (p0[c] > 0.0 && isfinite(p0[c]))", "if (p0[c] > 0.0 && !isnan(p0[c]))"),
]
core = [
 ("gauss: 2 sigma^2 -> sigma^2", "return exp(-(x * x) / (2.0 * sigma * sigma)) / (sqrt(2.0 * ORC_PI) * sigma);",
  "return exp(-(x * x) / (sigma * sigma)) / (sqrt(2.0 * ORC_PI) * sigma);"),
 ("gauss: normalisation sqrt(2 pi sigma)", "return exp(-(x * x) / (2.0 * sigma * sigma)) / (sqrt(2.0 * ORC_PI) * sigma);",
  "return exp(-(x * x) / (2.0 * sigma * sigma)) / sqrt(2.0 * ORC_PI * sigma);"),
 ("periodic kernel: sin(2 pi f dt)", "double s = sin(ORC_PI * f * dt);", "double s = sin(2.0 * ORC_PI * f * dt);"),
 ("periodic kernel: factor 2 dropped", "return exp(-2.0 * s * s / (sigma * sigma))", "return exp(-s * s / (sigma * sigma))"),
 ("IP: divided by N", "    return acc / ((double)n * (double)n);\n}\n\n/* Eq. (HP)", "    return acc / (double)n;\n}\n\n/* Eq. (HP)"),
 ("CKP: upper triangle only", "            for (int64_t j = 0; j < n; j++)\n                acc += (orc_gauss(y[i] - y[j]",
  "            for (int64_t j = i + 1; j < n; j++)\n                acc += (orc_gauss(y[i] - y[j]"),
 ("batch CKP: upper triangle only", "            for (int64_t j = 0; j < n; j++)\n                acc += (orc_gauss((double)mags",
  "            for (int64_t j = i + 1; j < n; j++)\n                acc += (orc_gauss((double)mags"),
 ("CKP: + IP", "sigma_y) - ip) *", "sigma_y) + ip) *"),
 ("nCKP: sqrt(N / sigma_t)", "sqrt((double)n * sigma_t) / ip", "sqrt((double)n / sigma_t) / ip"),
 ("median: upper middle value", "return 0.5 * (s[n / 2 - 1] + s[n / 2]);", "return s[n / 2];"),
 ("quantile: position q N", "double pos = q * (double)(n - 1);", "double pos = q * (double)n;"),
 ("pSNR: alpha dropped", "return 0.7413 * iqr / (alpha * orc_median(e, n));", "return 0.7413 * iqr / orc_median(e, n);"),
 ("Bowley: q3 - q1 in the numerator", "return (q3 + q1 - 2.0 * q2) / (q3 - q1);", "return (q3 - q1 - 2.0 * q2) / (q3 - q1);"),
 ("sigma_t rule: S instead of S^2", "return 0.1 + 0.5 * exp(-12.0 * sk * sk);", "return 0.1 + 0.5 * exp(-12.0 * sk);"),
 ("thresholds: bins right-closed", "if (psnr >= ORC_BIN_LO[k])", "if (psnr > ORC_BIN_LO[k])"),
 ("thresholds: digits swapped", "1.1153", "1.1513"),
 ("argmax: ties to the highest index", "if (v[k] > v[b])", "if (v[k] >= v[b])"),
 ("coarse maxima: non-strict left neighbour",
  "int left_ok = (k == 0) || (v[k] > v[k - 1]);\n        int right_ok = (k == n - 1) || (v[k] >= v[k + 1]);\n        if (n == 1)\n            left_ok = right_ok = 1;\n        if (!(left_ok && right_ok))\n",
  "int left_ok = (k == 0) || (v[k] >= v[k - 1]);\n        int right_ok = (k == n - 1) || (v[k] >= v[k + 1]);\n        if (n == 1)\n            left_ok = right_ok = 1;\n        if (!(left_ok && right_ok))\n"),
 ("coarse maxima with windows: non-strict left neighbour",
  "int left_ok = (k == 0) || (v[k] > v[k - 1]);\n        int right_ok = (k == n - 1) || (v[k] >= v[k + 1]);\n        if (n == 1)\n            left_ok = right_ok = 1;\n        if (!(left_ok && right_ok) || orc_is_excluded",
  "int left_ok = (k == 0) || (v[k] >= v[k - 1]);\n        int right_ok = (k == n - 1) || (v[k] >= v[k + 1]);\n        if (n == 1)\n            left_ok = right_ok = 1;\n        if (!(left_ok && right_ok) || orc_is_excluded"),
 ("fine window: half-width in coarse steps", "floor(g->fine_halfwidth / g->fine_df + 0.5)", "floor(g->fine_halfwidth / g->coarse_df + 0.5)"),
 ("sigma_y: largest error bar", "    double sy = orc_median(e, n);\n    double st = curve_sigma_t(o, y, n, c);",
  "    double sy = orc_quantile(e, n, 1.0);\n    double st = curve_sigma_t(o, y, n, c);"),
 ("discriminator: flipped", "r->is_periodic = r->best_stat > orc_threshold(r->psnr);", "r->is_periodic = r->best_stat < orc_threshold(r->psnr);"),
 ("exclusion: open intervals", "if (f >= exclude[2 * q] && f <= exclude[2 * q + 1])", "if (f > exclude[2 * q] && f < exclude[2 * q + 1])"),
 ("exclusion: coarse peaks unfiltered", "if (!(left_ok && right_ok) || orc_is_excluded(f_min + (double)k * df, n_exclude, exclude))",
  "if (!(left_ok && right_ok))"),
 ("exclusion: fine candidates unfiltered", "if (f < g->f_min || f > f_max || orc_is_excluded(f, g->n_exclude, g->exclude))",
  "if (f < g->f_min || f > f_max)"),
 ("exclusion: trial choice unfiltered", "int64_t b = argmax_allowed(v, fr, m, g);", "int64_t b = m > 0 ? orc_argmax(v, m) : -1;"),
 ("exclusion: full-grid choice unfiltered", "int64_t b = argmax_allowed(v, fr, g->n_freq, g);", "int64_t b = orc_argmax(v, g->n_freq);"),
]
tests = ["tests/test_oracle_bands.py", "tests/test_oracle_prep.py", "tests/test_oracle_whiten.py"]
core_tests = ["tests/test_oracle_pins.py", "tests/test_oracle_exclusion.py"]
results = []
only = sys.argv[1:]            # optional name prefixes: run just those mutations
for name, old, new, tfiles in [m + (core_tests,) for m in core] + [m + (tests,) for m in muts]:
    if only and not any(name.startswith(o) for o in only):
        continue
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
    r = subprocess.run([sys.executable, '-m', 'pytest', '-x', '-q', '-p', 'no:cacheprovider'] + tfiles, cwd=DST,
                       capture_output=True, text=True, timeout=600)
    caught = r.returncode != 0
    failed = [l for l in r.stdout.splitlines() if l.startswith('FAILED')]
    results.append((name, caught, failed[:1]))
    print("%-40s %s %s" % (name, "caught" if caught else "MISSED", failed[:1]), flush=True)
print("caught %d of %d" % (sum(c for _, c, _ in results), len(results)))
sys.exit(0 if all(c for _, c, _ in results) else 1)
