"""Writes `throughput_agreement_oracle.txt`: the oracle's best period, best
nCKP and periodic / non-periodic label for a fixed 1,000-curve sample of the
two-band throughput generator (500 sources, seed 5), searched coarse-then-fine
(coarse step 1e-3 over 0.002-5 1/d, the 10 highest local maxima refined at
step 1e-5 over +-2e-3) with sigma_t from the skewness rule.

Only `oracle/` computes the values; `synth/` supplies the inputs.  The oracle
takes hours for the whole sample, so the script works in chunks of curves and
appends each finished chunk to the file: run it again to continue.  Within a
chunk the curves go to the oracle largest first, so its threads finish
together.

    python tests/golden/make_throughput_agreement.py [--chunk 64]
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(HERE, "throughput_agreement_oracle.txt")
N_SOURCES, SEED = 500, 5


def sample():
    return synth.workload_throughput(N_SOURCES, SEED)


def input_checksum(batch) -> str:
    """Sums that change if the generator's output changes."""
    return "%.17g %.17g %.17g %d" % (float(np.sum(batch.times)), float(np.sum(batch.mags.astype(np.float64))),
                                     float(np.sum(batch.errs.astype(np.float64))), int(batch.offsets[-1]))


def done_curves(path: str) -> set:
    if not os.path.exists(path):
        return set()
    with open(path) as fh:
        return {int(line.split()[0]) for line in fh if line.strip() and not line.startswith("#")}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--chunk", type=int, default=64)
    args = ap.parse_args()
    b, g = sample()
    if not os.path.exists(OUT):
        with open(OUT, "w") as fh:
            fh.write("# Oracle (FP64) best period of a fixed 1,000-curve sample of the two-band throughput\n"
                     "# generator: synth.workload_throughput(%d, %d); coarse-then-fine search (coarse step 1e-3\n"
                     "# over 0.002-5 1/d, top 10 local maxima refined at 1e-5 over +-2e-3); sigma_t from the\n"
                     "# skewness rule (Section 3). nCKP is Eq. (CKP); the label thresholds it by Table \"tab:th\".\n"
                     "# Written by tests/golden/make_throughput_agreement.py, which runs only oracle/.\n"
                     "# inputs: %s\n"
                     "# curve n best_idx best_freq best_nckp is_periodic sigma_t psnr\n"
                     % (N_SOURCES, SEED, input_checksum(b)))
    else:
        with open(OUT) as fh:
            head = [ln for ln in fh if ln.startswith("# inputs:")]
        if not head or head[0].split(":", 1)[1].strip() != input_checksum(b):
            sys.exit("the generator's output differs from the one the file was written for")
    todo = [c for c in range(b.n_curves) if c not in done_curves(OUT)]
    sizes = b.sizes
    print("%d curves, %d left" % (b.n_curves, len(todo)), flush=True)
    while todo:
        chunk = todo[:args.chunk]
        todo = todo[args.chunk:]
        order = sorted(chunk, key=lambda c: -int(sizes[c]))
        t0 = time.time()
        r = oracle.batch_best(b.subset(order), g, sigma_t_mode=2)
        with open(OUT, "a") as fh:
            for k, c in sorted(enumerate(order), key=lambda kc: kc[1]):
                fh.write("%d %d %d %.17g %.17g %d %.17g %.17g\n" % (
                    c, int(sizes[c]), int(r["best_idx"][k]), float(r["best_freq"][k]), float(r["best_stat"][k]),
                    int(r["is_periodic"][k]), float(r["sigma_t"][k]), float(r["psnr"][k])))
        print("curves %d-%d done in %.0f s; %d left" % (min(chunk), max(chunk), time.time() - t0, len(todo)),
              flush=True)


if __name__ == "__main__":
    main()
