"""Writes oracle_c1_regression.txt: the oracle's tracks for the single-sector event (200 tracks,
10 % noise, seed 1001) and its FP64 refit of them.  Calls only the oracle and the seeded
generator.  A change of the oracle's arithmetic that changes this file is a change of a reading
of the paper, and the commit that regenerates the file names it.

    python tests/golden/make_oracle_regression.py
"""
import hashlib
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O                       # noqa: E402
from paper_1712_09434_gb300 import synth             # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_c1_regression.txt")


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def summary(ev):
    o = O.track_event(ev.pad_fp, ev.time_fp, ev.bin_off)
    f = O.fit(ev.pad_fp, ev.time_fp, ev.bin_off, o["trk_off"], o["trk_hits"])
    return o, f


def main():
    ev = synth.make_event(synth.single_sector())
    o, f = summary(ev)
    lines = [
        "# Oracle output for the single-sector event (200 tracks, 10 % noise, seed 1001), written by",
        "# make_oracle_regression.py from the oracle alone.  Tracks: S2-S7 (section 3 of arxiv",
        "# 1712.09434, tracking by cellular automaton seeding, following and merging); fit: S8, the",
        "# FP64 Kalman refit.  Digests are SHA-256 of the little-endian int32 arrays.",
        "n_clusters %d" % ev.n_clusters,
        "n_tracks %d" % (len(o["trk_off"]) - 1),
        "n_track_hits %d" % len(o["trk_hits"]),
        "trk_off_sha256 %s" % digest(o["trk_off"].astype("<i4")),
        "trk_hits_sha256 %s" % digest(o["trk_hits"].astype("<i4")),
        "label_sha256 %s" % digest(o["label"].astype("<i4")),
        "# track <id> <n_hits> <first hit> <last hit> <ndf> <chi2> <y> <z> <sinphi> <tanlambda> <q/pT>"
        " <sigma of the five parameters>",
    ]
    for t in range(len(o["trk_off"]) - 1):
        h = o["trk_hits"][o["trk_off"][t]:o["trk_off"][t + 1]]
        p = f["par"][t]
        sig = np.sqrt(np.maximum(f["cov"][t, [0, 2, 5, 9, 14]], 0.0))
        lines.append("track %d %d %d %d %d %.10e " % (t, len(h), h[0], h[-1], f["ndf"][t], f["chi2"][t])
                     + " ".join("%.10e" % v for v in p) + " " + " ".join("%.4e" % v for v in sig))
    with open(OUT, "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
