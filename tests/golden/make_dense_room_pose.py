"""Writes dense_room100k_pose.txt: the FP64 oracle's own solve of the dense
room pair (two ray-cast room frames, 95% of the valid pixels subsampled to
100,000 points each; Sec. 5's method on a synthetic stand-in for the paper's
RGB-D frames). Calls only synth (the seeded inputs) and oracle (the cell
search, which gives the exhaustive loop's bits). The benchmark compares its
GPU solve of the same pair with this pose; the input checksums let it tell
whether its own synth run produced the same clouds.

    python tests/golden/make_dense_room_pose.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(HERE, "dense_room100k_pose.txt")


def checksums(d):
    """Plain sums of the clouds (float64 accumulation of the float32 values)."""
    return {k: float(np.sum(d[k], dtype=np.float64)) for k in ("X", "FX", "Z", "FZ")}


def main():
    d = synth.room_pair(n_points=100000, seed=synth.seed_for(4), mode="valid")
    prm = oracle.Params(search="grid")
    t0 = time.time()
    r = oracle.align(d["X"], d["FX"], d["Z"], d["FZ"], np.eye(4), prm)
    dt = time.time() - t0
    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle solve (cell search) of the dense room pair: synth.room_pair(\n")
        fh.write("#   n_points=100000, seed=synth.seed_for(4), mode='valid'), default oracle.Params,\n")
        fh.write("#   identity start. Written by tests/golden/make_dense_room_pose.py.\n")
        for k, v in checksums(d).items():
            fh.write(f"sum_{k} {v!r}\n")
        fh.write(f"n_points {d['X'].shape[0]}\n")
        fh.write(f"iters {r['iters']}\n")
        fh.write(f"converged {int(r['converged'])}\n")
        fh.write(f"pair_evals {r['pair_evals']}\n")
        fh.write(f"oracle_seconds {dt:.1f} on {oracle.num_threads()} threads\n")
        fh.write("P " + " ".join(repr(float(v)) for v in r["P"].ravel()) + "\n")
    print(open(OUT).read())


if __name__ == "__main__":
    main()
