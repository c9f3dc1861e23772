"""Writes the oracle regression fixtures of tests/golden/ (calls only oracle/).

The paper prints no worked numeric example of its detector, so the stored
values here are the FP64 oracle's own outputs on small seeded synthetic
inputs; test_golden.py re-derives them and fails if the oracle drifts.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth   # noqa: E402


def cases():
    # (name, seed, H, W, n, tmin, tmax, thr, overlap, mode)
    return [
        ("c1_small_paper", 21, 96, 80, 10, 1.0, 10.0, 0.1, 0.5, 0),
        ("c1_small_local26", 21, 96, 80, 10, 1.0, 10.0, 0.1, 0.5, 1),
        ("c1_tiny_defocus_paper", 22, 40, 56, 4, 1.0, 4.0, 0.05, 0.5, 0),
    ]


def main():
    out = {"source": "FP64 oracle on synth 512x512-style uint8 scenes (seed, H, W given); "
                     "ladder per §2.2, DoG per Eq. 2, NMS per Eq. 3",
           "cases": []}
    for name, seed, H, W, n, tmin, tmax, thr, ov, mode in cases():
        sd = 2.0 if "defocus" in name else 0.0
        img = synth.make_scene(seed, synth.scene512_u8_spec(sd, H, W))
        r = oracle.detect(img, n, tmin, tmax, threshold=thr, overlap=ov, mode=mode)
        out["cases"].append(dict(
            name=name, seed=seed, H=H, W=W, sigma_d=sd, n=n, tmin=tmin, tmax=tmax,
            threshold=thr, overlap=ov, mode=mode, lo=r.lo, hi=r.hi,
            n_candidates=r.n_candidates, score=r.score,
            candidates=[[int(a), int(b), int(c), float(d), int(k)] for a, b, c, d, k in
                        zip(r.x, r.y, r.i, r.resp, r.keep)]))
    with open(os.path.join(HERE, "oracle_small.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
