"""Autotuner of the fused kernel's tile configuration.

The fused detection kernel is specialised per ladder and per tile shape
(strip width and tile height including the 1-pixel NMS border, rows per
step, threads per block, level groups).  The built-in heuristic picks a shape from a cost
model; this module measures instead: it compiles a filtered menu of shapes in
parallel (NVRTC, CPU processes), times each one's fused kernel with CUDA
events on a synthetic tile of the workload, and records the winner per
(ladder, mode, SM count) in a JSON table that ``Detector`` consults.

    python -m paper_2108_12050_gb300.tune --n 16 --tmin 1 --tmax 12 --side 4096
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import multiprocessing as mp
import os
import statistics
import sys
import time

PKG = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(PKG, "tuned_tiles.json")


def ladder_key(n, t_min, t_max, nms, truncate=4.0, response="dog", tensor_cores=False):
    key = "n%d_t%g-%g_%s_tr%g" % (n, t_min, t_max,
                                  "paper" if nms in (0, "paper") else "local26", truncate)
    if response not in ("dog", 0):
        key += "_log"
    return key + "_tc" if tensor_cores else key


def load_table():
    try:
        with open(TABLE) as f:
            return json.load(f)
    except Exception:
        return {}


def lookup(n, t_min, t_max, nms, sms, truncate=4.0, response="dog", tensor_cores=False):
    """Tuned tile shape (the six-field tile_shape of the parameters; a five-field
    entry means one row per horizontal item) for this
    ladder, response, kernel kind and SM count, or None (the built-in choice
    is used)."""
    ent = load_table().get(ladder_key(n, t_min, t_max, nms, truncate, response, tensor_cores))
    if not ent:
        return None
    best = ent.get(str(sms)) or ent.get("any")
    if not best:
        return None
    shape = best.get("shape")
    if not shape or len(shape) not in (5, 6):
        return None
    return [int(v) for v in shape] + ([1] if len(shape) == 5 else [])


def item_count(tx2, rb, item):
    """Horizontal items of one step: kind 1 is one row of four outputs, 2 two
    rows of four, 3 one row of two."""
    rows, cols = (2, 4) if item == 2 else (1, 2) if item == 3 else (1, 4)
    return (rb // rows) * (tx2 // cols)


def _rmax(n, t_min, t_max, truncate=4.0):
    import math
    dt = (t_max - t_min) / n
    return max(int(math.ceil(truncate * (t_min + i * dt))) for i in range(n + 1))


def candidates(n, t_min, t_max, nms, limit=None, min_width=0, response="dog"):
    """Balanced shapes of the FFMA kernel's built-in menu: every horizontal
    item has a thread and the vertical pass keeps most threads busy."""
    from . import _native
    menu = _native.tile_configs(n=n, t_min=t_min, t_max=t_max, nms=nms, response=response,
                                tensor_cores=False)
    rmax = _rmax(n, t_min, t_max) + (0 if response in ("dog", 0) else 1)
    seen, out = set(), []
    for (tx2, ty2, rb, nt, ng, item) in menu:
        if tx2 < min_width:
            continue
        wext = tx2 + 2 * rmax
        hitems = item_count(tx2, rb, item)
        if hitems > nt or hitems < 0.85 * nt:
            continue
        vutil = wext / (nt * -(-wext // nt))
        if vutil < 0.75:
            continue
        key = (tx2, ty2, rb, nt, ng, item)
        if key in seen:
            continue
        seen.add(key)
        out.append(key)
    return out[:limit] if limit else out


def width_candidates(n, t_min, t_max, nms, widths, rbs=(2, 3, 4, 5, 6, 8), groups=(2, 3, 4, 5),
                     response="dog", items=(1,)):
    """FFMA-kernel shapes off the menu's width grid (strip widths fitted to
    an image width).  Thread counts: at least one per horizontal item and one per
    halo'd column of the vertical pass (a single round), that count plus one
    warp, and rounded up to whole groups of four warps (the four schedulers
    of an SM); keeps those that fit in shared memory."""
    from . import _native
    rmax = _rmax(n, t_min, t_max) + (0 if response in ("dog", 0) else 1)
    out = []
    for tx2, rb, item in [(w, r, k) for w in widths for r in rbs for k in items
                          if k != 2 or r % 2 == 0]:
        ncol = -(-(tx2 + 2 * rmax) // 32) * 32
        if True:
            hitems = item_count(tx2, rb, item)
            base = max(-(-hitems // 32) * 32, ncol)
            for nt in sorted({base, base + 32, -(-base // 128) * 128}):
                if nt > 1024:
                    continue
                for ng in groups:
                    shape = (tx2, 18, rb, nt, ng, item)
                    try:
                        _native.chosen_tile(n=n, t_min=t_min, t_max=t_max, nms=nms,
                                            tile_shape=shape, response=response,
                                            tensor_cores=False)
                    except Exception:
                        continue
                    out.append(shape)
    return out


def _compile_one(args):
    n, t_min, t_max, nms, shape, response, tc = args
    sys.path.insert(0, os.path.dirname(PKG))
    from paper_2108_12050_gb300 import _native
    t0 = time.time()
    try:
        # the tuned tensor-core shapes are the vertical-pass kernel's (2)
        _native.precompile(n=n, t_min=t_min, t_max=t_max, nms=nms, tile_shape=shape,
                           response=response, tensor_cores=2 if tc else False)
        return shape, time.time() - t0, None
    except Exception as e:  # a shape the compiler rejects is skipped
        return shape, time.time() - t0, str(e)


def precompile_all(n, t_min, t_max, nms, cands, workers=None, response="dog",
                   tensor_cores=False):
    ctx = mp.get_context("spawn")
    workers = workers or (os.cpu_count() or 4)
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
        return list(ex.map(_compile_one, [(n, t_min, t_max, nms, c, response, tensor_cores)
                                          for c in cands]))


def measure(n, t_min, t_max, nms, threshold, img_dev, cands, reps=5, response="dog",
            tensor_cores=False):
    import paper_2108_12050_gb300 as mhfd
    res = []
    for shape in cands:
        try:
            det = mhfd.Detector(n, t_min, t_max, threshold=threshold, nms=nms, tile_shape=shape,
                                timing=True, response=response,
                                tensor_cores=2 if tensor_cores else False)
        except Exception as e:
            res.append((shape, None, str(e)))
            continue
        det(img_dev)
        ks = []
        for _ in range(reps):
            det(img_dev)
            ks.append(det.last_timing()[0])
        det.close()
        res.append((shape, statistics.median(ks), None))
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=16)
    ap.add_argument("--tmin", type=float, default=1.0)
    ap.add_argument("--tmax", type=float, default=12.0)
    ap.add_argument("--nms", default="paper")
    ap.add_argument("--threshold", type=float, default=0.05)
    ap.add_argument("--side", type=int, default=4096)
    ap.add_argument("--limit", type=int, default=0)
    ap.add_argument("--min-width", type=int, default=0, help="skip strips narrower than this")
    ap.add_argument("--widths", default="", help="extra strip widths off the menu, e.g. 312,344")
    ap.add_argument("--rbs", default="2,3,4,5,6,8", help="rows per step of the extra shapes")
    ap.add_argument("--groups", default="2,3,4,5", help="level groups of the extra shapes")
    ap.add_argument("--items", default="1",
                    help="horizontal item kinds of the extra shapes (1: 1x4, 2: 2x4, 3: 1x2)")
    ap.add_argument("--response", default="dog", choices=["dog", "log"])
    ap.add_argument("--tensor-cores", action="store_true",
                    help="tune the tensor-core kernel (its own shape menu)")
    ap.add_argument("--heights", default="",
                    help="tile heights (incl. the 2 border rows) to try for every candidate, "
                         "e.g. 10,14,18: the tiles of an image are split evenly over the "
                         "resident blocks, so the height sets how evenly")
    ap.add_argument("--write", action="store_true", help="record the winner in tuned_tiles.json")
    args = ap.parse_args()
    nms = 0 if args.nms == "paper" else 1
    if args.tensor_cores:
        from . import _native
        cands = [c for c in _native.tile_configs(n=args.n, t_min=args.tmin, t_max=args.tmax,
                                                 nms=nms, response=args.response,
                                                 tensor_cores=True)
                 if c[0] >= args.min_width]
        if args.limit:
            cands = cands[:args.limit]
    else:
        cands = candidates(args.n, args.tmin, args.tmax, nms, args.limit or None,
                           args.min_width, args.response)
    if args.widths and not args.tensor_cores:
        extra = width_candidates(args.n, args.tmin, args.tmax, nms,
                                 [int(w) for w in args.widths.split(",")],
                                 rbs=[int(v) for v in args.rbs.split(",")],
                                 groups=[int(v) for v in args.groups.split(",")],
                                 response=args.response,
                                 items=[int(v) for v in args.items.split(",")])
        cands += [c for c in extra if c not in cands]
    if args.heights:
        hs = [int(v) for v in args.heights.split(",")]
        cands = list(dict.fromkeys(tuple(c[:1]) + (h,) + tuple(c[2:]) for c in cands for h in hs))
    t0 = time.time()
    comp = precompile_all(args.n, args.tmin, args.tmax, nms, cands, response=args.response,
                          tensor_cores=args.tensor_cores)
    print("compiled %d shapes in %.1f s" % (len(comp), time.time() - t0), flush=True)
    bad = {tuple(c) for c, _, e in comp if e}
    cands = [c for c in cands if tuple(c) not in bad]

    import numpy as np
    import torch
    sys.path.insert(0, os.path.dirname(PKG))
    import synth
    img = synth.sweep_tile_4096_u16(0.0)[:args.side, :args.side].copy()
    dev = torch.from_numpy(img.view(np.int16)).cuda()
    res = measure(args.n, args.tmin, args.tmax, nms, args.threshold, dev, cands,
                  response=args.response, tensor_cores=args.tensor_cores)
    res.sort(key=lambda r: (r[1] is None, r[1] or 0))
    for shape, ms, err in res:
        print("%-28s %s" % (shape, ("%.3f ms" % ms) if ms else err), flush=True)
    best = res[0]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    print("best", best, "SMs", sms)
    if args.write and best[1]:
        tab = load_table()
        ent = tab.setdefault(ladder_key(args.n, args.tmin, args.tmax, nms,
                                        response=args.response,
                                        tensor_cores=args.tensor_cores), {})
        ent[str(sms)] = {"shape": list(best[0]), "ms": best[1], "side": args.side}
        with open(TABLE, "w") as f:
            json.dump(tab, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
