"""Write the oracle's label digest of a whole workload (test infrastructure).

The FP64 CPU oracle labels every point of the workload (Sec. 2.1.3, Eq. 1:
inside when Omega > 2 pi; Sec. 2.1: the first compartment of the priority
list wins) in chunks of consecutive points, and the digest keeps, per chunk,
a SHA-256 prefix of the chunk's int32 labels (little-endian) plus the label
counts of the whole workload.  The GPU test `test_gpu_digest.py` hashes its
own labels the same way and compares chunk by chunk; a chunk that differs is
recomputed with the oracle to name the points.

Only `oracle/` and the seeded input generators (`zef_synth`) are called.  The
run takes about 6e11 FP64 point x triangle pairs for the 5 M-point head, so
every chunk is cached as it finishes (`--cache`, default a directory under the
system temp dir) and a rerun resumes from the cached chunks.

The oracle's decision is ill-posed for a point on a surface; the digest also
records the smallest |Omega - 2 pi| seen over every (point, compartment)
pair, which must stay well above the FP64 rounding of the sum (1e-9).

    python tests/golden/make_label_digest.py --config 1
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

CHUNK = 65536


def chunk_hash(labels: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(labels, dtype="<i4").tobytes()).hexdigest()[:16]


def workload(cfg: int):
    import zef_synth as zs
    return zs.make_config(cfg)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", type=int, default=1)
    ap.add_argument("--chunk", type=int, default=CHUNK)
    ap.add_argument("--cache", default=os.path.join(tempfile.gettempdir(), "zef_oracle_cache"))
    ap.add_argument("--out", default="")
    args = ap.parse_args()

    import oracle
    oracle.build()
    w = workload(args.config)
    pts = w.points
    n = int(pts.shape[0])
    nchunks = (n + args.chunk - 1) // args.chunk
    src = open(os.path.join(ROOT, "oracle", "oracle.c"), "rb").read()
    oracle_sha = hashlib.sha256(src).hexdigest()[:16]
    geo = hashlib.sha256()
    for s in w.surfaces:
        geo.update(np.ascontiguousarray(s.verts, dtype="<f4").tobytes())
        geo.update(np.ascontiguousarray(s.tris, dtype="<i4").tobytes())
    geo.update(np.ascontiguousarray(pts, dtype="<f4").tobytes())
    key = f"config{args.config}_{geo.hexdigest()[:16]}_{oracle_sha}_{args.chunk}"
    cdir = os.path.join(args.cache, key)
    os.makedirs(cdir, exist_ok=True)

    hashes, min_margin = [], np.inf
    counts: dict[int, int] = {}
    t0 = time.time()
    for k in range(nchunks):
        path = os.path.join(cdir, f"chunk_{k:05d}.npz")
        if os.path.exists(path):
            z = np.load(path)
            lab, mm = z["labels"], float(z["min_margin"])
        else:
            p = pts[k * args.chunk:(k + 1) * args.chunk]
            lab, om = oracle.label_points(p, w.surfaces, w.priority)
            fin = np.isfinite(om)
            mm = float(np.min(np.abs(om[fin] - oracle.TWO_PI))) if fin.any() else np.inf
            tmp = path + ".tmp.npz"
            np.savez(tmp, labels=lab, min_margin=mm)
            os.replace(tmp, path)
            el = time.time() - t0
            print(f"chunk {k + 1}/{nchunks} {el:.0f} s", flush=True)
        hashes.append(chunk_hash(lab))
        min_margin = min(min_margin, mm)
        for v, c in zip(*np.unique(lab, return_counts=True)):
            counts[int(v)] = counts.get(int(v), 0) + int(c)

    out = {
        "workload": w.name,
        "config": args.config,
        "points": n,
        "triangles": w.total_tris,
        "priority": [int(i) for i in w.priority],
        "chunk": args.chunk,
        "hash": "sha256 of the chunk's labels as little-endian int32, first 16 hex digits",
        "inputs_sha256_prefix": geo.hexdigest()[:16],
        "oracle_c_sha256_prefix": oracle_sha,
        "min_abs_omega_minus_2pi": min_margin,
        "label_counts": {str(k): v for k, v in sorted(counts.items())},
        "chunk_hashes": hashes,
        "written_by": "tests/golden/make_label_digest.py (FP64 CPU oracle only)",
    }
    dest = args.out or os.path.join(HERE, f"config{args.config}_label_digest.json")
    with open(dest, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(f"wrote {dest}: {n} points, {nchunks} chunks, min |Omega - 2 pi| = {min_margin:.3e}")


if __name__ == "__main__":
    main()
