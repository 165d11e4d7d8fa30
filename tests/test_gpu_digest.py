"""Every label of the three-layer head workload against the FP64 oracle.

All 5,000,000 tet centroids of the 2 mm lattice (the three nested perturbed
ellipsoids, 122,880 triangles) are labelled on the GPU through the C ABI and
compared chunk by chunk with the digest of the oracle's labels of the same
points (`tests/golden/config1_label_digest.json`, written by
`tests/golden/make_label_digest.py`, which calls only the oracle): per chunk of
65,536 consecutive points a SHA-256 prefix of the int32 labels, plus the label
counts.  A chunk whose hash differs is recomputed with the oracle, which
names the differing points.  Bar: bit-exact, every point, in the launch the
benchmark times (no Omega: priority early exit and tile coherence on) and
with coherence off and in the strip kernel form.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import zef_synth as zs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DIGEST = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config1_label_digest.json")


@pytest.fixture(scope="module")
def zef():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_10000_gb300 import build
    build.build()
    from paper_2203_10000_gb300 import zef as z
    return z


@pytest.fixture(scope="module")
def head():
    d = json.load(open(DIGEST))
    w = zs.config1()
    geo = hashlib.sha256()
    for s in w.surfaces:
        geo.update(np.ascontiguousarray(s.verts, dtype="<f4").tobytes())
        geo.update(np.ascontiguousarray(s.tris, dtype="<i4").tobytes())
    geo.update(np.ascontiguousarray(w.points, dtype="<f4").tobytes())
    # the digest was written for exactly these inputs
    assert geo.hexdigest()[:16] == d["inputs_sha256_prefix"]
    assert d["points"] == w.points.shape[0] and d["priority"] == list(w.priority)
    # no point sits on a surface, where the decision itself is ill-posed
    assert d["min_abs_omega_minus_2pi"] > 1e-9
    return w, d


def _chunk_hash(lab):
    return hashlib.sha256(np.ascontiguousarray(lab, dtype="<i4").tobytes()).hexdigest()[:16]


@pytest.mark.parametrize("variant", ["default", "no_coherence", "strip_kernel"])
def test_config1_every_label_equals_oracle_digest(zef, oracle_mod, head, variant):
    w, d = head
    opts = {"default": zef.make_opts(), "no_coherence": zef.make_opts(coherence=False),
            "strip_kernel": zef.make_opts(kernel=1)}[variant]
    ctx = zef.Context(0)
    for s in w.surfaces:
        ctx.add_compartment(s.id, s.verts, s.tris)
    ctx.set_priority(w.priority)
    lab, _, st = ctx.label_points(torch.from_numpy(w.points).cuda(), opts=opts)
    torch.cuda.synchronize()
    lab = lab.cpu().numpy()
    ctx.close()
    chunk = d["chunk"]
    nchunks = len(d["chunk_hashes"])
    assert nchunks == (lab.size + chunk - 1) // chunk
    bad = [k for k in range(nchunks) if _chunk_hash(lab[k * chunk:(k + 1) * chunk]) != d["chunk_hashes"][k]]
    if bad:
        # name the differing points of the first two differing chunks
        msgs = []
        for k in bad[:2]:
            sl = slice(k * chunk, (k + 1) * chunk)
            olab, _ = oracle_mod.label_points(w.points[sl], w.surfaces, w.priority)
            diff = np.nonzero(lab[sl] != olab)[0] + k * chunk
            msgs.append(f"chunk {k}: points {diff[:10].tolist()} gpu {lab[diff[:10]].tolist()} "
                        f"oracle {olab[diff[:10] - k * chunk].tolist()}")
        pytest.fail(f"{len(bad)} of {nchunks} chunks differ from the oracle digest; " + "; ".join(msgs))
    got = {str(int(v)): int(c) for v, c in zip(*np.unique(lab, return_counts=True))}
    assert got == d["label_counts"]
    print(f"{variant}: all {lab.size} labels equal the oracle's ({nchunks} chunks), "
          f"{st['pairs_evaluated']:.3e} pairs evaluated, {st['uncertain_pairs']} re-evaluated in FP64")
