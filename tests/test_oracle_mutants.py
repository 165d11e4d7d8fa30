"""Planted mistakes in the oracle must be caught by its pins.

Each case copies oracle.c, changes one expression the way a plausible slip
would (a dropped term, a wrong index, a flipped sign, transposed operands),
compiles the copy on the CPU and checks that the closed-form / L'Huilier /
unit-sphere pins reject it.  The committed oracle is never modified.
"""
import ctypes
import json
import math
import os
import subprocess

import numpy as np
import pytest

import zef_synth as zs
from test_oracle_pins import lhuilier

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "drop_d23_term": ("+ d23 * r1;", ";"),
    "wrong_radius_index": ("d13 * r2", "d13 * r3"),
    "missing_factor_two": ("return 2.0 * atan2(N, D);", "return atan2(N, D);"),
    "wrong_vector_in_triple": ("R1[0] * cx", "R2[0] * cx"),
    "cross_sign_flip": ("R2[1] * R3[2] - R2[2] * R3[1]", "R2[2] * R3[1] - R2[1] * R3[2]"),
    "atan2_transposed": ("return 2.0 * atan2(N, D);", "return 2.0 * atan2(D, N);"),
    "dropped_radius_factor": ("r1 * r2 * r3", "r1 * r2"),
}


def _build_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    mutated = src.replace(old, new, 1)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(mutated)
    subprocess.run(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                    "-o", str(so), str(c), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    P, I64 = ctypes.c_void_p, ctypes.c_int64
    lib.oracle_triangle_terms.argtypes = [P, P, I64, P, I64, P]
    lib.oracle_omega.argtypes = [P, I64, P, I64, P, I64, P, ctypes.c_int]
    return lib


def _terms(lib, p, v, t):
    p = np.ascontiguousarray(p, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.int32)
    out = np.empty(t.shape[0])
    lib.oracle_triangle_terms(p.ctypes.data, v.ctypes.data, v.shape[0], t.ctypes.data,
                              t.shape[0], out.ctypes.data)
    return out


def _pins_pass(lib):
    cases = json.load(open(os.path.join(ROOT, "tests", "golden", "closed_forms.json")))["cases"]
    for c in cases:
        if abs(_terms(lib, c["point"], c["verts"], c["tris"]).sum() - c["expected_total"]) > 1e-9:
            return False
    rng = np.random.default_rng(7)
    for _ in range(50):
        tri = rng.uniform(-1, 1, size=(3, 3))
        p = rng.uniform(-2, 2, size=3)
        if abs(_terms(lib, p, tri, [[0, 1, 2]])[0] - lhuilier(p, *tri)) > 1e-9:
            return False
    s = zs.config0().surfaces[0]
    pts = np.array([[0.0, 0.0, 0.0], [0.3, -0.2, 0.1], [2.0, 0.0, 0.0]])
    want = [4 * math.pi, 4 * math.pi, 0.0]
    for p, w in zip(pts, want):
        if abs(_terms(lib, p, s.verts, s.tris).sum() - w) > 1e-9:
            return False
    return True


def test_unmutated_copy_passes(tmp_path):
    src = open(SRC).read()
    c = tmp_path / "same.c"
    so = tmp_path / "same.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                    "-o", str(so), str(c), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    lib.oracle_triangle_terms.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int64, ctypes.c_void_p,
                                                                   ctypes.c_int64, ctypes.c_void_p]
    assert _pins_pass(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    assert not _pins_pass(_build_mutant(tmp_path, name))
