"""Checkpoint and resume: a lattice saved mid-run (odd step, so the A-A
layout of g is swapped) and loaded into a fresh lattice of the same geometry
continues bitwise like the original; wall ghosts, wall populations, the
rest-population remainder of the 16-bit formats and the step counter all
travel in the file.  A mismatched lattice is refused."""
import os

import numpy as np
import pytest

from tests import _cases as CS

pytestmark = pytest.mark.gpu

FIELDS = ("phi", "rho", "P", "ux", "uy", "uz")


def _lattice(storage, n=32):
    from paper_2512_01032_gb300 import pflb
    g, p, init = CS.sessile_case(n, 60.0)
    L = pflb.Lattice(g.nx, g.ny, g.nz, solid=g.solid, wall_normal=g.normals(),
                     theta_cells=g.theta(), storage=storage, **p)
    return L, init


@pytest.mark.parametrize("storage", ["fp64", "fp32", "bf16"])
def test_save_load_resumes_bitwise(storage, tmp_path):
    A, init = _lattice(storage)
    A.init_tanh(0, init["center"], init["R"])
    A.step(13)
    ck = os.path.join(str(tmp_path), "a.ckpt")
    A.save(ck)
    B, _ = _lattice(storage)
    B.load(ck)
    assert B.t == A.t == 13
    for L in (A, B):
        L.step(20)
    for k in FIELDS:
        assert np.array_equal(A.read(k), B.read(k)), k
    # the diagnostics add block sums with FP64 atomics in no fixed order
    assert A.diag()["mass"] == pytest.approx(B.diag()["mass"], rel=1e-13)


def test_load_refuses_a_different_lattice(tmp_path):
    from paper_2512_01032_gb300 import pflb
    A, init = _lattice("fp32")
    A.init_tanh(0, init["center"], init["R"])
    ck = os.path.join(str(tmp_path), "a.ckpt")
    A.save(ck)
    C, _ = _lattice("fp32", n=24)
    with pytest.raises(pflb.PflbError):
        C.load(ck)
    D, _ = _lattice("fp64")
    with pytest.raises(pflb.PflbError):
        D.load(ck)


@pytest.mark.parametrize("damage", ["truncated", "trailing", "negative_step"])
def test_load_of_a_damaged_checkpoint_leaves_the_lattice_unchanged(damage, tmp_path):
    """A checkpoint cut short inside its population sections, one with bytes
    beyond what its header states, or one with a negative step is refused
    with PFLB_ERR_ARG before any device buffer or the step counter changes:
    the lattice keeps its own state and continues exactly like an untouched
    twin."""
    import struct

    from paper_2512_01032_gb300 import pflb
    A, init = _lattice("fp32")
    A.init_tanh(0, init["center"], init["R"])
    A.step(9)
    ck = os.path.join(str(tmp_path), "a.ckpt")
    A.save(ck)
    raw = bytearray(open(ck, "rb").read())
    if damage == "truncated":
        raw = raw[: 56 + (len(raw) - 56) * 2 // 3]  # ends inside the g section
    elif damage == "trailing":
        raw += b"\0"
    else:
        raw[48:56] = struct.pack("<q", -4)
    bad = os.path.join(str(tmp_path), "bad.ckpt")
    open(bad, "wb").write(bytes(raw))

    B, _ = _lattice("fp32")
    B.init_tanh(0, init["center"], init["R"])
    B.step(4)
    T, _ = _lattice("fp32")  # untouched twin of B
    T.init_tanh(0, init["center"], init["R"])
    T.step(4)
    with pytest.raises(pflb.PflbError) as ei:
        B.load(bad)
    assert ei.value.status == pflb.ERR_ARG
    assert B.t == 4
    for L in (B, T):
        L.step(7)
    for k in FIELDS:
        assert np.array_equal(B.read(k), T.read(k)), k
