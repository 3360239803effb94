"""The single-lattice multi-GPU design, tested on CPU ranks: a lattice cut
into z-slabs that exchange one phi plane and the populations streaming
through each face per step reproduces the undecomposed step bit for bit
(no GPU; the oracle's per-cell routines do the arithmetic)."""
import numpy as np
import pytest

from tests import _slab as S

DIMS, KW = S.DIMS, S.KW
STEPS = 4


@pytest.fixture(scope="module")
def reference():
    L, (solid3, nrm, theta, h, g, ghost) = S.case()
    one = S.run(DIMS, solid3, nrm, theta, KW, h, g, ghost, [(0, DIMS[2])], STEPS)
    L.step(STEPS)
    hc, gc = L.populations()
    return (solid3, nrm, theta, h, g, ghost), one, (hc, gc, L.ghosts())


def test_one_slab_is_the_oracle_step(reference):
    """The slab stepper with a single slab is the oracle's step (to
    rounding: the angle's cosine and sine are formed on different sides)."""
    _, (h1, g1, gh1, _), (hc, gc, ghc) = reference
    assert np.abs(h1 - hc).max() < 1e-14
    assert np.abs(g1 - gc).max() < 1e-14
    assert np.abs(gh1 - ghc).max() < 1e-14
    assert np.abs(h1).max() > 0.01


@pytest.mark.parametrize("parts", [2, 3])
def test_slabs_reproduce_the_undecomposed_step_bitwise(reference, parts):
    """Cut into 2 or 3 slabs, exchanging per step and per face one phi
    plane (the neighbours' stencil halo) and the 5 + 5 populations that
    stream through it (free-slip reflections that cross the face included,
    in slots ordinary streaming leaves empty), the run equals the one-slab
    run bit for bit."""
    inputs, (h1, g1, gh1, _), _ = reference
    h, g, gh, sent = S.run(DIMS, *inputs[:3], KW, *inputs[3:], S.split(DIMS[2], parts), STEPS)
    assert S.run.reflected_across > 0  # free-slip reflections crossed a face
    assert np.array_equal(h, h1) and np.array_equal(g, g1) and np.array_equal(gh, gh1)
    face = DIMS[0] * DIMS[1]
    assert sent == [2 * 11 * face] * parts  # 11 values per face cell, two faces


def test_a_missing_exchange_is_visible(reference):
    """Without the phi halo (stale zeros) the slab faces diverge at once:
    the exchange is needed, not incidental."""
    inputs, (h1, _, _, _), _ = reference
    solid3, nrm, theta, h, g, ghost = inputs
    slabs = [S.Slab(DIMS, z0, z1, solid3, nrm, theta, KW, h, g, ghost)
             for z0, z1 in S.split(DIMS[2], 2)]
    for s in slabs:
        s.compute_phi()
        s.halo_lo = s.halo_hi = np.zeros((DIMS[1], DIMS[0]))
    for s in slabs:
        s.update_ghosts()
    outs = [s.collide_and_stream() for s in slabs]
    for k, s in enumerate(slabs):
        b, a = outs[(k - 1) % 2], outs[(k + 1) % 2]
        s.receive((b["hi_h"], b["hi_g"]), (a["lo_h"], a["lo_g"]))
        s.swap()
    one_step = S.run(DIMS, solid3, nrm, theta, KW, h, g, ghost, [(0, DIMS[2])], 1)[0]
    got = np.concatenate([s.h for s in slabs])
    assert np.abs(got - one_step).max() > 1e-4


def _free_port():
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def test_two_gloo_ranks_exchange_the_faces(reference, tmp_path):
    """The same decomposition with one slab per process: two gloo ranks
    that swap the phi planes and the face populations by point-to-point
    messages end bit for bit where the undecomposed step does."""
    import torch.multiprocessing as mp
    out = tmp_path / "slabs.npz"
    mp.spawn(S.rank_main, args=(2, _free_port(), STEPS, str(out)), nprocs=2, join=True)
    got = np.load(out)
    _, (h1, g1, gh1, _), _ = reference
    assert np.array_equal(got["h"], h1) and np.array_equal(got["g"], g1)
    assert np.array_equal(got["ghost"], gh1)
    assert list(got["sent"]) == [2 * 11 * DIMS[0] * DIMS[1]] * 2


def test_slabs_with_open_x_boundaries():
    """Open x boundaries (a velocity inlet at x = 0, a pressure outlet at
    x = nx - 1) do not change the exchange: 2 and 3 slabs still equal one
    slab bit for bit, and one slab is the oracle's step."""
    L, (solid3, nrm, theta, h, g, gh) = S.case()
    xbc = (dict(type="velocity", u=(3e-3, 1e-3, 0.0), phi=0.2), dict(type="pressure", P=1e-3))
    L.set_x_boundaries(*xbc)
    one = S.run(DIMS, solid3, nrm, theta, KW, h, g, gh, [(0, DIMS[2])], STEPS, xbc)
    L.step(STEPS)
    hc, gc = L.populations()
    assert np.abs(one[0] - hc).max() < 1e-14 and np.abs(one[1] - gc).max() < 1e-14
    assert np.abs(one[2] - L.ghosts()).max() < 1e-14
    for parts in (2, 3):
        got = S.run(DIMS, solid3, nrm, theta, KW, h, g, gh, S.split(DIMS[2], parts), STEPS, xbc)
        for a, b in zip(got[:3], one[:3]):
            assert np.array_equal(a, b)
