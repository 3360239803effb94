"""Failure detection without a GPU fault: a bounded wait that runs out
(the self-test waits on an mbarrier that nothing completes) raises the
lattice's device error flag; the host reads it at the next synchronising
call as PFLB_ERR_TIMEOUT, the lattice is poisoned, and the GPU context and
other lattices stay usable."""
import numpy as np
import pytest

from tests import _cases as CS

pytestmark = pytest.mark.gpu


def test_bounded_wait_timeout_is_reported_and_contained():
    from paper_2512_01032_gb300 import pflb
    g, p, init = CS.droplet_case(16, 4.0)
    A = pflb.Lattice(g.nx, g.ny, g.nz, storage="fp32", **p)
    B = pflb.Lattice(g.nx, g.ny, g.nz, storage="fp32", **p)
    for L in (A, B):
        L.init_tanh(0, init["center"], init["R"])
        L.step(3)
    A.selftest_wait_timeout(1000)
    with pytest.raises(pflb.PflbError) as ei:
        A.read("phi")
    assert ei.value.status == pflb.ERR_TIMEOUT
    with pytest.raises(pflb.PflbError) as ei:
        A.step(1)
    assert ei.value.status == pflb.ERR_STATE
    # the context and the other lattice are unaffected
    B.step(5)
    assert np.isfinite(B.read("phi")).all()
    C = pflb.Lattice(g.nx, g.ny, g.nz, storage="fp32", **p)
    C.init_tanh(0, init["center"], init["R"])
    C.step(2)
    assert C.diag()["mass"] > 0
    with pytest.raises(pflb.PflbError):
        C.selftest_wait_timeout(0)
