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


@pytest.mark.parametrize("storage", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("kernel", [0, 3])
def test_non_finite_state_is_reported_as_err_nan(storage, kernel):
    """A non-finite value injected on the host (one NaN cell in the initial
    phi field given to pflb_init_phi, which does not screen its input) is
    counted by the next diagnostic step and reported as PFLB_ERR_NAN by
    pflb_last_diag and pflb_diag, with the diagnostics filled in.  Nothing
    faults: it is a state error, not a CUDA error, so the lattice is not
    poisoned, and initialising it again gives a clean run."""
    import oracle as O
    from paper_2512_01032_gb300 import pflb
    g, p, init = CS.droplet_case(16, 4.0)
    L = pflb.Lattice(g.nx, g.ny, g.nz, storage=storage, **p)
    L.set_kernel(kernel)
    phi = O.tanh_phi(0, (g.nx, g.ny, g.nz), init["center"], init["R"], p["W"])
    phi[7 + g.nx * (8 + g.ny * 6)] = np.nan
    L.init_phi(phi)
    L.set_diag_every(1)
    L.step(2)
    with pytest.raises(pflb.PflbError) as ei:
        L.last_diag()
    assert ei.value.status == pflb.ERR_NAN
    d = L.last_diag(allow_nan=True)
    assert d["step"] == 1 and d["nonfinite"] >= 1
    with pytest.raises(pflb.PflbError) as ei:
        L.diag()
    assert ei.value.status == pflb.ERR_NAN
    assert L.diag(allow_nan=True)["nonfinite"] >= 1
    # not poisoned: a fresh state steps cleanly
    L.init_tanh(0, init["center"], init["R"])
    L.step(3)
    d = L.last_diag()
    assert d["nonfinite"] == 0 and d["mass"] > 0
    assert np.isfinite(L.read("phi")).all()
