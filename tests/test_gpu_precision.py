"""Reduced-precision population storage (FP16 and BF16 weight-scaled
deviations, FP32 arithmetic) against the FP64 oracle.

Pointwise bound after n steps, derived from the formats: h_i / w_i lies in
about [0, 1], where FP16 spacing is at most 2^-11 and BF16 spacing 2^-8, so
each stored moving h_i is off by at most w_i 2^-12 (FP16) or w_i 2^-9
(BF16); a cell's phi collects those of its 18 incoming populations and the
compensation of its own outgoing ones (rest population), at most
2 (1 - w_0) 2^-12 = 3.3e-4 (FP16) or 2.6e-3 (BF16) per step; the test allows
n times that.  Total phi is conserved (mass-conserving rounding of h).

Physics: the Laplace pressure jump of the static droplet and the mass drift
after 2000 steps, against the FP64 oracle (target for the reduced-precision
form: Laplace pressure within 1 % of the oracle)."""
import numpy as np
import pytest

from tests import _cases as CS

pytestmark = pytest.mark.gpu

PER_STEP = {"fp16": 2 * (2.0 / 3.0) * 2.0 ** -12, "bf16": 2 * (2.0 / 3.0) * 2.0 ** -9}


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
@pytest.mark.parametrize("kernel", [0, 1])
def test_reduced_storage_pointwise_bound(storage, kernel):
    g, p, init = CS.droplet_case()
    G, Orc = CS.make_pair(g, p, init, storage=storage, kernel=kernel)
    t = 0
    for s in (1, 4, 10):
        G.step(s - t)
        Orc.step(s - t)
        t = s
        e = CS.rel_errors(CS.gpu_fields(G), Orc.macros(), 2 * p["sigma"] / init["R"])
        assert e["phi"] <= max(s, 1) * PER_STEP[storage] * 1.0001, (storage, s, e)


@pytest.mark.slow
def test_reduced_storage_laplace_and_mass():
    """Static droplet (32^3, R=8): pressure jump p_heavy - p_light and mass
    after 2000 steps for FP32, FP16 and BF16 storage against the oracle."""
    import os
    import oracle as O
    from paper_2512_01032_gb300 import pflb
    g, p, init = CS.droplet_case()
    op = {k: v for k, v in p.items() if k in CS.ORACLE_KEYS}
    Orc = O.OracleLattice(g.nx, g.ny, g.nz, nthreads=os.cpu_count() or 1, **op)
    phi0 = O.tanh_phi(0, (g.nx, g.ny, g.nz), init["center"], init["R"], p["W"])
    Orc.init_phi(phi0)
    m0 = Orc.macros()
    Orc.step(2000)
    m = Orc.macros()
    ref_dp = m["P"][m["phi"] > 0.95].mean() - m["P"][m["phi"] < 0.05].mean()
    ref_mass0 = m0["phi"].sum()
    out = {}
    for storage in ("fp32", "fp16", "bf16"):
        L = pflb.Lattice(g.nx, g.ny, g.nz, storage=storage, **p)
        L.init_tanh(0, init["center"], init["R"])
        d0 = L.diag()
        L.step(2000)
        d = L.diag()
        out[storage] = dict(dp_err=abs(d["dp"] - ref_dp) / abs(ref_dp),
                            drift=abs(d["mass"] - d0["mass"]) / ref_mass0)
    print("precision errors vs FP64 oracle:", out, "reference dp", ref_dp)
    assert out["fp32"]["dp_err"] < 1e-3
    assert out["fp16"]["dp_err"] < 1e-2
    assert out["fp32"]["drift"] < 1e-5
    assert out["fp16"]["drift"] < 1e-5
    assert out["bf16"]["drift"] < 1e-5
    assert out["bf16"]["dp_err"] < 0.2
