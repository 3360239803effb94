"""The allocation-free field/diagnostic entry point (pflb_fields_noalloc).

It serves callers that cannot allocate device memory (their memory belongs
to another allocator, or they cannot afford cudaMalloc's implicit device
synchronisation); its scratch lives in fixed file-scope device arrays.  The
test hands it a lattice's populations, obtained through the existing
checkpoint call, in caller-owned device buffers, and checks its fields and
diagnostics against the existing pflb_read / pflb_diag of that lattice, on
two calls in a row (the shared scratch keeps the previous call's contents
and must be cleared by each call).  This file is collected last.
"""
import os
import struct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _read_checkpoint(path, N):
    with open(path, "rb") as f:
        magic = f.read(8)
        hdr = struct.unpack("<6q", f.read(48))
        h = np.frombuffer(f.read(19 * N * 4), dtype=np.float32).copy()
        g = np.frombuffer(f.read(19 * N * 4), dtype=np.float32).copy()
    assert magic == b"PFLBCKP1" and hdr[3] == 0 and hdr[4] == 1
    return hdr, h, g


def test_fields_noalloc_matches_existing_pass(tmp_path):
    import torch
    from paper_2512_01032_gb300 import pflb

    nx, ny, nz = 40, 36, 28
    N = nx * ny * nz
    p = pflb.default_params(storage="fp32", sigma=0.01, W=4.0, M=0.02, blend=0.0)
    L = pflb.Lattice(nx, ny, nz, params=p)
    L.init_tanh(0, (19.3, 17.6, 13.2), 8.0)
    L.step(10)  # even step count: g in natural layout, as the entry point expects
    ref_d = L.diag()
    ref_f = {k: L.read(k) for k in ("phi", "rho", "P", "ux", "uy", "uz")}
    ck = os.path.join(str(tmp_path), "state.ckpt")
    L.save(ck)
    hdr, h, g = _read_checkpoint(ck, N)
    assert hdr[5] == 10

    dev = torch.device("cuda", torch.cuda.current_device())
    h_t = torch.from_numpy(h).to(dev)
    g_t = torch.from_numpy(g).to(dev)
    fields = torch.empty(6 * N, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    for call in range(2):
        fields.fill_(float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        d = pflb.fields_noalloc(nx, ny, nz, h_t.data_ptr(), g_t.data_ptr(), p,
                                fields_ptr=fields.data_ptr(), stream=None)
        torch.cuda.synchronize()
        if call == 1:
            # the first call on a device loads the entry point's code and
            # scratch; a later call must not take any device memory
            assert torch.cuda.mem_get_info()[0] == free0
        f = fields.cpu().numpy().reshape(6, N)
        for k, name in enumerate(("phi", "rho", "P", "ux", "uy", "uz")):
            ref = ref_f[name]
            err = np.max(np.abs(f[k] - ref))
            if name in ("phi", "rho"):
                assert err <= 1e-5 * np.max(np.abs(ref)), (call, name, err)
            elif name == "P":
                assert err <= 1e-5 * max(np.max(np.abs(ref)), 2 * 0.01 / 8.0), (call, name, err)
            else:
                assert err <= 2e-5, (call, name, err)
        assert abs(d["mass"] - ref_d["mass"]) <= 2e-6 * ref_d["mass"], call
        assert d["n_heavy"] == ref_d["n_heavy"], call
        assert abs(d["p_heavy"] - ref_d["p_heavy"]) <= 1e-5 * 0.0025, call
        assert abs(d["p_light"] - ref_d["p_light"]) <= 1e-5 * 0.0025, call
        assert abs(d["u_max"] - ref_d["u_max"]) <= 2e-5, call
        assert abs(d["kinetic"] - ref_d["kinetic"]) <= 1e-4 * ref_d["kinetic"] + 1e-15, call
        assert d["nonfinite"] == 0


def test_fields_noalloc_rejects_oversize_lattice():
    import torch
    from paper_2512_01032_gb300 import pflb

    p = pflb.default_params(storage="fp32")
    buf = torch.zeros(1, device="cuda")
    with pytest.raises(pflb.PflbError) as ei:
        pflb.fields_noalloc(128, 128, 128, buf.data_ptr(), buf.data_ptr(), p)
    assert ei.value.status == pflb.ERR_ARG
    assert "at most" in str(ei.value)


def test_fields_noalloc_rejects_16_bit_storage():
    """The entry point reads FP32 populations; parameters that name another
    storage are refused instead of being reinterpreted."""
    import torch
    from paper_2512_01032_gb300 import pflb

    buf = torch.zeros(19 * 8 * 8 * 8, device="cuda")
    out = torch.empty(6 * 8 * 8 * 8, dtype=torch.float64, device="cuda")
    for st in ("bf16", "fp16", "fp64"):
        p = pflb.default_params(storage=st)
        with pytest.raises(pflb.PflbError) as ei:
            pflb.fields_noalloc(8, 8, 8, buf.data_ptr(), buf.data_ptr(), p,
                                fields_ptr=out.data_ptr())
        assert ei.value.status == pflb.ERR_ARG
        assert "FP32" in str(ei.value)
