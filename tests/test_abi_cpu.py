"""C ABI checks that need no GPU: the library builds and exports every
function declared in include/pflb.h, the ctypes structs match the C layout,
and argument validation rejects bad input before any device work."""
import json
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pflb.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pflb_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    from paper_2512_01032_gb300 import pflb
    pflb.load()
    out = subprocess.run(["nm", "-D", "--defined-only", pflb.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pflb_\w+)", out))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing
    assert len(_declared()) >= 18


def test_struct_layouts_match_header(tmp_path):
    """sizeof/offsetof of the C structs equal the ctypes mirrors."""
    import ctypes as C
    from paper_2512_01032_gb300 import pflb
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stddef.h>
#include <stdio.h>
#include "pflb.h"
int main(void) {
  printf("{\"params\": %zu, \"geom\": %zu, \"diag\": %zu, "
         "\"storage\": %zu, \"Fex\": %zu, \"nonfinite\": %zu, \"cl_m2\": %zu}\n",
         sizeof(pflb_params), sizeof(pflb_geometry), sizeof(pflb_diag_t),
         offsetof(pflb_params, storage), offsetof(pflb_params, Fex),
         offsetof(pflb_diag_t, nonfinite), offsetof(pflb_diag_t, cl_m2));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = json.loads(subprocess.run([str(exe)], capture_output=True, text=True,
                                    check=True).stdout)
    assert got["params"] == C.sizeof(pflb.Params)
    assert got["geom"] == C.sizeof(pflb.Geometry)
    assert got["diag"] == C.sizeof(pflb.Diag)
    assert got["storage"] == pflb.Params.storage.offset
    assert got["Fex"] == pflb.Params.Fex.offset
    assert got["nonfinite"] == pflb.Diag.nonfinite.offset
    assert got["cl_m2"] == pflb.Diag.cl_m2.offset


def test_server_struct_layouts_match_header(tmp_path):
    """The serving structs: sizeof and every field offset equal the ctypes
    mirrors."""
    import ctypes as C
    from paper_2512_01032_gb300 import pflb
    structs = {"pflb_diag_raw_t": pflb.DiagRaw, "pflb_xbc": pflb.XBC,
               "pflb_server_config": pflb.ServerConfig, "pflb_solve_spec": pflb.SolveSpec,
               "pflb_solve_result": pflb.SolveResult, "pflb_server_stats": pflb.ServerStats}
    lines = []
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    src = tmp_path / "layout2.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"pflb.h\"\n"
                   "int main(void) {\n" + "\n".join(lines) + "\n  return 0;\n}\n")
    exe = tmp_path / "layout2"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    for line in out.strip().splitlines():
        cname, f, v = line.split()
        py = structs[cname]
        want = C.sizeof(py) if f == "size" else getattr(py, f).offset
        assert int(v) == want, (cname, f)


def test_default_params_are_the_papers():
    from paper_2512_01032_gb300 import pflb
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    p = pflb.default_params()
    for k, attr in (("gamma", "gamma"), ("phi_M", "phi_M"), ("phi_m", "phi_m"), ("D", "D"),
                    ("eps_dtheta", "eps"), ("blend", "blend"), ("band_lo", "band_lo"),
                    ("band_hi", "band_hi"), ("F_tilde", "F_tilde"), ("F_width", "F_width")):
        assert getattr(p, attr) == gold[k]["value"], k


@pytest.mark.parametrize("bad", [dict(nu_H=0.0), dict(nu_L=-0.1), dict(W=0.0), dict(M=0.0),
                                 dict(rho_L=0.0), dict(blend=1.5), dict(storage=7),
                                 dict(F_mode=3), dict(D=0.0)])
def test_create_rejects_bad_parameters(bad):
    """tau = nu/T + 1/2 must exceed 1/2 and the other parameters be valid:
    PFLB_ERR_ARG before any device call."""
    from paper_2512_01032_gb300 import pflb
    with pytest.raises(pflb.PflbError) as ei:
        pflb.Lattice(4, 4, 4, **bad)
    assert ei.value.status == pflb.ERR_ARG


def test_create_rejects_bad_geometry():
    import ctypes as C
    from paper_2512_01032_gb300 import pflb
    lib = pflb.load()
    p = pflb.default_params()
    h = C.c_void_p()
    g, keep = pflb.make_geometry(2, 2, 2)
    g.nx = 0
    assert lib.pflb_create(C.byref(g), C.byref(p), None, C.byref(h)) == pflb.ERR_ARG
    assert lib.pflb_create(None, C.byref(p), None, C.byref(h)) == pflb.ERR_ARG
    assert b"null" in lib.pflb_last_error()
    # null handles are rejected, not dereferenced
    assert lib.pflb_step(None, 1) == pflb.ERR_ARG
    assert lib.pflb_tune(None, 10, None) == pflb.ERR_ARG
    assert lib.pflb_get_step(None) == -1
    lib.pflb_destroy(None)
    # batches: empty or null lattice lists and null batches are rejected
    b = C.c_void_p()
    assert lib.pflb_batch_create(None, 0, None, C.byref(b)) == pflb.ERR_ARG
    arr = (C.c_void_p * 2)(None, None)
    assert lib.pflb_batch_create(arr, 2, None, C.byref(b)) == pflb.ERR_ARG
    assert lib.pflb_batch_step(None, 1, 0) == pflb.ERR_ARG
    assert lib.pflb_batch_set_launch(None, 32, 4, 16, 0) == pflb.ERR_ARG
    assert lib.pflb_batch_tune(None, 1, None) == pflb.ERR_ARG
    lib.pflb_batch_destroy(None)
    # server: null and invalid arguments are rejected before any device call
    srv = C.c_void_p()
    assert lib.pflb_server_create(None, None, C.byref(srv)) == pflb.ERR_ARG
    cfg = pflb.ServerConfig(1 << 30, pflb.STORAGE_FP32, 0, 0, 1, 0)
    assert lib.pflb_server_create(C.byref(cfg), None, C.byref(srv)) == pflb.ERR_ARG
    cfg = pflb.ServerConfig(0, pflb.STORAGE_FP32, 10, 0, 1, 0)
    assert lib.pflb_server_create(C.byref(cfg), None, C.byref(srv)) == pflb.ERR_ARG
    t = C.c_int64()
    assert lib.pflb_server_submit(None, None, None, None, C.byref(t)) == pflb.ERR_ARG
    assert lib.pflb_server_tick(None, None) == pflb.ERR_ARG
    r = pflb.SolveResult()
    assert lib.pflb_server_poll(None, 1, C.byref(r)) == pflb.ERR_ARG
    st = pflb.ServerStats()
    assert lib.pflb_server_stats_get(None, C.byref(st)) == pflb.ERR_ARG
    lib.pflb_server_destroy(None)
    assert lib.pflb_step_ex(None, 1, 0) == pflb.ERR_ARG
    assert lib.pflb_get_kernel(None, (C.c_int * 4)()) == pflb.ERR_ARG
    assert lib.pflb_set_x_boundaries(None, None, None) == pflb.ERR_ARG
    assert lib.pflb_selftest_wait_timeout(None, 100) == pflb.ERR_ARG
    raw = pflb.DiagRaw()
    assert lib.pflb_last_diag_async(None, C.byref(raw), C.byref(t)) == pflb.ERR_ARG
    assert lib.pflb_diag_wait(None, 0, C.byref(raw), C.byref(pflb.Diag())) == pflb.ERR_ARG


def test_estimate_bytes_counts_wall_nodes():
    """Host-side footprint estimate (used for admission by memory budget)."""
    from paper_2512_01032_gb300 import pflb
    n = 16
    empty = pflb.estimate_bytes(n, n, n)
    solid = np.zeros((n, n, n), np.uint8)
    solid[0] = 1
    walled = pflb.estimate_bytes(n, n, n, solid)
    N = n ** 3
    assert empty == 3 * 19 * N * 4 + N * 5 + N * 4 + 96 * 8 + 4
    nw = 2 * n * n  # planes z = 1 and z = n-1 (periodic) touch the solid layer
    # per wall node: two wall-population buffers, link mask, cell index,
    # geometry (5), ghosts (18) and its slot in the pipelined kernel's
    # per-block wall lists; plus the lists' block offsets (32 x 4 tiles,
    # one plane per block: 1 x 4 x 16 blocks, and one more offset)
    blocks = 1 * (n // 4) * n
    assert walled - empty == nw * (2 * 18 * 4 + 4 + 4 + 5 * 4 + 18 * 4 + 4) + (blocks + 1) * 4


def test_estimate_bytes_with_cut_cells():
    """Sub-voxel walls: the cells next to a cut row become wall nodes, and a
    lattice with cut cells keeps a cut-link word per wall node and a
    fraction per cell; a fluid fraction outside [0, 1) is refused (-1)."""
    from paper_2512_01032_gb300 import pflb
    n = 16
    N = n ** 3
    solid = np.zeros((n, n, n), np.uint8)
    solid[0] = 1
    walled = pflb.estimate_bytes(n, n, n, solid)
    frac = np.zeros((n, n, n))
    frac[1] = 0.3  # the plane z = 1 is cut
    cut = pflb.estimate_bytes(n, n, n, solid, solid_frac=frac)
    per_node = 2 * 18 * 4 + 4 + 4 + 5 * 4 + 18 * 4 + 4
    # z = 2 joins the wall nodes (z = 1 and z = n - 1 already are)
    assert cut - walled == n * n * per_node + 3 * n * n * 4 + N * 4
    frac[1, 0, 0] = 1.0
    assert pflb.estimate_bytes(n, n, n, solid, solid_frac=frac) == -1


def test_no_cpu_fallback_without_a_gpu():
    """With the library built but no GPU, a valid lattice is refused with a
    CUDA error; nothing falls back to host computation.  (Skipped where a
    GPU is present: there the lattice is simply created.)"""
    from paper_2512_01032_gb300 import pflb
    try:
        L = pflb.Lattice(8, 8, 8)
    except pflb.PflbError as e:
        assert e.status == pflb.ERR_CUDA, e
        return
    L.close() if hasattr(L, "close") else None
    pytest.skip("a GPU is present")


@pytest.mark.parametrize("kw,exc", [(dict(sigmaa=0.1), KeyError), (dict(storage="fp8"), KeyError),
                                    (dict(solid=[1, 0]), ValueError),
                                    (dict(theta_cells=[1.0, 0.0]), ValueError),
                                    (dict(wall_normal=[1.0, 0.0]), ValueError)])
def test_binding_rejects_malformed_arguments(kw, exc):
    """The binding refuses misspelt parameters, unknown storage names and
    geometry arrays of the wrong size before any library call."""
    from paper_2512_01032_gb300 import pflb
    with pytest.raises(exc):
        pflb.Lattice(4, 4, 4, **kw)


@pytest.mark.parametrize("lang,std", [("c", "c99"), ("c++", "c++11")])
def test_header_is_self_contained(tmp_path, lang, std):
    """include/pflb.h compiles on its own, warning-free, as strict C99 and
    C++11 (a C ABI must not rely on what the caller included before it)."""
    src = tmp_path / "only.c"
    src.write_text('#include "pflb.h"\nint main(void) { return 0; }\n')
    cc = "gcc" if lang == "c" else "g++"
    r = subprocess.run([cc, f"-std={std}", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-fsyntax-only", "-x", lang, "-I", os.path.join(ROOT, "include"),
                        str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_program_links_and_calls_the_library(tmp_path):
    """A plain C99 program includes pflb.h, links libpflb.so and calls the
    entry points that need no GPU: default parameters, argument checks with
    their error messages, the footprint estimate and the null-tolerant
    destructors."""
    from paper_2512_01032_gb300 import pflb
    lib = pflb.lib_path()
    src = tmp_path / "use.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "pflb.h"
int main(void) {
  pflb_params p;
  pflb_default_params(&p);
  if (p.gamma != -22.5 || p.blend != 0.95 || p.storage != PFLB_STORAGE_FP32) return 1;
  pflb_lattice *L = NULL;
  if (pflb_create(NULL, &p, NULL, &L) != PFLB_ERR_ARG || L != NULL) return 2;
  if (strlen(pflb_last_error()) == 0) return 3;
  uint8_t solid[8 * 8 * 8];
  memset(solid, 0, sizeof solid);
  memset(solid, 1, 8 * 8);  /* the plane z = 0 */
  pflb_geometry g = {8, 8, 8, solid, NULL, NULL};
  int64_t bytes = pflb_estimate_bytes(&g, PFLB_STORAGE_FP32);
  if (bytes <= 0) return 4;
  p.nu_H = 0.0;  /* tau = 1/2 */
  if (pflb_create(&g, &p, NULL, &L) != PFLB_ERR_ARG) return 5;
  if (pflb_step(NULL, 1) != PFLB_ERR_ARG) return 6;
  pflb_destroy(NULL);
  pflb_batch_destroy(NULL);
  pflb_server_destroy(NULL);
  printf("%lld\n", (long long)bytes);
  return 0;
}
''')
    exe = tmp_path / "use"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), lib, f"-Wl,-rpath,{os.path.dirname(lib)}", "-o", str(exe)],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stderr)
    solid = np.zeros((8, 8, 8), np.uint8)
    solid[0] = 1
    assert int(r.stdout) == pflb.estimate_bytes(8, 8, 8, solid)


def test_binding_declares_every_entry_point():
    """Every function of include/pflb.h has ctypes argument types and the
    return type of its C declaration (an undeclared int64_t return would be
    truncated to int)."""
    import ctypes as C
    from paper_2512_01032_gb300 import pflb
    lib = pflb.load()
    txt = open(os.path.join(ROOT, "include", "pflb.h")).read()
    want = {"pflb_status": C.c_int, "void": None, "int64_t": C.c_int64,
            "const char *": C.c_char_p}
    decls = re.findall(r"^\s*([a-z_0-9 ]+?\**)\s*\b(pflb_[a-z_0-9]+)\s*\(", txt, re.M)
    assert len(decls) == len(_declared())
    for rt, name in decls:
        f = getattr(lib, name)
        assert f.argtypes is not None, name
        assert f.restype == want[rt.strip()], (name, rt, f.restype)
