"""The C ABI without a GPU: the library builds for sm_103a, loads, exports every
function include/directcut.h declares, and the Python binding's structures
match the header's layouts (checked by compiling the header with gcc)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1711_07663_gb300 as dc
from paper_1711_07663_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "directcut.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return dc.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(dc_[a-z_]+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert set(names) == set(dc.EXPORTED), names
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", dc.lib_path()], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}$", out, flags=re.M), n


def test_version_and_error_without_gpu(lib):
    assert "sm_103a" in dc.dc_version()
    assert isinstance(dc.dc_last_error(), str)


def test_allocation_counter_and_failure_arming_without_gpu(lib):
    n0 = dc.dc_fail_alloc(-1)
    assert n0 >= 0
    # arming and disarming make no allocation
    assert dc.dc_fail_alloc(0) == n0
    assert dc.dc_fail_alloc(5) == n0
    assert dc.dc_fail_alloc(-1) == n0
    # without a device, dc_create fails before its first allocation
    cfg = dc.dc_config()
    dc.load().dc_config_default(ctypes.byref(cfg))
    if not _has_device():
        nodes = (ctypes.c_double * 24)()
        md = dc.dc_mesh_desc(p=1, n_elem=1, nodes=ctypes.cast(nodes, ctypes.c_void_p), nodes_on_device=0)
        out = ctypes.c_void_p()
        st = dc.load().dc_create(ctypes.byref(cfg), ctypes.byref(md), 1, ctypes.byref(out))
        assert st != 0 and not out.value
        assert dc.dc_fail_alloc(-1) == n0


def _has_device():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_struct_layouts_match_header(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "directcut.h"\n'
        "#define F(T, m) printf(#T \".\" #m \" %zu\\n\", offsetof(T, m))\n"
        "#define S(T) printf(#T \" %zu\\n\", sizeof(T))\n"
        "int main(void){\n"
        "S(dc_mesh_desc); F(dc_mesh_desc,p); F(dc_mesh_desc,n_elem); F(dc_mesh_desc,nodes); F(dc_mesh_desc,nodes_on_device);\n"
        "S(dc_config); F(dc_config,device); F(dc_config,precision); F(dc_config,mem_budget_bytes); F(dc_config,tol);\n"
        "F(dc_config,holemap_cells); F(dc_config,bin_cubes); F(dc_config,max_inflight); F(dc_config,profile); F(dc_config,reserve_faces);\n"
        "S(dc_request); F(dc_request,q); F(dc_request,n_faces); F(dc_request,face_nodes); F(dc_request,pose);\n"
        "F(dc_request,flags_out); F(dc_request,dist_out); F(dc_request,on_device); F(dc_request,async); F(dc_request,stream);\n"
        "F(dc_request,fp32_dist_out);\n"
        "S(dc_stats); F(dc_stats,holemap_rows_undecided); F(dc_stats,ms_surface); F(dc_stats,ms_total);\n"
        "S(dc_tuning); F(dc_tuning,cubes_per_edge); F(dc_tuning,bin_cubes); F(dc_tuning,warps_per_cta);\n"
        "F(dc_tuning,cands_per_warp); F(dc_tuning,ms);\n"
        "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)], check=True)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    rename = {"async": "async_"}
    for cname, pyt in (("dc_mesh_desc", dc.dc_mesh_desc), ("dc_config", dc.dc_config), ("dc_request", dc.dc_request),
                       ("dc_stats", dc.dc_stats), ("dc_tuning", dc.dc_tuning)):
        assert int(got[cname]) == ctypes.sizeof(pyt), cname
        for key, val in got.items():
            if key.startswith(cname + "."):
                field = rename.get(key.split(".", 1)[1], key.split(".", 1)[1])
                assert getattr(pyt, field).offset == int(val), key


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(dc, "_lib", None)
    monkeypatch.setattr(dc, "lib_path", lambda: str(tmp_path / "absent.so"))
    with pytest.raises(dc.DirectCutError):
        dc.load()


def test_argument_errors_are_status_codes_without_a_gpu(lib):
    """Every entry point checks its arguments before it touches the device:
    bad values come back as DC_EINVAL with a message, never a crash."""
    EINVAL = -1
    P = ctypes.c_void_p
    out = P()
    cfg = dc.dc_config()
    assert lib.dc_config_default(ctypes.byref(cfg)) == 0
    assert cfg.precision == dc.DC_FP32_RECHECK and cfg.holemap_cells == 0 and cfg.bin_cubes == 4

    def bad(status, what):
        assert status == EINVAL, what
        assert dc.dc_last_error() != "", what

    desc = (dc.dc_mesh_desc * 1)()
    desc[0].p, desc[0].n_elem, desc[0].nodes = 9, 1, None
    bad(lib.dc_create(ctypes.byref(cfg), desc, 1, ctypes.byref(out)), "order p=9")
    for field, val in (("tol", -1.0), ("holemap_cells", 5), ("bin_cubes", 17), ("max_inflight", 65), ("precision", 7)):
        c2 = dc.dc_config()
        lib.dc_config_default(ctypes.byref(c2))
        setattr(c2, field, val)
        desc[0].p, desc[0].n_elem = 2, 1
        bad(lib.dc_create(ctypes.byref(c2), desc, 1, ctypes.byref(out)), field)
    bad(lib.dc_create(ctypes.byref(cfg), desc, 0, ctypes.byref(out)), "no meshes")
    bad(lib.dc_create(ctypes.byref(cfg), desc, 1, None), "out NULL")
    # after-cut set logic
    bad(lib.dc_blank_union(0, None, None, 10, None, None), "n_cuts 0")
    bad(lib.dc_blank_union(9, None, None, 10, None, None), "n_cuts 9")
    bad(lib.dc_ab_faces(0, None, None, None, None, None), "n_elem 0")
    bad(lib.dc_unblank(5, 10, None, None, None, None, None, None, None), "kind 5")
    # donor search
    bad(lib.dc_pc_create(0, 0, 10, None, 0, ctypes.byref(out)), "order p=0")
    bad(lib.dc_pc_create(0, 5, 10, None, 0, ctypes.byref(out)), "order p=5")
    bad(lib.dc_pc_create(0, 2, 0, None, 0, ctypes.byref(out)), "n_elem 0")
    bad(lib.dc_pc_locate(None, 0, None, None, None, None, 0, None), "pc NULL")
    # tuning on a NULL context
    t = dc.dc_tuning()
    bad(lib.dc_set_tuning(None, ctypes.byref(t)), "ctx NULL")
    bad(lib.dc_get_stats(None, None), "ctx NULL")
    lib.dc_destroy(None)
    lib.dc_pc_destroy(None)
