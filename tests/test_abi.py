"""The C-ABI library builds for sm_103a and exports every entry point that
include/fmm.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(fmm_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fmm_create", "fmm_solve", "fmm_reinit_signed_distance",
                     "fmm_adjoint", "fmm_destroy", "fmm_get_stats", "fmm_last_error"):
        assert required in names


def test_library_builds_and_exports_every_symbol():
    from paper_1502_07303_gb300 import build
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_1502_07303_gb300 import fmm
    assert set(fmm.EXPORTED) <= set(declared_functions())


def test_create_error_without_gpu_is_reported():
    """Argument checking happens before any CUDA call: a bad config returns
    FMM_ERR_INVALID with a message, even on a machine without a GPU."""
    from paper_1502_07303_gb300 import fmm
    lib = fmm.load()
    cfg = fmm.FmmConfig()
    cfg.nx, cfg.ny, cfg.nz, cfg.h, cfg.dtype = 0, 4, 4, 0.1, 0
    h = ctypes.c_void_p()
    rc = lib.fmm_create(ctypes.byref(cfg), None, 1.0, None, 0, ctypes.byref(h))
    assert rc == fmm.FMM_ERR_INVALID
    assert b"grid" in lib.fmm_last_error(None)
    cfg.nx, cfg.h = 4, -1.0
    assert lib.fmm_create(ctypes.byref(cfg), None, 1.0, None, 0, ctypes.byref(h)) == fmm.FMM_ERR_INVALID
    cfg.h, cfg.dtype = 0.1, 7
    assert lib.fmm_create(ctypes.byref(cfg), None, 1.0, None, 0, ctypes.byref(h)) == fmm.FMM_ERR_INVALID
    cfg.dtype = 0
    src = (ctypes.c_int64 * 3)(9, 0, 0)
    assert lib.fmm_create(ctypes.byref(cfg), None, 1.0, src, 1, ctypes.byref(h)) == fmm.FMM_ERR_INVALID
    assert b"outside" in lib.fmm_last_error(None)
    assert lib.fmm_solve(None, None, None) == fmm.FMM_ERR_INVALID
    assert lib.fmm_solve_fixed(None, None, None, None) == fmm.FMM_ERR_INVALID
    lib.fmm_destroy(None)


def _struct_fields(name):
    """Field names of the C struct typedef `name` in include/fmm.h, in order."""
    text = open(os.path.join(ROOT, "include", "fmm.h")).read()
    bodies = dict((n, b) for b, n in re.findall(r"typedef struct \{([^{}]*)\}\s*(\w+);", text))
    body = bodies[name]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        for part in decl.split(","):   # int64_t nx, ny, nz
            ids = re.findall(r"[A-Za-z_][A-Za-z_0-9]*", part)
            if ids:
                fields.append(ids[-1])
    return fields


def test_binding_structs_match_header():
    """The ctypes structs carry the header's fields in the header's order."""
    from paper_1502_07303_gb300 import fmm
    for cname, pyst in (("fmm_config", fmm.FmmConfig), ("fmm_stats", fmm.FmmStats),
                        ("fmm_trace_entry", fmm.FmmTraceEntry)):
        assert [f[0] for f in pyst._fields_] == _struct_fields(cname), cname


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "fmm.h"

int main(void)
{
    fmm_config cfg;
    fmm_handle *h = NULL;
    memset(&cfg, 0, sizeof(cfg));
    cfg.nx = cfg.ny = cfg.nz = 8;
    cfg.h = 0.125;
    cfg.hy = -1.0;                   /* negative cell size: rejected */
    cfg.dtype = FMM_F32;
    if (fmm_create(&cfg, NULL, 1.0, NULL, 0, &h) != FMM_ERR_INVALID || h != NULL)
        return 1;
    if (strlen(fmm_last_error(NULL)) == 0)
        return 2;
    int64_t bytes = 0;
    if (fmm_checkpoint_size(NULL, &bytes) != FMM_ERR_INVALID)
        return 3;
    printf("%zu %zu\n", sizeof(fmm_config), sizeof(fmm_stats));
    return 0;
}
"""


def test_header_compiles_as_c_and_links(tmp_path):
    """include/fmm.h is plain C11 (warnings are errors): a C caller compiles
    against it, links the library, gets argument errors without a GPU, and
    sees the struct sizes the binding uses."""
    import subprocess
    from paper_1502_07303_gb300 import build, fmm
    lib = build.build()
    src = tmp_path / "caller.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "caller"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe), lib,
                    f"-Wl,-rpath,{os.path.dirname(lib)}"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr)
    cfg_size, stats_size = (int(v) for v in r.stdout.split())
    assert cfg_size == ctypes.sizeof(fmm.FmmConfig)
    assert stats_size == ctypes.sizeof(fmm.FmmStats)


def test_deterministic_mode_needs_the_phased_schedule():
    """fmm_create refuses deterministic = 1 with the persistent or continuous
    schedule (argument checks run before any CUDA call: no GPU needed)."""
    from paper_1502_07303_gb300 import fmm
    lib = fmm.load()
    for sched in (2, 3):
        cfg = fmm.FmmConfig()
        cfg.nx = cfg.ny = cfg.nz = 8
        cfg.h = 0.125
        cfg.dtype = 0
        cfg.schedule = sched
        cfg.deterministic = 1
        h = ctypes.c_void_p()
        rc = lib.fmm_create(ctypes.byref(cfg), None, 1.0, None, 0, ctypes.byref(h))
        assert rc == fmm.FMM_ERR_INVALID and not h.value
        assert b"deterministic" in lib.fmm_last_error(None)


def test_second_order_and_cell_schedule_argument_checks():
    """fmm_create refuses the second-order march off the cell-parallel
    schedule, with a tape or in deterministic mode, an accuracy outside
    0..2 and a schedule above 4; fmm_create_batch refuses schedule 4 and
    accuracy 2 (argument checks run before any CUDA call: no GPU needed)."""
    from paper_1502_07303_gb300 import fmm
    lib = fmm.load()

    def cfg_of(**kw):
        cfg = fmm.FmmConfig()
        cfg.nx = cfg.ny = cfg.nz = 8
        cfg.h = 0.125
        cfg.dtype = 1
        for k, v in kw.items():
            setattr(cfg, k, v)
        return cfg

    cases = [
        (dict(accuracy=2, schedule=1), b"cell-parallel"),
        (dict(accuracy=2, schedule=3), b"cell-parallel"),
        (dict(accuracy=2, record_tape=1), b"tape"),
        (dict(schedule=4, record_tape=1), b"tape"),
        (dict(accuracy=2, deterministic=1), b"deterministic"),
        (dict(accuracy=3), b"accuracy"),
        (dict(accuracy=-1), b"accuracy"),
        (dict(schedule=5), b"schedule"),
    ]
    for kw, word in cases:
        cfg = cfg_of(**kw)
        h = ctypes.c_void_p()
        rc = lib.fmm_create(ctypes.byref(cfg), None, 1.0, None, 0, ctypes.byref(h))
        assert rc == fmm.FMM_ERR_INVALID and not h.value, kw
        assert word in lib.fmm_last_error(None), (kw, lib.fmm_last_error(None))
    dims = (ctypes.c_int64 * 3)(8, 8, 8)
    hs = (ctypes.c_double * 1)(0.125)
    for kw in (dict(schedule=4), dict(accuracy=2)):
        cfg = cfg_of(**kw)
        h = ctypes.c_void_p()
        rc = lib.fmm_create_batch(1, dims, hs, ctypes.byref(cfg), ctypes.byref(h))
        assert rc == fmm.FMM_ERR_INVALID and not h.value, kw
        assert b"single-grid" in lib.fmm_last_error(None)
