"""CPU checks of the C ABI: the library builds, loads and exports every
function that include/sph.h declares; the ctypes structs match the C layout;
without a GPU the calls fail with an error code instead of falling back."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

from paper_2104_00537_gb300 import sph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sph.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_[a-z_]+)\s*\(", text)) -
                  {"sph_alloc_fn", "sph_free_fn"})


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sph_create", "sph_step", "sph_get_state", "sph_destroy", "sph_batch_create",
                 "sph_pool_create", "sph_pool_admit", "sph_pool_step", "sph_pool_release",
                 "sph_get_raw", "sph_create_from_raw", "sph_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = sph.load()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", sph.lib_path()], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (sph_[a-z_]+)\b", out))
    assert set(declared_functions()) <= exported


def test_struct_layout_matches_c():
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "sph.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(sph_case_params), sizeof(sph_particles),
         sizeof(sph_motion), sizeof(sph_stats), sizeof(sph_options));
  printf("%zu %zu %zu\n", offsetof(sph_case_params, cell_mode),
         offsetof(sph_particles, n_motions), offsetof(sph_stats, n));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(src, "w").write(prog)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        sizes, offs = subprocess.check_output([exe], text=True).strip().split("\n")
    assert [int(x) for x in sizes.split()] == [
        C.sizeof(sph.CaseParams), C.sizeof(sph.Particles), C.sizeof(sph.Motion),
        C.sizeof(sph.Stats), C.sizeof(sph.Options)]
    assert [int(x) for x in offs.split()] == [
        sph.CaseParams.cell_mode.offset, sph.Particles.n_motions.offset, sph.Stats.n.offset]


def test_every_field_offset_matches_c():
    """Every field of every struct the binding passes, at the offset the C
    compiler gives it (a field added, dropped or reordered on one side only
    fails here)."""
    structs = {"sph_case_params": sph.CaseParams, "sph_particles": sph.Particles,
               "sph_motion": sph.Motion, "sph_stats": sph.Stats, "sph_options": sph.Options}
    lines = []
    for cname, cls in structs.items():
        for fname, _ in cls._fields_:
            lines.append('  printf("%%s %%s %%zu\\n", "%s", "%s", offsetof(%s, %s));'
                         % (cname, fname, cname, fname))
    prog = ("#include <stdio.h>\n#include <stddef.h>\n#include \"sph.h\"\n"
            "int main(void) {\n" + "\n".join(lines) + "\n  return 0;\n}\n")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(src, "w").write(prog)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        out = subprocess.check_output([exe], text=True).split("\n")
    got = {(c, f): int(o) for c, f, o in (x.split() for x in out if x.strip())}
    for cname, cls in structs.items():
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
        # the last field ends where the C struct (with its tail padding) allows
        assert C.sizeof(cls) >= max(getattr(cls, f).offset for f, _ in cls._fields_)


def test_calls_without_gpu_fail_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2104_00537_gb300 import cases
    with pytest.raises(sph.SphError) as ei:
        sph.Engine.create(cases.free_particle(), torch_alloc=False)
    assert ei.value.code in (-3, -2)


def test_null_arguments_are_rejected():
    L = sph.load()
    assert L.sph_step(None, 1) == -1
    assert L.sph_get_state(None, 0, None, None, None, None, None, None, None) == -1
    assert L.sph_create(None, None, None, sph._NULL_ALLOC, sph._NULL_FREE, None, None) == -1
    assert "null" in sph.last_error()
    L.sph_destroy(None)
