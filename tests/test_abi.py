"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/*.h declares (no compute call: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1409_5474_gb300 import build as nb_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(nb_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    path = nb_build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for core in ("nb_create", "nb_set_particles", "nb_predict", "nb_force", "nb_correct",
                 "nb_step", "nb_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1409_5474_gb300 import nbody
    assert set(_declared()) <= set(nbody.declared_symbols()) | set()


def test_status_strings_and_create_without_device(lib):
    from paper_1409_5474_gb300 import nbody
    nbody.load()
    assert nbody.nb_status_string(0) == "NB_OK"
    assert nbody.nb_status_string(6) == "NB_ERR_NONFINITE"
    assert "sm_103a" in nbody.nb_version()
    cfg = nbody.nb_config_default(n_max=16)
    assert cfg.variant == nbody.NB_F32DS and cfg.dt_max == 1.0 / 16 and cfg.eta == 0.01
    # argument checks run before any device work
    for bad in ({"eps": -1.0}, {"eta": 0.0}, {"dt_max": 0.1}, {"n_max": 0}, {"variant": 7},
                {"dt_min": 0.25, "dt_max": 0.125}):
        kw = dict(n_max=16)
        kw.update(bad)
        c = nbody.nb_config_default(**kw)
        with pytest.raises(nbody.NBodyError) as ei:
            nbody.nb_create(c)
        assert ei.value.status == nbody.NB_ERR_ARG


def test_missing_library_fails_loudly(tmp_path):
    """No library means an error, never a CPU fallback."""
    from paper_1409_5474_gb300 import nbody
    saved = nbody._lib
    nbody._lib = None
    try:
        with pytest.raises(RuntimeError):
            nbody.load(str(tmp_path / "none.so"))
    finally:
        nbody._lib = saved


def test_struct_layouts_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets the C compiler
    gives the header's struct of the same name (a field added on one side only fails)."""
    import subprocess
    from paper_1409_5474_gb300 import nbody
    structs = [nbody.nb_config, nbody.nb_plan, nbody.nb_stats, nbody.nb_server_cfg,
               nbody.nb_request, nbody.nb_result, nbody.nb_server_stats]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nbody.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for field in st._fields_:
            f = field[0]
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c_vals = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for st in structs:
        name = st.__name__
        assert c_vals[(name, "size")] == ctypes.sizeof(st), name
        for field in st._fields_:
            f = field[0]
            assert c_vals[(name, f)] == getattr(st, f).offset, (name, f)


def test_binding_constants_match_the_header():
    """Every integer #define NB_* of the header has the same value in the binding."""
    from paper_1409_5474_gb300 import nbody
    seen = 0
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        for m in re.finditer(r"^#define\s+(NB_\w+)\s+(-?\d+)\b", open(hdr).read(), flags=re.M):
            name, value = m.group(1), int(m.group(2))
            assert getattr(nbody, name) == value, name
            seen += 1
    assert seen >= 10
