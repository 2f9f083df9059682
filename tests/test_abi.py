"""CPU checks of the boundary: the library builds for sm_103a, loads
without a GPU, and exports every entry point that include/hydro.h declares;
the Python binding's structs match the header's layout."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hydro.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(hydro_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2211_12243_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_2211_12243_gb300 import hydro
    assert sorted(hydro.EXPORTS) == _declared()


def test_struct_sizes_match_header(lib):
    """Compile a tiny C program against the header and compare sizeof with
    the ctypes mirrors."""
    import subprocess
    import tempfile
    from paper_2211_12243_gb300 import hydro
    prog = r'''
#include <stdio.h>
#include "hydro.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(hydro_config), sizeof(hydro_particles),
         sizeof(hydro_nbrlist), sizeof(hydro_stats), sizeof(hydro_tuning));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = list(map(int, out))
    assert sizes == [ctypes.sizeof(hydro.Config), ctypes.sizeof(hydro.Particles),
                     ctypes.sizeof(hydro.NbrList), ctypes.sizeof(hydro.Stats),
                     ctypes.sizeof(hydro.Tuning)]


def test_defaults_and_strerror(lib):
    from paper_2211_12243_gb300 import hydro
    cfg = hydro.default_config()
    assert cfg.ncond_crit == 100.0 and cfg.ngb_grow == 1.2
    assert cfg.psi1 == 0.5 and cfg.psi2 == 0.25 and cfg.n_ngb == 32.0
    L = hydro._load()
    for code in range(0, -11, -1):
        assert L.hydro_strerror(code)
