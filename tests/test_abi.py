"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/gempic.h
declares; the ctypes structures match the C layout.  No compute calls (no GPU needed)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gempic.h")


@pytest.fixture(scope="module")
def built():
    from paper_2509_16793_gb300 import build
    return build.build()


def declared_functions():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(gempic_\w+)\s*\(", txt, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("gempic_create", "gempic_step", "gempic_get_fields", "gempic_get_particles",
              "gempic_get_state", "gempic_get_diagnostics", "gempic_destroy", "gempic_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    for n in declared_functions():
        assert hasattr(lib, n), n
    from paper_2509_16793_gb300 import gempic
    assert set(gempic.SIGNATURES) == set(declared_functions())


def test_strerror_without_gpu(built):
    from paper_2509_16793_gb300 import gempic
    lib = gempic.load(built)
    assert lib.gempic_strerror(-4).decode().startswith("Delta h omega_p^2 > 4")
    assert lib.gempic_strerror(0).decode() == "ok"


def test_ctypes_layout_matches_c():
    from paper_2509_16793_gb300 import gempic as G
    src = r"""
    #include <stdio.h>
    #include <stddef.h>
    #include "gempic.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu\n", sizeof(gempic_grid), sizeof(gempic_species),
             sizeof(gempic_laser), sizeof(gempic_config), sizeof(gempic_diag));
      printf("%zu %zu %zu %zu\n", offsetof(gempic_config, species), offsetof(gempic_config, laser),
             offsetof(gempic_config, pipeline_depth), offsetof(gempic_config, cuda_stream));
      printf("%zu %zu %zu\n", sizeof(gempic_channel), offsetof(gempic_config, channel),
             offsetof(gempic_config, hz));
      printf("%zu %zu %zu %zu %zu\n", sizeof(gempic_beam), offsetof(gempic_beam, n_macro),
             offsetof(gempic_beam, seed), offsetof(gempic_config, beam),
             offsetof(gempic_laser, fwhm_intensity));
      return 0;
    }
    """
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        r = subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe],
                           capture_output=True, text=True)
        if r.returncode != 0:
            pytest.skip("no C compiler")
        out = subprocess.run([exe], capture_output=True, text=True).stdout.split()
    sizes = [int(v) for v in out]
    assert sizes[:5] == [ctypes.sizeof(t) for t in (G.gempic_grid, G.gempic_species, G.gempic_laser,
                                                     G.gempic_config, G.gempic_diag)]
    assert sizes[5:9] == [G.gempic_config.species.offset, G.gempic_config.laser.offset,
                          G.gempic_config.pipeline_depth.offset, G.gempic_config.cuda_stream.offset]
    assert sizes[9:12] == [ctypes.sizeof(G.gempic_channel), G.gempic_config.channel.offset,
                           G.gempic_config.hz.offset]
    assert sizes[12:] == [ctypes.sizeof(G.gempic_beam), G.gempic_beam.n_macro.offset,
                          G.gempic_beam.seed.offset, G.gempic_config.beam.offset,
                          G.gempic_laser.fwhm_intensity.offset]


def test_plain_c_caller_links_and_runs(built):
    """The boundary is usable from C alone: a C99 program compiled against include/gempic.h
    with warnings as errors links libgempic.so and makes calls that need no GPU (argument
    checks happen before any CUDA call)."""
    src = r"""
    #include <stdio.h>
    #include <string.h>
    #include "gempic.h"
    int main(void) {
      struct gempic_sim* sim = NULL;
      gempic_config c;
      gempic_status st;
      memset(&c, 0, sizeof c);
      c.grid.nx = 100; c.grid.ny = 1; c.grid.nzeta = 16;     /* nx not a power of two */
      c.grid.hx = 1.0; c.grid.hy = 1.0; c.grid.h = 0.1; c.precision = 32;
      st = gempic_create(&c, &sim);
      printf("%d %d %s\n", (int)st, sim == NULL, gempic_strerror(st));
      gempic_destroy(NULL);
      return 0;
    }
    """
    libdir = os.path.dirname(built)
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "caller.c")
        exe = os.path.join(d, "caller")
        open(c, "w").write(src)
        r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                            "-I", os.path.join(ROOT, "include"), c, "-o", exe,
                            built, "-Wl,-rpath," + libdir], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    st, null, msg = out.stdout.split(maxsplit=2)
    assert st == "-1" and null == "1" and "invalid argument" in msg
