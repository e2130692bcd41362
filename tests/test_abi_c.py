"""The boundary is a plain C ABI: include/tomo.h compiles as strict C99 and as
C++, a C program links against the built library and calls it (entry points
that need no GPU), and the binding's ctypes structures have the same size and
field offsets as the header's structs on this machine."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "include")

PROBE = r"""
#include <stddef.h>
#include <stdio.h>
#include "tomo.h"
#define OFF(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
    printf("version %d\n", tomo_version());
    printf("error '%s'\n", tomo_last_error());
    printf("dadmm_config %zu\n", sizeof(dadmm_config));
    printf("dadmm_state %zu\n", sizeof(dadmm_state));
    OFF(dadmm_config, N); OFF(dadmm_config, M); OFF(dadmm_config, node_ang_ptr);
    OFF(dadmm_config, eta1); OFF(dadmm_config, eta2); OFF(dadmm_config, rho);
    OFF(dadmm_config, E1); OFF(dadmm_config, jpeg_quality); OFF(dadmm_config, seed);
    OFF(dadmm_config, mode); OFF(dadmm_config, max_stale); OFF(dadmm_config, variant);
    OFF(dadmm_config, tune);
    OFF(dadmm_state, u); OFF(dadmm_state, iter);
    return 0;
}
"""


def need(tool):
    if shutil.which(tool) is None:
        pytest.skip(tool + " not found")


@pytest.fixture(scope="module")
def libpath():
    from paper_2410_06106_gb300 import build
    return build.build()


@pytest.mark.parametrize("cc,flags", [("gcc", ["-x", "c", "-std=c99", "-pedantic"]),
                                      ("g++", ["-x", "c++", "-std=c++17", "-pedantic"])])
def test_header_compiles_as_c_and_cpp(tmp_path, cc, flags):
    need(cc)
    src = tmp_path / "h.c"
    src.write_text('#include "tomo.h"\nint tomo_header_probe;\n')
    r = subprocess.run([cc] + flags + ["-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-I", INC, str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.fixture(scope="module")
def probe_output(libpath, tmp_path_factory):
    need("gcc")
    d = tmp_path_factory.mktemp("probe")
    src = d / "probe.c"
    src.write_text(PROBE)
    exe = d / "probe"
    libdir = os.path.dirname(libpath)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", INC, str(src), "-o", str(exe),
                        "-L", libdir, "-l:" + os.path.basename(libpath), "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    return dict(line.rsplit(" ", 1) for line in out.stdout.splitlines())


def test_c_program_links_and_calls_the_library(probe_output):
    assert int(probe_output["version"]) > 0
    assert probe_output["error"] == "''"


def test_ctypes_structs_match_the_header(probe_output):
    from paper_2410_06106_gb300 import api
    assert ctypes.sizeof(api.DadmmConfig) == int(probe_output["dadmm_config"])
    assert ctypes.sizeof(api.DadmmState) == int(probe_output["dadmm_state"])
    for key, val in probe_output.items():
        if key.startswith("dadmm_config."):
            assert getattr(api.DadmmConfig, key.split(".")[1]).offset == int(val), key
        if key.startswith("dadmm_state."):
            assert getattr(api.DadmmState, key.split(".")[1]).offset == int(val), key
