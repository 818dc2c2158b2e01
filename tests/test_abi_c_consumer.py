"""The C-ABI as a C program sees it: include/ubs.h compiles as strict C99 and
C++11, and a C99 program linked against the library gets the same answers
from the host-side calls (workspace sizes, status strings, argument checks)
as the Python binding.  No GPU is used: every call below returns before any
launch."""
import os
import shutil
import subprocess

import pytest

from paper_2510_03312_gb300 import build as B
from paper_2510_03312_gb300 import ubs as U

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "include")


def _cuda_include():
    nv = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nv))), "include")
    return inc if os.path.exists(os.path.join(inc, "cuda_runtime.h")) else None


@pytest.fixture(scope="module")
def cc():
    c = shutil.which("gcc")
    if not c or not _cuda_include():
        pytest.skip("gcc or the CUDA headers are not installed")
    return c


@pytest.mark.parametrize("lang,std", [("c", "c99"), ("c", "c11"), ("c++", "c++11"), ("c++", "c++17")])
def test_header_compiles_on_its_own(cc, lang, std, tmp_path):
    src = tmp_path / ("h.c" if lang == "c" else "h.cpp")
    src.write_text('#include "ubs.h"\nint main(void) { return 0; }\n')
    comp = cc if lang == "c" else (shutil.which("g++") or cc)
    r = subprocess.run([comp, "-x", lang, f"-std={std}", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-I", INC, "-I", _cuda_include(), "-fsyntax-only", str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


PROGRAM = r"""
#include <stdio.h>
#include "ubs.h"

int main(void) {
  int32_t w[2] = {1600, 33}, h[2] = {1060, 17}, bad[1] = {0};
  char* fake = (char*)0x10000;
  printf("loss_ws %zu\n", ubs_loss_workspace_size(2, w, h));
  printf("loss_ws_bad %zu\n", ubs_loss_workspace_size(1, bad, h));
  printf("mcmc_ws %zu\n", ubs_mcmc_workspace_size(123457));
  printf("mcmc_ws_zero %zu\n", ubs_mcmc_workspace_size(0));
  /* a null image: rejected before any launch */
  printf("loss_null %d\n", (int)ubs_image_loss(1, w, h, NULL, (float*)fake, 0.2f, (float*)fake, (float*)fake,
                                               fake, ubs_loss_workspace_size(1, w, h), 0));
  /* a workspace one byte short */
  printf("loss_short %d\n", (int)ubs_image_loss(1, w, h, (float*)fake, (float*)fake, 0.2f, (float*)fake,
                                                (float*)fake, fake, ubs_loss_workspace_size(1, w, h) - 1, 0));
  printf("ws_null %zu\n", ubs_workspace_size(NULL));
  printf("str_ok %s\n", ubs_status_string(UBS_OK));
  printf("str_ws %s\n", ubs_status_string(UBS_ERR_WORKSPACE));
  return 0;
}
"""


def test_c_program_links_and_matches_the_binding(cc, tmp_path):
    lib = B.build()
    U.load()
    src = tmp_path / "consumer.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "consumer"
    libdir = os.path.dirname(lib)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", INC, "-I", _cuda_include(), str(src),
                        "-o", str(exe), lib, f"-Wl,-rpath,{libdir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    got = dict(line.split(" ", 1) for line in r.stdout.strip().splitlines())
    assert int(got["loss_ws"]) == U.ubs_loss_workspace_size([1600, 33], [1060, 17]) > 0
    assert int(got["loss_ws_bad"]) == 0
    assert int(got["mcmc_ws"]) == U.ubs_mcmc_workspace_size(123457) > 0
    assert int(got["mcmc_ws_zero"]) == 0
    assert int(got["loss_null"]) == U.UBS_ERR_INVALID_ARG
    assert int(got["loss_short"]) == U.UBS_ERR_WORKSPACE
    assert int(got["ws_null"]) == 0
    assert got["str_ok"] == U.ubs_status_string(U.UBS_OK)
    assert got["str_ws"] == U.ubs_status_string(U.UBS_ERR_WORKSPACE)
