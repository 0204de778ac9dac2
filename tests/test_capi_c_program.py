"""include/negf.h is a C header: a C99 program includes it, links
libnegf.so and calls the entry points that need no GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "negf.h"

int main(void) {
  int32_t sizes[1024];
  for (int i = 0; i < 1024; ++i) sizes[i] = 64;
  negf_desc d;
  memset(&d, 0, sizeof d);           /* the descriptor is a plain C struct */
  d.n_blocks = 4;
  d.block_sizes = sizes;
  d.band_n = 4;                      /* even: invalid, rejected before any device call */
  d.n_energies = 1;
  d.n_domains = 1;
  negf_plan_t* p = NULL;
  printf("%d %s\n", (int)negf_plan(&p, &d, NULL), p == NULL ? "null" : "plan");
  printf("%s\n", negf_status_string(NEGF_ERR_SINGULAR));
  printf("%d %d\n", (int)negf_auto_domains(64, sizes, 3, 512, 152), (int)negf_auto_domains(1024, sizes, 3, 1, 152));
  printf("%d\n", (int)negf_plan_n_domains(NULL));
  return 0;
}
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no C compiler")
def test_c99_program_uses_the_header_and_library(tmp_path):
    import __graft_entry__ as g
    g.build()
    src = tmp_path / "use_negf.c"
    exe = tmp_path / "use_negf"
    src.write_text(PROGRAM)
    libdir = os.path.join(ROOT, "paper_2605_19910_gb300")
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-L", libdir, "-lnegf", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    lines = out.stdout.split("\n")
    assert lines[0] == "1 null"                       # NEGF_ERR_ARG, no plan
    assert "zero pivot" in lines[1]
    d1, d2 = (int(x) for x in lines[2].split())
    assert d1 == 1 and d2 > 1                         # many energies: RGF; one energy, long chain: DDRGF
    assert lines[3] == "-1"
