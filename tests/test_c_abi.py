"""The boundary is plain C: a C11 program that includes include/bvf.h and
include/bvf_fno.h compiles with gcc (-Wall -Werror -pedantic), links against
libbvf.so, and gets the documented host-side answers (version, Courant limit,
status strings, argument errors, weight counts) without a GPU."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SRC = r"""
#include <stdio.h>
#include <string.h>
#include "bvf.h"
#include "bvf_fno.h"

static int fails = 0;
#define CHECK(c) do { if (!(c)) { printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #c); ++fails; } } while (0)

int main(void)
{
    bvf_ctx *ctx = (bvf_ctx *)1;
    bvf_grid g;
    bvf_physics ph;
    bvf_fno_dims d;
    bvf_fno *f = (bvf_fno *)1;
    float w[4] = {0, 0, 0, 0};

    CHECK(bvf_version() == BVF_VERSION);
    CHECK(bvf_courant_limit() > 0.49 && bvf_courant_limit() < 0.50);
    CHECK(strlen(bvf_strerror(BVF_E_CFL)) > 0);

    memset(&g, 0, sizeof g);
    memset(&ph, 0, sizeof ph);
    g.nx = 0; g.ny = 8; g.nz = 8; g.dx = 1e-3; g.dt = 1e-7;
    ph.f0 = 5e5; ph.qc = 1.0; ph.n_sls = 2;
    CHECK(bvf_create(&g, &ph, &ctx) == BVF_E_ARG);
    CHECK(ctx == NULL);
    CHECK(strlen(bvf_last_error(NULL)) > 0);
    CHECK(bvf_run_acoustic(NULL, 1, NULL, NULL) == BVF_E_ARG);

    d.c_in = 8; d.width = 32; d.modes = 12; d.n_layers = 4; d.hidden = 128; d.c_out = 1;
    CHECK(bvf_fno_weight_count(&d) > 0);
    d.width = 30;
    CHECK(bvf_fno_weight_count(&d) == 0);
    d.width = 32;
    CHECK(bvf_fno_create(&f, &d, w, 4) == BVF_E_ARG);
    CHECK(f == NULL);
    CHECK(bvf_fno_forward(NULL, 8, 8, 8, NULL, NULL, NULL) == BVF_E_ARG);
    CHECK(bvf_fno_synchronize(NULL, NULL) == BVF_E_ARG);
    printf("c-abi checks failed: %d\n", fails);
    return fails != 0;
}
"""


def test_headers_compile_as_c_and_link(tmp_path):
    from paper_2301_12727_gb300 import build
    lib = build.build()
    src = tmp_path / "abi.c"
    src.write_text(C_SRC)
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib)
    cmd = ["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic",
           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
           "-L", libdir, "-l:libbvf.so", "-Wl,-rpath," + libdir]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "failed: 0" in run.stdout
