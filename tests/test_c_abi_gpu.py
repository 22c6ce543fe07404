"""A plain C program drives one FDTD run through the C ABI on the GPU (device
buffers from cudaMalloc, no Python in the loop) and its pressure field equals,
bit for bit, the same run through the Python binding."""
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SRC = r"""
#include <stdio.h>
#include <stdlib.h>
#include <cuda_runtime.h>
#include "bvf.h"

#define NX 48
#define NY 40
#define NZ 36
#define CK(x) do { int rc_ = (x); if (rc_ != BVF_OK) { \
    fprintf(stderr, "%s -> %d: %s\n", #x, rc_, bvf_last_error(NULL)); return 1; } } while (0)

int main(int argc, char **argv)
{
    const size_t N = (size_t)NX * NY * NZ;
    bvf_grid g = {NX, NY, NZ, 0.5e-3, 6.0e-8, 6, 1e-4};
    bvf_physics ph = {5e5, 1.0, 2, BVF_STORAGE_F32, 0.0};
    bvf_material tab[2] = {{1000.0, 1500.0, 0.0, 0.0, 0.0, 0.6, 4180.0, 0.0, 1.0},
                           {1850.0, 2800.0, 1500.0, 85.0, 170.0, 0.32, 1300.0, 0.0, 0.16}};
    uint8_t *h_idx = (uint8_t *)malloc(N);
    float *h_plane = (float *)malloc(2 * NX * NY * sizeof(float));
    float *h_p = (float *)malloc(N * sizeof(float));
    uint8_t *d_idx;
    float *d_plane, *d_p;
    bvf_ctx *ctx = NULL;
    bvf_capture cap = {0, 0, 0};
    size_t q;
    int i, j;
    FILE *f;

    for (q = 0; q < N; ++q) {
        int k = (int)(q / (NX * NY));
        h_idx[q] = (k >= 18 && k < 24) ? 1 : 0;      /* a 3 mm bone slab */
    }
    for (j = 0; j < NY; ++j)
        for (i = 0; i < NX; ++i) {
            h_plane[2 * (j * NX + i)] = 1.0e4f;
            h_plane[2 * (j * NX + i) + 1] = 0.0f;
        }
    if (cudaMalloc((void **)&d_idx, N) || cudaMalloc((void **)&d_plane, 2 * NX * NY * sizeof(float)) ||
        cudaMalloc((void **)&d_p, N * sizeof(float)))
        return 2;
    cudaMemcpy(d_idx, h_idx, N, cudaMemcpyHostToDevice);
    cudaMemcpy(d_plane, h_plane, 2 * NX * NY * sizeof(float), cudaMemcpyHostToDevice);

    CK(bvf_create(&g, &ph, &ctx));
    CK(bvf_set_materials(ctx, d_idx, tab, 2));
    CK(bvf_set_source(ctx, 8, d_plane, 1500.0, BVF_ENV_BURST, 2, NULL));
    CK(bvf_run_acoustic(ctx, 150, &cap, NULL));
    CK(bvf_get_pressure(ctx, d_p, NULL));
    CK(bvf_synchronize(ctx, NULL));
    cudaMemcpy(h_p, d_p, N * sizeof(float), cudaMemcpyDeviceToHost);
    bvf_destroy(ctx);
    f = fopen(argv[1], "wb");
    if (!f || fwrite(h_p, sizeof(float), N, f) != N) return 3;
    fclose(f);
    cudaFree(d_idx);
    cudaFree(d_plane);
    cudaFree(d_p);
    free(h_idx);
    free(h_plane);
    free(h_p);
    printf("c driver done\n");
    return 0;
}
"""


def test_c_program_run_equals_the_python_binding(tmp_path):
    import torch
    from paper_2301_12727_gb300 import build
    lib = build.build()
    from paper_2301_12727_gb300 import bvf
    cuda = "/usr/local/cuda"
    src = tmp_path / "drive.c"
    src.write_text(C_SRC)
    exe = tmp_path / "drive"
    libdir = os.path.dirname(lib)
    cmd = ["gcc", "-std=c11", "-O2", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(cuda, "include"), str(src), "-o", str(exe),
           "-L", libdir, "-l:libbvf.so", "-Wl,-rpath," + libdir,
           "-L", os.path.join(cuda, "lib64"), "-lcudart", "-Wl,-rpath," + os.path.join(cuda, "lib64")]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    out = tmp_path / "p.bin"
    run = subprocess.run([str(exe), str(out)], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0, run.stdout + run.stderr
    p_c = np.fromfile(out, dtype=np.float32).reshape(36, 40, 48)

    idx = np.zeros((36, 40, 48), np.uint8)
    idx[18:24] = 1
    table = [(1000.0, 1500.0, 0.0, 0.0, 0.0, 0.6, 4180.0, 0.0, 1.0),
             (1850.0, 2800.0, 1500.0, 85.0, 170.0, 0.32, 1300.0, 0.0, 0.16)]
    s = bvf.Solver(48, 40, 36, 0.5e-3, 6.0e-8, 5e5, n_sls=2, n_pml=6)
    s.set_materials(idx, np.array(table))
    s.set_source(np.full((40, 48), 1.0e4, dtype=np.complex128), 8, 1500.0, bvf.BVF_ENV_BURST, 2)
    s.run(150, peak_from=0)
    s.synchronize()
    p_py = s.pressure().cpu().numpy()
    s.close()
    assert np.abs(p_py).max() > 0.0
    assert np.array_equal(p_c, p_py)
