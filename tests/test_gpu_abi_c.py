"""The C ABI driven from a plain C99 program on the GPU: the program
allocates its own device buffers with the CUDA runtime (cudaMalloc), creates
a geometry, projects an image (Eq. 4) with tomo_project, creates a dADMM
solver (Algorithm 4, four nodes on a ring with K-means and JPEG messages
alternated per edge), sizes and allocates the state and workspace from the
*_size queries, runs iterations with dadmm_step and reads the
reconstruction with dadmm_home_view, all through include/tomo.h. Its outputs
are compared with the FP64 oracle: the projection at the operator tolerance
(1e-5), and the reconstruction and statistics after three iterations at the
smoke check's 1e-3."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from gpu_common import need_gpu, rel_l2
from paper_2410_06106_gb300 import synth
from problems import oracle_eta1, small_problem

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "include")

PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <cuda_runtime_api.h>
#include "tomo.h"

static const char* dir;

static void* load(const char* name, size_t bytes) {
    char path[4096];
    snprintf(path, sizeof path, "%s/%s", dir, name);
    FILE* f = fopen(path, "rb");
    if (!f) { fprintf(stderr, "cannot open %s\n", path); exit(2); }
    void* p = malloc(bytes ? bytes : 1);
    if (fread(p, 1, bytes, f) != bytes) { fprintf(stderr, "short read %s\n", path); exit(2); }
    fclose(f);
    return p;
}

static void save(const char* name, const void* p, size_t bytes) {
    char path[4096];
    snprintf(path, sizeof path, "%s/%s", dir, name);
    FILE* f = fopen(path, "wb");
    if (!f || fwrite(p, 1, bytes, f) != bytes) { fprintf(stderr, "cannot write %s\n", path); exit(2); }
    fclose(f);
}

#define TOMO(call) do { tomo_status s_ = (call); if (s_ != TOMO_OK) { \
    fprintf(stderr, "%s -> %d: %s\n", #call, s_, tomo_last_error()); return 3; } } while (0)
#define CUDA(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { \
    fprintf(stderr, "%s -> %s\n", #call, cudaGetErrorString(e_)); return 4; } } while (0)

int main(int argc, char** argv) {
    if (argc != 2) return 1;
    dir = argv[1];
    int N, B, A, M, E1, E2, iters, km_k, km_iters, jq;
    double rho, eta2;
    unsigned long long seed;
    char path[4096];
    snprintf(path, sizeof path, "%s/params.txt", dir);
    FILE* f = fopen(path, "r");
    if (!f || fscanf(f, "%d %d %d %d %d %d %d %d %d %d %lf %lf %llu", &N, &B, &A, &M, &E1, &E2, &iters,
                     &km_k, &km_iters, &jq, &rho, &eta2, &seed) != 13) return 2;
    fclose(f);
    const size_t n = (size_t)N * N;
    double* theta = (double*)load("theta.f64", sizeof(double) * A);
    float* img = (float*)load("img.f32", sizeof(float) * n);
    float* sino = (float*)load("sino.f32", sizeof(float) * A * B);
    int32_t* ptr = (int32_t*)load("ptr.i32", sizeof(int32_t) * (M + 1));
    int32_t* ang = (int32_t*)load("ang.i32", sizeof(int32_t) * A);
    int32_t* seg = (int32_t*)load("seg.i32", sizeof(int32_t) * (M + 1));
    int32_t* adj = (int32_t*)load("adj.i32", sizeof(int32_t) * M * M);
    int32_t* edge_q = (int32_t*)load("edge_q.i32", sizeof(int32_t) * M * M);
    int32_t* home_q = (int32_t*)load("home_q.i32", sizeof(int32_t) * M);
    double* eta1 = (double*)load("eta1.f64", sizeof(double) * M);

    tomo_geometry_t g;
    TOMO(tomo_geometry_create(N, B, A, theta, &g));

    /* Eq. 4 on every angle */
    float *d_img, *d_proj, *d_sino;
    CUDA(cudaMalloc((void**)&d_img, sizeof(float) * n));
    CUDA(cudaMalloc((void**)&d_proj, sizeof(float) * A * B));
    CUDA(cudaMalloc((void**)&d_sino, sizeof(float) * A * B));
    CUDA(cudaMemcpy(d_img, img, sizeof(float) * n, cudaMemcpyHostToDevice));
    CUDA(cudaMemcpy(d_sino, sino, sizeof(float) * A * B, cudaMemcpyHostToDevice));
    TOMO(tomo_project(g, d_img, d_proj, NULL, A, 1, NULL, NULL));
    float* proj = (float*)malloc(sizeof(float) * A * B);
    CUDA(cudaMemcpy(proj, d_proj, sizeof(float) * A * B, cudaMemcpyDeviceToHost));
    TOMO(tomo_sync_status(g, NULL));
    save("proj.f32", proj, sizeof(float) * A * B);

    /* Algorithm 4: one slice, M nodes */
    dadmm_config cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.N = N; cfg.n_bins = B; cfg.n_angles = A; cfg.S = 1; cfg.M = M;
    cfg.node_ang_ptr = ptr; cfg.node_ang = ang; cfg.seg_row_ptr = seg;
    cfg.adj = adj; cfg.edge_q = edge_q; cfg.home_q = home_q; cfg.eta1 = eta1;
    cfg.eta2 = eta2; cfg.rho = rho; cfg.E1 = E1; cfg.E2 = E2;
    cfg.km_k = km_k; cfg.km_iters = km_iters; cfg.jpeg_quality = jq; cfg.seed = seed;
    cfg.mode = DADMM_MODE_BATCHED; cfg.max_stale = 0; cfg.variant = DADMM_VARIANT_SEGMENTS;
    cfg.tune = DADMM_TUNE_AUTO;
    dadmm_t h;
    TOMO(dadmm_create(g, &cfg, &h));
    const int D = dadmm_ring_depth(h);
    dadmm_state st;
    CUDA(cudaMalloc((void**)&st.u, sizeof(float) * M * n));
    CUDA(cudaMalloc((void**)&st.lam, sizeof(float) * M * n));
    CUDA(cudaMalloc((void**)&st.xseg, sizeof(float) * n));
    CUDA(cudaMalloc((void**)&st.hist, sizeof(float) * (size_t)D * 3 * n));
    CUDA(cudaMalloc((void**)&st.iter, sizeof(int32_t)));
    const size_t want = sizeof(float) * (2 * M * n + n + (size_t)D * 3 * n) + sizeof(int32_t);
    if (dadmm_state_size(h) > want + 4096) { fprintf(stderr, "state size %zu\n", dadmm_state_size(h)); return 5; }
    const size_t wb = dadmm_workspace_size(h);
    void* ws;
    CUDA(cudaMalloc(&ws, wb));
    TOMO(dadmm_state_init(h, &st, NULL));
    double* stats = (double*)malloc(sizeof(double) * iters * DADMM_NSTAT);
    TOMO(dadmm_step(h, &st, d_sino, iters, ws, wb, stats, NULL));
    float* d_home;
    CUDA(cudaMalloc((void**)&d_home, sizeof(float) * n));
    TOMO(dadmm_home_view(h, &st, d_home, NULL));
    float* home = (float*)malloc(sizeof(float) * n);
    CUDA(cudaMemcpy(home, d_home, sizeof(float) * n, cudaMemcpyDeviceToHost));
    save("home.f32", home, sizeof(float) * n);
    save("stats.f64", stats, sizeof(double) * iters * DADMM_NSTAT);

    TOMO(dadmm_destroy(h));
    TOMO(tomo_geometry_destroy(g));
    cudaFree(d_img); cudaFree(d_proj); cudaFree(d_sino); cudaFree(d_home); cudaFree(ws);
    cudaFree(st.u); cudaFree(st.lam); cudaFree(st.xseg); cudaFree(st.hist); cudaFree(st.iter);
    printf("ok\n");
    return 0;
}
"""


def cuda_home():
    nv = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nv)))


def test_c_program_drives_projector_and_dadmm_through_the_abi(tmp_path):
    need_gpu()
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    from paper_2410_06106_gb300 import build
    lib = build.build()
    ch = cuda_home()
    src = tmp_path / "drive.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "drive"
    libdir = os.path.dirname(lib)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", INC, "-I", os.path.join(ch, "include"),
                        str(src), "-o", str(exe), "-L", libdir, "-l:" + os.path.basename(lib),
                        "-L", os.path.join(ch, "lib64"), "-lcudart",
                        "-Wl,-rpath," + libdir + ":" + os.path.join(ch, "lib64")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr

    N, A, B, M, iters = 64, 48, 91, 4, 3
    p = small_problem(N=N, A=A, B=B, M=M, graph="ring", quant="alternate", part="blocks", noise=0.01,
                      seed=17, E1=5, E2=5, km_k=16, jpeg_quality=50)
    eta = oracle_eta1(p, iters=40)
    img = np.random.default_rng(3).random((N, N)).astype(np.float32)
    d = tmp_path
    (d / "params.txt").write_text("%d %d %d %d %d %d %d %d %d %d %r %r %d\n" % (
        N, B, A, M, p["E1"], p["E2"], iters, p["km_k"], p["km_iters"], p["jpeg_quality"], p["rho"], p["eta2"],
        p["seed"]))
    for name, arr, dt in [("theta.f64", p["geometry"]["theta"], np.float64), ("img.f32", img, np.float32),
                          ("sino.f32", p["sino"][0], np.float32), ("ptr.i32", p["node_ang_ptr"], np.int32),
                          ("ang.i32", p["node_ang"], np.int32), ("seg.i32", p["seg_row_ptr"], np.int32),
                          ("adj.i32", p["adj"], np.int32), ("edge_q.i32", p["edge_q"], np.int32),
                          ("home_q.i32", p["home_q"], np.int32), ("eta1.f64", eta, np.float64)]:
        np.ascontiguousarray(arr, dt).tofile(str(d / name))
    out = subprocess.run([str(exe), str(d)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr

    proj = np.fromfile(str(d / "proj.f32"), np.float32).reshape(A, B)
    og = O.Geometry(N, B, p["geometry"]["theta"])
    assert rel_l2(proj, og.project(img)) <= 1e-5
    o = O.DADMM(p, eta)
    ost = np.stack([o.iterate(p["sino"]) for _ in range(iters)])
    home = np.fromfile(str(d / "home.f32"), np.float32).reshape(1, N, N)
    stats = np.fromfile(str(d / "stats.f64"), np.float64).reshape(iters, 1, 5)
    assert rel_l2(home, o.home_view()) <= 1e-3
    assert rel_l2(stats[:, 0, 3], ost[:, 0, 3]) <= 1e-3  # residual norms
    assert np.all(np.isfinite(stats))
