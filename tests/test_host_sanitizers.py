"""The host C/C++ under AddressSanitizer and UndefinedBehaviorSanitizer.

Two small drivers, written here into a temporary directory, are compiled
with -fsanitize=address,undefined together with the library's host mesh
builder (csrc/build.cpp: face matching, Hilbert and region orders, record
packing) and with the oracle (oracle/oracle.c), then run on the tiny scene
and on a random mesh.  Any out-of-bounds access, use after free, leak,
signed overflow or misaligned access aborts the driver.  The builder's
device upload is never called (the drivers only link the CUDA runtime to
resolve it), so nothing here needs a GPU.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import scenegen as sg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2103_02309_gb300", "csrc")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
SAN = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer",
       "-g", "-O1"]
ENV = dict(os.environ, ASAN_OPTIONS="abort_on_error=1:detect_leaks=1",
           UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")

BUILD_DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "tm_internal.h"

tm_status tm_build_host(const float *points, int64_t np, const int32_t *tets, int64_t nt,
                        const int32_t *tris, int64_t nc, const tm_build_opts *opts, tm_mesh *m);
// the builder's device path is not exercised here
void tm_set_error(const char *, cudaError_t) { std::abort(); }
tm_status launch_locate(const MeshView &, const float *, int64_t, const int32_t *, int32_t,
                        int32_t *, uint32_t, cudaStream_t) { std::abort(); }

template <class T> std::vector<T> load(const char *path, size_t n) {
    std::vector<T> v(n);
    FILE *f = std::fopen(path, "rb");
    if (!f || std::fread(v.data(), sizeof(T), n, f) != n) std::exit(3);
    std::fclose(f);
    return v;
}

int main(int argc, char **argv) {
    const int64_t np = std::atoll(argv[1]), nt = std::atoll(argv[2]), nc = std::atoll(argv[3]);
    auto P = load<float>(argv[4], 3 * np);
    auto T = load<int32_t>(argv[5], 4 * nt);
    auto C = load<int32_t>(argv[6], 3 * nc);
    for (int order = 0; order < 3; ++order) {
        tm_build_opts o{};
        o.order = order;
        o.tet20 = 1;
        o.faces = 1;
        o.faces16 = 1;
        tm_mesh *m = new tm_mesh();
        const tm_status st = tm_build_host(P.data(), np, T.data(), nt, C.data(), nc, &o, m);
        if (st != TM_OK) { std::printf("status %d\n", (int)st); return 2; }
        // every neighbour is a tet, or a flagged face id within range
        for (int64_t t = 0; t < nt; ++t)
            for (int k = 0; k < 4; ++k) {
                const uint32_t nb = (uint32_t)m->cold[8 * t + 4 + k];
                if (nb & 0x80000000u) {
                    const uint32_t c = nb & 0x7fffffffu;
                    if (c != 0x7fffffffu && c >= (uint32_t)nc) return 4;
                } else if (nb >= (uint32_t)nt) {
                    return 5;
                }
            }
        delete m;
    }
    // a mesh the builder must reject: a triangle that is no tet face
    std::vector<int32_t> bad = {0, 1, 2};
    tm_mesh *m = new tm_mesh();
    tm_build_opts o{};
    const tm_status st = tm_build_host(P.data(), np, T.data(), nt, bad.data(), 1, &o, m);
    delete m;
    std::printf("build OK %d\n", (int)st);
    return 0;
}
"""

ORACLE_DRIVER = r"""
#include <stdio.h>
#include <stdlib.h>
#include <stdint.h>

typedef struct orc_mesh orc_mesh;
int orc_mesh_create(int64_t, const float *, int64_t, const int32_t *, int64_t, const int32_t *,
                    orc_mesh **);
void orc_mesh_destroy(orc_mesh *);
int64_t orc_count_nonpositive(const orc_mesh *);
int64_t orc_count_asymmetric(const orc_mesh *);
int64_t orc_count_boundary(const orc_mesh *);
void orc_trace(const orc_mesh *, int64_t, const float *, const float *, const float *,
               const int32_t *, const int32_t *, int64_t, int, int32_t *, double *, double *,
               double *, int32_t *, int32_t *, int32_t *, int32_t *);
void orc_bruteforce(const orc_mesh *, int64_t, const float *, const float *, const float *,
                    const int32_t *, int, int32_t *, double *, double *, double *);
void orc_locate(const orc_mesh *, int64_t, const float *, int, int32_t *, double *);

static void *load(const char *path, size_t bytes) {
    void *p = malloc(bytes ? bytes : 1);
    FILE *f = fopen(path, "rb");
    if (!p || !f || fread(p, 1, bytes, f) != bytes) exit(3);
    fclose(f);
    return p;
}

int main(int argc, char **argv) {
    int64_t np = atoll(argv[1]), nt = atoll(argv[2]), nc = atoll(argv[3]), nr = atoll(argv[4]);
    float *P = load(argv[5], 12 * np);
    int32_t *T = load(argv[6], 16 * nt), *C = load(argv[7], 12 * nc);
    float *o = load(argv[8], 12 * nr), *d = load(argv[9], 12 * nr), *tm = load(argv[10], 4 * nr);
    orc_mesh *m = NULL;
    if (orc_mesh_create(np, P, nt, T, nc, C, &m) != 0) return 2;
    if (orc_count_nonpositive(m) != 0 || orc_count_asymmetric(m) != 0) return 4;
    (void)orc_count_boundary(m);
    int32_t *start = malloc(4 * nr), *tri = malloc(4 * nr), *tri2 = malloc(4 * nr);
    int32_t *tet = malloc(4 * nr), *cf = malloc(4 * nr), *st = malloc(4 * nr), *fl = malloc(4 * nr);
    int32_t *entry = malloc(4 * nr);
    double *t = malloc(8 * nr), *b1 = malloc(8 * nr), *b2 = malloc(8 * nr), *mb = malloc(8 * nr);
    orc_locate(m, nr, o, 4, start, mb);
    for (int64_t i = 0; i < nr; ++i) entry[i] = -1;
    orc_trace(m, nr, o, d, tm, start, entry, 16 * nt + 64, 4, tri, t, b1, b2, tet, cf, st, fl);
    orc_bruteforce(m, nr, o, d, tm, entry, 4, tri2, t, b1, b2);  /* entry: all -1, nothing excluded */
    int64_t same = 0;
    for (int64_t i = 0; i < nr; ++i) same += tri[i] == tri2[i];
    orc_mesh_destroy(m);
    free(P); free(T); free(C); free(o); free(d); free(tm); free(start); free(tri); free(tri2);
    free(tet); free(cf); free(st); free(fl); free(entry); free(t); free(b1); free(b2); free(mb);
    printf("oracle OK %lld/%lld\n", (long long)same, (long long)nr);
    return 0;
}
"""


def scenes():
    tiny = sg.make_config("tiny")
    yield "tiny", tiny.points, tiny.tets, tiny.tris
    n, seed = 5, 41
    pts, tets = sg.freudenthal_grid(n, 0.2, seed)
    inside = np.random.default_rng(seed).random((n, n, n)) < 0.3
    yield "random", pts, tets, sg.constrained_faces(n, inside)


def dump(tmp, name, **arrays):
    paths = {}
    for k, a in arrays.items():
        p = tmp / f"{name}_{k}.bin"
        np.ascontiguousarray(a).tofile(p)
        paths[k] = str(p)
    return paths


def compile_driver(tmp, name, src, lang, sources, extra):
    path = tmp / f"{name}.{lang}"
    path.write_text(src)
    exe = str(tmp / name)
    cc = "g++" if lang == "cpp" else "gcc"
    std = ["-std=c++17"] if lang == "cpp" else ["-std=c99"]
    cmd = [cc, *std, *SAN, str(path), *sources, "-o", exe, *extra]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-3000:]
    return exe


@pytest.fixture(scope="module")
def tools():
    if shutil.which("gcc") is None or shutil.which("g++") is None:
        pytest.skip("gcc/g++ missing")
    if not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime.h")):
        pytest.skip("CUDA headers missing")


def test_mesh_builder_under_sanitizers(tmp_path, tools):
    exe = compile_driver(
        tmp_path, "build_driver", BUILD_DRIVER, "cpp", [os.path.join(CSRC, "build.cpp")],
        [f"-I{os.path.join(ROOT, 'include')}", f"-I{CSRC}", f"-I{CUDA}/include", "-fopenmp",
         f"-L{CUDA}/lib64", "-lcudart", f"-Wl,-rpath,{CUDA}/lib64"])
    for name, pts, tets, tris in scenes():
        p = dump(tmp_path, name, P=np.asarray(pts, np.float32), T=np.asarray(tets, np.int32),
                 C=np.asarray(tris, np.int32))
        res = subprocess.run([exe, str(len(pts)), str(len(tets)), str(len(tris)), p["P"], p["T"],
                              p["C"]], capture_output=True, text=True, env=dict(ENV, OMP_NUM_THREADS="4"),
                             timeout=300)
        assert res.returncode == 0, (name, res.stdout[-2000:], res.stderr[-4000:])
        assert "build OK 5" in res.stdout        # the bad triangle: TM_ERR_CFACE_UNMATCHED


def test_oracle_under_sanitizers(tmp_path, tools):
    exe = compile_driver(tmp_path, "oracle_driver", ORACLE_DRIVER, "c",
                         [os.path.join(ROOT, "oracle", "oracle.c")],
                         ["-ffp-contract=off", "-lpthread", "-lm"])
    for name, pts, tets, tris in scenes():
        g = np.random.default_rng(7)
        nr = 600
        o = g.uniform(0.05, 0.95, size=(nr, 3)).astype(np.float32)
        d = g.normal(size=(nr, 3))
        d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
        tm = np.where(np.arange(nr) % 3 == 0, np.float32(0.2), np.float32(np.inf)).astype(np.float32)
        p = dump(tmp_path, name, P=np.asarray(pts, np.float32), T=np.asarray(tets, np.int32),
                 C=np.asarray(tris, np.int32), o=o, d=d, tm=tm)
        res = subprocess.run([exe, str(len(pts)), str(len(tets)), str(len(tris)), str(nr), p["P"],
                              p["T"], p["C"], p["o"], p["d"], p["tm"]], capture_output=True,
                             text=True, env=ENV, timeout=300)
        assert res.returncode == 0, (name, res.stdout[-2000:], res.stderr[-4000:])
        # the sanitized build computes what the oracle library computes
        om = oracle.OracleMesh(pts, tets, tris)
        start, _ = om.locate(o)
        w, b = om.trace(o, d, tm, start), om.bruteforce(o, d, tm)
        assert f"oracle OK {int((w['tri'] == b['tri']).sum())}/{nr}" in res.stdout
